// dem_walls.cuh -- distances to the analytic boundaries.
#pragma once
#include "dem_internal.cuh"

namespace dem {

__device__ __forceinline__ double dot3d(const double a[3], const double b[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// Mesh facet, FP64: dd = x - p(t) with p the first vertex.  A facet is
// one-sided: a centre behind its plane (dd.n < 0) does not touch it (+inf).
// In front: inside the face region (barycentric coordinates of the
// projection from the normal equations of the edge vectors all >= 0) the
// distance to the plane; otherwise the distance to the nearest of the edges
// p->b, p->c, b->c (first wins a tie), the foot at the clamped perpendicular
// parameter.
__device__ __forceinline__ double facet_distance64(const WallDev& w, const double dd[3], double nw[3]) {
  const double ax = dot3d(dd, w.n);
  if (ax < 0.0) {
    for (int k = 0; k < 3; ++k) nw[k] = w.n[k];
    return __longlong_as_double(0x7ff0000000000000ll);  // +inf
  }
  const double d00 = dot3d(w.e1, w.e1), d01 = dot3d(w.e1, w.e2), d11 = dot3d(w.e2, w.e2);
  const double b0 = dot3d(dd, w.e1), b1 = dot3d(dd, w.e2);
  const double den = __dsub_rn(__dmul_rn(d00, d11), __dmul_rn(d01, d01));
  const double u = __ddiv_rn(__dsub_rn(__dmul_rn(d11, b0), __dmul_rn(d01, b1)), den);
  const double v = __ddiv_rn(__dsub_rn(__dmul_rn(d00, b1), __dmul_rn(d01, b0)), den);
  if (u >= 0.0 && v >= 0.0 && __dadd_rn(u, v) <= 1.0) {
    for (int k = 0; k < 3; ++k) nw[k] = w.n[k];
    return ax;
  }
  double best = -1.0, qb[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double r[3], e[3], q[3];
    for (int k = 0; k < 3; ++k) {
      r[k] = j == 2 ? __dsub_rn(dd[k], w.e1[k]) : dd[k];
      e[k] = j == 0 ? w.e1[k] : (j == 1 ? w.e2[k] : __dsub_rn(w.e2[k], w.e1[k]));
    }
    double t = __ddiv_rn(dot3d(r, e), dot3d(e, e));
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    for (int k = 0; k < 3; ++k) q[k] = __dsub_rn(r[k], __dmul_rn(t, e[k]));
    const double dist = __dsqrt_rn(dot3d(q, q));
    if (best < 0.0 || dist < best) {
      best = dist;
      for (int k = 0; k < 3; ++k) qb[k] = q[k];
    }
  }
  for (int k = 0; k < 3; ++k) nw[k] = best > 0.0 ? __ddiv_rn(qb[k], best) : w.n[k];
  return best;
}

// Signed distance from x to the wall at time t (positive on the grains' side),
// with exactly the operation order of its definition; nw: unit normal of the
// surface at the closest point, towards the grains.
__device__ __forceinline__ double wall_distance64(const WallDev& w, double t, const double x[3], double nw[3]) {
  double p[3], dd[3];
  for (int k = 0; k < 3; ++k) {
    p[k] = __dadd_rn(w.p[k], __dmul_rn(w.vel[k], t));
    dd[k] = __dsub_rn(x[k], p[k]);
  }
  if (w.type == 0) {
    for (int k = 0; k < 3; ++k) nw[k] = w.n[k];
    return dot3d(dd, w.n);
  }
  if (w.type == 3) return facet_distance64(w, dd, nw);
  const double ax = dot3d(dd, w.n);
  double rv[3];
  for (int k = 0; k < 3; ++k) rv[k] = __dsub_rn(dd[k], __dmul_rn(ax, w.n[k]));
  const double rho = __dsqrt_rn(dot3d(rv, rv));
  if (w.type == 1) {
    if (rho > 0.0) {
      for (int k = 0; k < 3; ++k) nw[k] = __ddiv_rn(-rv[k], rho);
    } else {
      nw[0] = nw[1] = nw[2] = 0.0;
    }
    return __dsub_rn(w.radius, rho);
  }
  const double H = w.height, Rb = w.rb;
  double tl = __ddiv_rn(__dadd_rn(__dmul_rn(rho, Rb), __dmul_rn(ax, H)),
                        __dadd_rn(__dmul_rn(Rb, Rb), __dmul_rn(H, H)));
  tl = tl < 0.0 ? 0.0 : (tl > 1.0 ? 1.0 : tl);
  const double ql0 = __dmul_rn(tl, Rb), ql1 = __dmul_rn(tl, H);
  const double dl = __dsqrt_rn(__dadd_rn(__dmul_rn(__dsub_rn(rho, ql0), __dsub_rn(rho, ql0)),
                                         __dmul_rn(__dsub_rn(ax, ql1), __dsub_rn(ax, ql1))));
  double tb = __ddiv_rn(rho, Rb);
  tb = tb < 0.0 ? 0.0 : (tb > 1.0 ? 1.0 : tb);
  const double qb0 = __dmul_rn(tb, Rb), qb1 = H;
  const double db = __dsqrt_rn(__dadd_rn(__dmul_rn(__dsub_rn(rho, qb0), __dsub_rn(rho, qb0)),
                                         __dmul_rn(__dsub_rn(ax, qb1), __dsub_rn(ax, qb1))));
  const bool inside = (ax >= 0.0 && ax <= H && __dmul_rn(rho, H) <= __dmul_rn(ax, Rb));
  double q0, q1, dm;
  if (dl <= db) { q0 = ql0; q1 = ql1; dm = dl; } else { q0 = qb0; q1 = qb1; dm = db; }
  double n0, n1;
  if (dm > 0.0) {
    n0 = inside ? (q0 - rho) / dm : (rho - q0) / dm;
    n1 = inside ? (q1 - ax) / dm : (ax - q1) / dm;
  } else {
    const double len = sqrt(H * H + Rb * Rb);
    n0 = H / len;
    n1 = -Rb / len;
  }
  double er[3];
  if (rho > 0.0) {
    for (int k = 0; k < 3; ++k) er[k] = rv[k] / rho;
  } else {
    const double e0 = fabs(w.n[0]) < 0.9 ? 1.0 : 0.0, e1 = fabs(w.n[0]) < 0.9 ? 0.0 : 1.0;
    double c0 = -w.n[2] * e1, c1 = w.n[2] * e0, c2 = w.n[0] * e1 - w.n[1] * e0;
    const double cl = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    er[0] = c0 / cl; er[1] = c1 / cl; er[2] = c2 / cl;
  }
  for (int k = 0; k < 3; ++k) nw[k] = n0 * er[k] + n1 * w.n[k];
  return inside ? -dm : dm;
}


// Contact geometry of a sphere centre (fixed point, 2^-44 m) with a wall whose
// reference point at the current time is wf (same fixed-point frame), in
// float-float so that delta_n = r - distance keeps its relative accuracy.
// Returns delta_n (float, metres) and the unit normal n from the sphere
// towards the wall.
__device__ __forceinline__ float wall_geom32(const WallDev& w, const long long wf[3], long long x,
                                             long long y, long long z, float r, V3<float>& n) {
  const ff d[3] = {fix_to_ff(x - wf[0]), fix_to_ff(y - wf[1]), fix_to_ff(z - wf[2])};
  const ff a[3] = {{w.nh[0], w.nl[0]}, {w.nh[1], w.nl[1]}, {w.nh[2], w.nl[2]}};
  const ff ax = ff_add(ff_add(ff_mul(d[0], a[0]), ff_mul(d[1], a[1])), ff_mul(d[2], a[2]));
  V3<float> nw;
  ff dist;
  if (w.type == 0) {
    dist = ax;
    nw = {w.nh[0], w.nh[1], w.nh[2]};
  } else if (w.type == 3) {
    // mesh facet: one-sided (a centre behind its plane does not touch it);
    // in front the region is classified in float (the distance is
    // continuous across the regions' borders there), the distance in
    // float-float
    if (ax.h < 0.f || (ax.h == 0.f && ax.l < 0.f)) {
      n = {-w.nh[0], -w.nh[1], -w.nh[2]};
      return -1.f;
    }
    const V3<float> df = {d[0].h, d[1].h, d[2].h};
    const V3<float> e1 = {w.e1h[0], w.e1h[1], w.e1h[2]}, e2 = {w.e2h[0], w.e2h[1], w.e2h[2]};
    const float d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2);
    const float b0 = dot(df, e1), b1 = dot(df, e2);
    const float den = d00 * d11 - d01 * d01;
    const float u = (d11 * b0 - d01 * b1) / den, v = (d00 * b1 - d01 * b0) / den;
    if (u >= 0.f && v >= 0.f && u + v <= 1.f) {
      dist = ax;
      nw = {w.nh[0], w.nh[1], w.nh[2]};
    } else {
      const ff E1[3] = {{w.e1h[0], w.e1l[0]}, {w.e1h[1], w.e1l[1]}, {w.e1h[2], w.e1l[2]}};
      const ff E2[3] = {{w.e2h[0], w.e2l[0]}, {w.e2h[1], w.e2l[1]}, {w.e2h[2], w.e2l[2]}};
      ff best = {-1.f, 0.f};
      V3<float> qb = {0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        ff r[3], e[3];
        for (int k = 0; k < 3; ++k) {
          r[k] = j == 2 ? ff_sub(d[k], E1[k]) : d[k];
          e[k] = j == 0 ? E1[k] : (j == 1 ? E2[k] : ff_sub(E2[k], E1[k]));
        }
        const V3<float> rh = {r[0].h, r[1].h, r[2].h}, eh = {e[0].h, e[1].h, e[2].h};
        const float t = fminf(fmaxf(dot(rh, eh) / dot(eh, eh), 0.f), 1.f);
        const ff q[3] = {ff_sub(r[0], ff_mulf(e[0], t)), ff_sub(r[1], ff_mulf(e[1], t)),
                         ff_sub(r[2], ff_mulf(e[2], t))};
        const ff dq = ff_sqrt(ff_add(ff_add(ff_mul(q[0], q[0]), ff_mul(q[1], q[1])), ff_mul(q[2], q[2])));
        if (best.h < 0.f || dq.h < best.h) {
          best = dq;
          qb = {q[0].h, q[1].h, q[2].h};
        }
      }
      dist = best;
      nw = best.h > 0.f ? (1.f / best.h) * qb : V3<float>{w.nh[0], w.nh[1], w.nh[2]};
    }
  } else {
    const ff rv[3] = {ff_sub(d[0], ff_mul(ax, a[0])), ff_sub(d[1], ff_mul(ax, a[1])),
                      ff_sub(d[2], ff_mul(ax, a[2]))};
    const ff rho = ff_sqrt(ff_add(ff_add(ff_mul(rv[0], rv[0]), ff_mul(rv[1], rv[1])),
                                  ff_mul(rv[2], rv[2])));
    V3<float> er;
    if (rho.h > 0.f) {
      er = {rv[0].h / rho.h, rv[1].h / rho.h, rv[2].h / rho.h};
    } else {
      const float e0 = fabsf(a[0].h) < 0.9f ? 1.f : 0.f, e1 = 1.f - e0;
      V3<float> c = {-a[2].h * e1, a[2].h * e0, a[0].h * e1 - a[1].h * e0};
      const float cl = sqrtf(dot(c, c));
      er = {c.x / cl, c.y / cl, c.z / cl};
    }
    const V3<float> av = {a[0].h, a[1].h, a[2].h};
    if (w.type == 1) {
      dist = ff_sub({w.rh, w.rl}, rho);
      nw = -1.f * er;
    } else {
      // cone: meridian half plane (rho, ax); tip (0,0), rim (Rb,H), base centre (0,H)
      const float rf = ff_to_float(rho), af = ff_to_float(ax);
      const float H = w.hh, Rb = w.rbh;
      float tl = (rf * Rb + af * H) / (Rb * Rb + H * H);
      tl = fminf(fmaxf(tl, 0.f), 1.f);
      const float dl = sqrtf((rf - tl * Rb) * (rf - tl * Rb) + (af - tl * H) * (af - tl * H));
      float tb = fminf(fmaxf(rf / Rb, 0.f), 1.f);
      const float db = sqrtf((rf - tb * Rb) * (rf - tb * Rb) + (af - H) * (af - H));
      const bool inside = (af >= 0.f && af <= H && rf * H <= af * Rb);
      float n0, n1;
      if (inside) {
        // centre inside the solid: deep contact, float accuracy is enough
        const float q0 = dl <= db ? tl * Rb : tb * Rb, q1 = dl <= db ? tl * H : H;
        const float dm = fmaxf(fminf(dl, db), 1e-30f);
        dist = {-fminf(dl, db), 0.f};
        n0 = (q0 - rf) / dm;
        n1 = (q1 - af) / dm;
      } else if (dl <= db && tl > 0.f && tl < 1.f) {
        // lateral surface: signed distance to its line, rho cos - ax sin
        dist = ff_sub(ff_mul(rho, {w.ch, w.cl}), ff_mul(ax, {w.sh, w.sl}));
        n0 = w.ch;
        n1 = -w.sh;
      } else if (dl > db && tb < 1.f) {
        dist = ff_sub(ax, {w.hh, w.hl});  // base disk
        n0 = 0.f;
        n1 = 1.f;
      } else {
        // a vertex: the tip or the rim circle
        const bool tip = (dl <= db) && !(tl > 0.f);
        const ff e0 = tip ? rho : ff_sub(rho, {w.rbh, w.rbl});
        const ff e1 = tip ? ax : ff_sub(ax, {w.hh, w.hl});
        dist = ff_sqrt(ff_add(ff_mul(e0, e0), ff_mul(e1, e1)));
        const float dm = fmaxf(dist.h, 1e-30f);
        n0 = e0.h / dm;
        n1 = e1.h / dm;
      }
      nw = n0 * er + n1 * av;
    }
  }
  n = -1.f * nw;
  return ff_to_float(ff_sub({r, 0.f}, dist));
}

}  // namespace dem
