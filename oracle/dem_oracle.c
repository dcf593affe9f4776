/*
 * dem_oracle.c -- plain FP64 CPU oracle for the clump-of-spheres DEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Written from the
 * paper (arXiv 2307.03445) independently of the CUDA library; nothing is shared.
 *
 * Compile with -ffp-contract=off: the detection coordinates are integers
 * decided by floating point, and they are defined by the exact sequence of
 * IEEE double operations written below (one rounding per operation).
 *
 * Readings of points the paper leaves open (listed with the same letters in
 * the design notes):
 *   A1  k_n = 4/3 E*, k_t = 8 G*; the damping terms f*gamma*m are
 *       -2 sqrt(5/6) beta sqrt(S m) with S_n = 2 E* f, S_t = 8 G* f and
 *       beta = ln(e) / sqrt(ln(e)^2 + pi^2); no clipping of a tensile F_n.
 *   A2  1/E* = sum (1 - nu^2)/E, 1/G* = sum 2 (2 - nu)(1 + nu)/E; mu and CoR
 *       mixed by mean (default), min or max.
 *   A3  n points from sphere a to sphere b; F acts on b, -F on a.
 *   A4  torque is the moment of the whole contact force about the owner CoM.
 *   A5  contact point = x_a + (r_a - delta_n / 2) n.
 *   A6  the cap rescales F_t to mu |F_n| and stores u_t with f k_t |u_t| = mu |F_n|.
 *   A7  u_t is reset when a listed contact has delta_n <= 0.
 *   A9  semi-implicit Euler for v and X; body-frame Euler equations for omega;
 *       q <- normalise(q * exp(h omega_body / 2)).
 *   A11 multi-bin registration of the enlarged AABB, pair reported by the bin
 *       holding the per-axis max of the two lower corners; exact int64 test.
 *   A15 sphere-wall contacts: R = r_sphere, m = m_clump, wall material given.
 *   B1 mesh facets (section 4 funnel, cone and wheel meshes): distance to
 *       the closed triangle; the signed plane distance where the centre
 *       projects inside it, else the unsigned distance to the nearest edge;
 *       every sphere-facet pair is its own contact.
 */
#include "dem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Rotation of p by the unit quaternion q = (w, x, y, z), written as the
 * rotation matrix with this exact operation order (the detection lattice is
 * defined by it). */
static void rotate(const double q[4], const double p[3], double out[3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double xx = x * x, yy = y * y, zz = z * z;
    const double xy = x * y, xz = x * z, yz = y * z;
    const double wx = w * x, wy = w * y, wz = w * z;
    const double r00 = 1.0 - 2.0 * (yy + zz), r01 = 2.0 * (xy - wz), r02 = 2.0 * (xz + wy);
    const double r10 = 2.0 * (xy + wz), r11 = 1.0 - 2.0 * (xx + zz), r12 = 2.0 * (yz - wx);
    const double r20 = 2.0 * (xz - wy), r21 = 2.0 * (yz + wx), r22 = 1.0 - 2.0 * (xx + yy);
    out[0] = (r00 * p[0] + r01 * p[1]) + r02 * p[2];
    out[1] = (r10 * p[0] + r11 * p[1]) + r12 * p[2];
    out[2] = (r20 * p[0] + r21 * p[1]) + r22 * p[2];
}
/* Transpose rotation (world -> body). */
static void rotate_t(const double q[4], const double p[3], double out[3]) {
    const double qc[4] = {q[0], -q[1], -q[2], -q[3]};
    rotate(qc, p, out);
}
static void qmul(const double a[4], const double b[4], double c[4]) {
    c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static long long floordiv(long long a, long long b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}
static long long clampll(long long v, long long lo, long long hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* ------------------------------------------------------------------ */
/* sphere centres (section 2.1: a clump is a rigid union of spheres)    */
/* ------------------------------------------------------------------ */
long long orc_num_spheres(const orc_model* m, int n, const int* tpl) {
    long long ns = 0;
    for (int c = 0; c < n; ++c) ns += m->tpl_off[tpl[c] + 1] - m->tpl_off[tpl[c]];
    return ns;
}

void orc_sphere_centres(const orc_model* m, int n, const int* tpl, const double* pos,
                        const double* quat, double* xs, int* owner, int* tsph) {
    long long s = 0;
    for (int c = 0; c < n; ++c) {
        for (int j = m->tpl_off[tpl[c]]; j < m->tpl_off[tpl[c] + 1]; ++j, ++s) {
            double rp[3];
            rotate(quat + 4 * c, m->tpl_pos + 3 * j, rp);
            for (int k = 0; k < 3; ++k) xs[3 * s + k] = pos[3 * c + k] + rp[k];
            if (owner) owner[s] = c;
            if (tsph) tsph[s] = j;
        }
    }
}

/* ------------------------------------------------------------------ */
/* detection lattice (section 2.2: enlarged geometry, binning)          */
/* ------------------------------------------------------------------ */
void orc_detect_coords(const orc_model* m, long long ns, const double* xs, const int* tsph,
                       const double* margin, long long* qc, long long* rho) {
    const double scale = 16777216.0; /* 2^ORC_EPS_LOG2 */
    for (long long s = 0; s < ns; ++s) {
        for (int k = 0; k < 3; ++k) qc[3 * s + k] = llrint((xs[3 * s + k] - m->lo[k]) * scale);
        /* enlarged radius in lattice units, plus one unit covering the rounding
           of both centres: a touching pair always passes the test */
        double r = m->tpl_rad[tsph[s]] + margin[s];
        rho[s] = (long long)ceil(r * scale) + 1;
    }
}

void orc_grid_dims(const orc_model* m, long long dims[3], long long* bin_edge) {
    const double scale = 16777216.0;
    long long L = (long long)ceil(m->bin_size * scale);
    if (L < 1) L = 1;
    for (int k = 0; k < 3; ++k) {
        long long ext = llrint((m->hi[k] - m->lo[k]) * scale);
        long long d = (ext + L - 1) / L;
        dims[k] = d < 1 ? 1 : d;
    }
    *bin_edge = L;
}

static void bin_range(const long long dims[3], long long L, const long long* q, long long r,
                      long long lo[3], long long hi[3]) {
    for (int k = 0; k < 3; ++k) {
        lo[k] = clampll(floordiv(q[k] - r, L), 0, dims[k] - 1);
        hi[k] = clampll(floordiv(q[k] + r, L), 0, dims[k] - 1);
    }
}

typedef struct { unsigned int key; int id; } kv_t;
static int kv_cmp(const void* x, const void* y) {
    const kv_t* a = (const kv_t*)x;
    const kv_t* b = (const kv_t*)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Every (bin, sphere) registration of the enlarged AABBs, sorted by bin key
 * then sphere id.  Returns the total (entries beyond cap are not written). */
long long orc_bin_entries(const orc_model* m, long long ns, const long long* qc,
                          const long long* rho, long long cap, unsigned int* keys, int* ids) {
    long long dims[3], L;
    orc_grid_dims(m, dims, &L);
    long long total = 0;
    for (long long s = 0; s < ns; ++s) {
        long long lo[3], hi[3];
        bin_range(dims, L, qc + 3 * s, rho[s], lo, hi);
        total += (hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    }
    kv_t* e = (kv_t*)malloc(sizeof(kv_t) * (size_t)(total > 0 ? total : 1));
    long long k = 0;
    for (long long s = 0; s < ns; ++s) {
        long long lo[3], hi[3];
        bin_range(dims, L, qc + 3 * s, rho[s], lo, hi);
        for (long long z = lo[2]; z <= hi[2]; ++z)
            for (long long y = lo[1]; y <= hi[1]; ++y)
                for (long long x = lo[0]; x <= hi[0]; ++x) {
                    e[k].key = (unsigned int)((z * dims[1] + y) * dims[0] + x);
                    e[k].id = (int)s;
                    ++k;
                }
    }
    qsort(e, (size_t)total, sizeof(kv_t), kv_cmp);
    for (long long i = 0; i < total && i < cap; ++i) {
        keys[i] = e[i].key;
        ids[i] = e[i].id;
    }
    free(e);
    return total;
}

/* The exact contact-candidate predicate on the lattice: the enlarged spheres
 * of two different clumps overlap or touch. */
static int near_pair(const long long* qa, long long ra, const long long* qb, long long rb) {
    long long dx = qb[0] - qa[0], dy = qb[1] - qa[1], dz = qb[2] - qa[2];
    long long rr = ra + rb;
    return dx * dx + dy * dy + dz * dz <= rr * rr;
}

long long orc_pairs_brute(long long ns, const int* owner, const long long* qc,
                          const long long* rho, long long cap, int* a, int* b) {
    long long n = 0;
    for (long long i = 0; i < ns; ++i)
        for (long long j = i + 1; j < ns; ++j) {
            if (owner[i] == owner[j]) continue;
            if (!near_pair(qc + 3 * i, rho[i], qc + 3 * j, rho[j])) continue;
            if (n < cap) { a[n] = (int)i; b[n] = (int)j; }
            ++n;
        }
    return n;
}

typedef struct { int a, b; } pair_t;
static int pair_cmp(const void* x, const void* y) {
    const pair_t* p = (const pair_t*)x;
    const pair_t* q = (const pair_t*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    return (p->b > q->b) - (p->b < q->b);
}

/* Bin-by-bin narrow phase: within each bin, every pair of registered spheres
 * of different clumps passing the predicate, kept only in the bin that holds
 * the per-axis max of the two AABB lower corners.  Sorted by (a, b). */
long long orc_pairs_binned(const orc_model* m, long long ns, const int* owner,
                           const long long* qc, const long long* rho, long long cap,
                           int* a, int* b) {
    long long dims[3], L;
    orc_grid_dims(m, dims, &L);
    long long ne = orc_bin_entries(m, ns, qc, rho, 0, NULL, NULL);
    unsigned int* keys = (unsigned int*)malloc(sizeof(unsigned int) * (size_t)(ne + 1));
    int* ids = (int*)malloc(sizeof(int) * (size_t)(ne + 1));
    orc_bin_entries(m, ns, qc, rho, ne, keys, ids);
    size_t pcap = 1024;
    long long np = 0;
    pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * pcap);
    long long i0 = 0;
    while (i0 < ne) {
        long long i1 = i0;
        while (i1 < ne && keys[i1] == keys[i0]) ++i1;
        const long long key = keys[i0];
        for (long long i = i0; i < i1; ++i)
            for (long long j = i + 1; j < i1; ++j) {
                const int s = ids[i], t = ids[j];
                if (owner[s] == owner[t]) continue;
                if (!near_pair(qc + 3 * (long long)s, rho[s], qc + 3 * (long long)t, rho[t])) continue;
                long long ob[3];
                for (int k = 0; k < 3; ++k) {
                    long long la = qc[3 * (long long)s + k] - rho[s];
                    long long lb = qc[3 * (long long)t + k] - rho[t];
                    ob[k] = clampll(floordiv(la > lb ? la : lb, L), 0, dims[k] - 1);
                }
                if ((ob[2] * dims[1] + ob[1]) * dims[0] + ob[0] != key) continue;
                if ((size_t)np == pcap) {
                    pcap *= 2;
                    pr = (pair_t*)realloc(pr, sizeof(pair_t) * pcap);
                }
                pr[np].a = s < t ? s : t;
                pr[np].b = s < t ? t : s;
                ++np;
            }
        i0 = i1;
    }
    qsort(pr, (size_t)np, sizeof(pair_t), pair_cmp);
    for (long long i = 0; i < np && i < cap; ++i) { a[i] = pr[i].a; b[i] = pr[i].b; }
    free(pr);
    free(keys);
    free(ids);
    return np;
}

/* ------------------------------------------------------------------ */
/* analytic boundaries                                                  */
/* ------------------------------------------------------------------ */
/* Mesh facet with vertices p, b, c (translating rigidly, so the edge
 * vectors e1 = b - p, e2 = c - p do not depend on time) and d = x - p(t).
 * A facet is one-sided (reading B1): a centre behind its plane (d.n < 0)
 * does not touch it, whatever its distance; the result is +infinity, which
 * no candidate threshold reaches and which gives no overlap.  (Without this a
 * sphere on the far side of a convex mesh, behind a far facet and inside that
 * facet's prism, would be in deep contact with it.)  In front (d.n >= 0):
 * barycentric coordinates (u, v) of the projection of x on the facet's plane
 * solve the normal equations [e1.e1 e1.e2; e1.e2 e2.e2] (u, v) = (d.e1, d.e2).
 * Inside the facet (u, v >= 0, u + v <= 1) the closest point is the
 * projection: distance d.n, normal n.  Outside it the closest point of the
 * closed triangle lies on its boundary: the nearest of the three edges
 * (p -> b, p -> c, b -> c), each the segment point at the clamped parameter
 * of the perpendicular foot; normal from that point to x.  The distance is
 * continuous across the regions' borders on the front side. */
static double facet_distance(const orc_wall* w, const double d[3], double nw[3]) {
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = w->b[k] - w->p[k];
        e2[k] = w->c[k] - w->p[k];
    }
    const double ax = dot3(d, w->n);
    if (ax < 0.0) {
        for (int k = 0; k < 3; ++k) nw[k] = w->n[k];
        return HUGE_VAL;
    }
    const double d00 = dot3(e1, e1), d01 = dot3(e1, e2), d11 = dot3(e2, e2);
    const double b0 = dot3(d, e1), b1 = dot3(d, e2);
    const double den = d00 * d11 - d01 * d01;
    const double u = (d11 * b0 - d01 * b1) / den;
    const double v = (d00 * b1 - d01 * b0) / den;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
        for (int k = 0; k < 3; ++k) nw[k] = w->n[k];
        return ax;
    }
    const double zero[3] = {0.0, 0.0, 0.0};
    double e3[3];
    for (int k = 0; k < 3; ++k) e3[k] = e2[k] - e1[k];
    const double* org[3] = {zero, zero, e1};
    const double* dir[3] = {e1, e2, e3};
    double best = -1.0, qb[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < 3; ++j) {
        double r[3], q[3];
        for (int k = 0; k < 3; ++k) r[k] = d[k] - org[j][k];
        double t = dot3(r, dir[j]) / dot3(dir[j], dir[j]);
        t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
        for (int k = 0; k < 3; ++k) q[k] = r[k] - t * dir[j][k];
        const double dist = sqrt(dot3(q, q));
        if (best < 0.0 || dist < best) {
            best = dist;
            for (int k = 0; k < 3; ++k) qb[k] = q[k];
        }
    }
    for (int k = 0; k < 3; ++k) nw[k] = best > 0.0 ? qb[k] / best : w->n[k];
    return best;
}

/* Signed distance from x to the wall surface at time t (positive on the
 * grains' side) and the unit normal nw of the surface at the closest point,
 * pointing towards the grains. */
double orc_wall_distance(const orc_wall* w, double t, const double x[3], double nw[3]) {
    double p[3], d[3];
    for (int k = 0; k < 3; ++k) {
        p[k] = w->p[k] + w->vel[k] * t;
        d[k] = x[k] - p[k];
    }
    if (w->type == ORC_WALL_PLANE) {
        for (int k = 0; k < 3; ++k) nw[k] = w->n[k];
        return dot3(d, w->n);
    }
    if (w->type == ORC_WALL_TRIANGLE) return facet_distance(w, d, nw);
    const double ax = dot3(d, w->n);
    double rv[3];
    for (int k = 0; k < 3; ++k) rv[k] = d[k] - ax * w->n[k];
    const double rho = sqrt(dot3(rv, rv));
    if (w->type == ORC_WALL_CYLINDER) {
        if (rho > 0.0) {
            for (int k = 0; k < 3; ++k) nw[k] = -rv[k] / rho;
        } else {
            nw[0] = nw[1] = nw[2] = 0.0;
        }
        return w->radius - rho;
    }
    /* solid cone: in the meridian half plane (rho, ax) the section is the
       triangle tip (0,0), rim (Rb,H), base centre (0,H); its boundary seen from
       rho >= 0 is the lateral segment and the base segment. */
    const double H = w->height;
    const double Rb = H * tan(w->half_angle);
    double tl = (rho * Rb + ax * H) / (Rb * Rb + H * H);
    tl = tl < 0.0 ? 0.0 : (tl > 1.0 ? 1.0 : tl);
    const double ql0 = tl * Rb, ql1 = tl * H;
    const double dl = sqrt((rho - ql0) * (rho - ql0) + (ax - ql1) * (ax - ql1));
    double tb = rho / Rb;
    tb = tb < 0.0 ? 0.0 : (tb > 1.0 ? 1.0 : tb);
    const double qb0 = tb * Rb, qb1 = H;
    const double db = sqrt((rho - qb0) * (rho - qb0) + (ax - qb1) * (ax - qb1));
    const int inside = (ax >= 0.0 && ax <= H && rho * H <= ax * Rb);
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
        /* on the axis the radial direction is arbitrary; pick one normal to the axis */
        const double e[3] = {fabs(w->n[0]) < 0.9 ? 1.0 : 0.0, fabs(w->n[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        double c[3];
        cross3(w->n, e, c);
        const double cl = sqrt(dot3(c, c));
        for (int k = 0; k < 3; ++k) er[k] = c[k] / cl;
    }
    for (int k = 0; k < 3; ++k) nw[k] = n0 * er[k] + n1 * w->n[k];
    return inside ? -dm : dm;
}

long long orc_wall_candidates(const orc_model* m, long long ns, const double* xs,
                              const int* tsph, const double* margin, double t,
                              double wall_travel_time, long long cap, int* s, int* w) {
    long long n = 0;
    for (long long i = 0; i < ns; ++i)
        for (int k = 0; k < m->n_walls; ++k) {
            const orc_wall* wl = m->walls + k;
            double nw[3];
            const double dist = orc_wall_distance(wl, t, xs + 3 * i, nw);
            const double travel = sqrt(dot3(wl->vel, wl->vel)) * wall_travel_time;
            if (dist <= m->tpl_rad[tsph[i]] + margin[i] + travel) {
                if (n < cap) { s[n] = (int)i; w[n] = k; }
                ++n;
            }
        }
    return n;
}

/* ------------------------------------------------------------------ */
/* contact law                                                          */
/* ------------------------------------------------------------------ */
void orc_pair_material(const orc_model* m, int ia, int ib, double* Estar, double* Gstar,
                       double* mu, double* cor) {
    const double Ea = m->E[ia], Eb = m->E[ib], na = m->nu[ia], nb = m->nu[ib];
    *Estar = 1.0 / ((1.0 - na * na) / Ea + (1.0 - nb * nb) / Eb);
    *Gstar = 1.0 / (2.0 * (2.0 - na) * (1.0 + na) / Ea + 2.0 * (2.0 - nb) * (1.0 + nb) / Eb);
    const double ma = m->mu[ia], mb = m->mu[ib], ca = m->cor[ia], cb = m->cor[ib];
    switch (m->mix_rule) {
        case ORC_MIX_MIN: *mu = ma < mb ? ma : mb; *cor = ca < cb ? ca : cb; break;
        case ORC_MIX_MAX: *mu = ma > mb ? ma : mb; *cor = ca > cb ? ca : cb; break;
        default: *mu = 0.5 * (ma + mb); *cor = 0.5 * (ca + cb); break;
    }
}

int orc_contact(const orc_model* m, int mat_a, int mat_b, const double xa[3],
                const double xb[3], const double Xa[3], const double Xb[3],
                const double va[3], const double wa[3], const double vb[3],
                const double wb[3], double ra, double rb, double ma, double mb,
                const double n_wall[3], double delta_wall, double u[3], double F[3],
                double ca[3], double cb[3]) {
    const int wall = !(mb > 0.0);
    double n[3], dn;
    if (!wall) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = xb[k] - xa[k];
        const double dist = sqrt(dot3(d, d));
        dn = (ra + rb) - dist;
        if (dn > 0.0)
            for (int k = 0; k < 3; ++k) n[k] = d[k] / dist;
    } else {
        dn = delta_wall;
        for (int k = 0; k < 3; ++k) n[k] = n_wall[k];
    }
    if (!(dn > 0.0)) {
        /* false positive of the enlarged list (section 2.2): no force; A7 */
        for (int k = 0; k < 3; ++k) { F[k] = 0.0; u[k] = 0.0; ca[k] = 0.0; cb[k] = 0.0; }
        return 0;
    }
    /* A5: contact point and the lever arms r_i, r_j of Eq. (2a) */
    const double sa = ra - 0.5 * dn;
    for (int k = 0; k < 3; ++k) {
        const double c = xa[k] + sa * n[k];
        ca[k] = c - Xa[k];
        cb[k] = wall ? 0.0 : c - Xb[k];
    }
    /* Eq. (2a)-(2c) */
    double pa[3], pb[3], vrel[3], vn[3], vt[3];
    cross3(wa, ca, pa);
    if (wall) { pb[0] = pb[1] = pb[2] = 0.0; } else { cross3(wb, cb, pb); }
    for (int k = 0; k < 3; ++k) vrel[k] = (vb[k] + pb[k]) - (va[k] + pa[k]);
    const double vns = dot3(vrel, n);
    for (int k = 0; k < 3; ++k) { vn[k] = vns * n[k]; vt[k] = vrel[k] - vn[k]; }
    /* Eq. (3) */
    double up[3], upt[3];
    for (int k = 0; k < 3; ++k) up[k] = u[k] + m->h * vt[k];
    const double upn = dot3(up, n);
    for (int k = 0; k < 3; ++k) upt[k] = up[k] - upn * n[k];
    /* Eq. (1c)-(1e) */
    const double Rbar = wall ? ra : ra * rb / (ra + rb);
    const double mbar = wall ? ma : ma * mb / (ma + mb);
    const double f = sqrt(Rbar * dn);
    double Es, Gs, mu, e;
    orc_pair_material(m, mat_a, mat_b, &Es, &Gs, &mu, &e);
    double beta;
    if (e >= 1.0) beta = 0.0;
    else if (e <= 0.0) beta = -1.0;
    else { const double le = log(e); beta = le / sqrt(le * le + PI_D * PI_D); }
    const double kn = 4.0 / 3.0 * Es, kt = 8.0 * Gs;
    const double Dn = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(2.0 * Es * f * mbar);
    const double Dt = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(8.0 * Gs * f * mbar);
    /* Eq. (1a), (1b) */
    double Fn[3], Ft[3];
    for (int k = 0; k < 3; ++k) {
        Fn[k] = f * kn * dn * n[k] - Dn * vn[k];
        Ft[k] = -f * kt * upt[k] - Dt * vt[k];
    }
    /* Eq. (4) with A6 */
    const double fn = sqrt(dot3(Fn, Fn)), ft = sqrt(dot3(Ft, Ft));
    if (ft > mu * fn) {
        const double s = ft > 0.0 ? mu * fn / ft : 0.0;
        for (int k = 0; k < 3; ++k) Ft[k] *= s;
        const double ul = sqrt(dot3(upt, upt));
        const double us = ul > 0.0 ? mu * fn / (f * kt) / ul : 0.0;
        for (int k = 0; k < 3; ++k) u[k] = us * upt[k];
    } else {
        for (int k = 0; k < 3; ++k) u[k] = upt[k];
    }
    for (int k = 0; k < 3; ++k) F[k] = Fn[k] + Ft[k];
    return 1;
}

long long orc_forces(const orc_model* m, int n, const int* tpl, const double* pos,
                     const double* quat, const double* vel, const double* angvel,
                     double t, long long np, const int* pa, const int* pb, double* up,
                     long long nw, const int* ws, const int* ww, double* uw, double* F,
                     double* T, double* Fw, double* Tw, double* mag) {
    const long long ns = orc_num_spheres(m, n, tpl);
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(ns + 1));
    int* owner = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    int* tsph = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    orc_sphere_centres(m, n, tpl, pos, quat, xs, owner, tsph);
    for (long long i = 0; i < 3LL * n; ++i) { F[i] = 0.0; T[i] = 0.0; }
    if (Fw) for (int i = 0; i < 3 * m->n_walls; ++i) Fw[i] = 0.0;
    if (Tw) for (int i = 0; i < 3 * m->n_walls; ++i) Tw[i] = 0.0;
    if (mag) for (long long i = 0; i < 2LL * n; ++i) mag[i] = 0.0;
    long long active = 0;
    for (long long c = 0; c < np; ++c) {
        const int a = pa[c], b = pb[c];
        const int A = owner[a], B = owner[b];
        const int ja = tsph[a], jb = tsph[b];
        double f[3], ca[3], cb[3];
        active += orc_contact(m, m->tpl_mat[ja], m->tpl_mat[jb], xs + 3 * (long long)a,
                              xs + 3 * (long long)b, pos + 3 * A, pos + 3 * B, vel + 3 * A,
                              angvel + 3 * A, vel + 3 * B, angvel + 3 * B, m->tpl_rad[ja],
                              m->tpl_rad[jb], m->tpl_mass[tpl[A]], m->tpl_mass[tpl[B]], NULL,
                              0.0, up + 3 * c, f, ca, cb);
        double tq[3], mf[3] = {-f[0], -f[1], -f[2]};
        for (int k = 0; k < 3; ++k) { F[3 * B + k] += f[k]; F[3 * A + k] -= f[k]; }
        const double fl = sqrt(dot3(f, f));
        cross3(cb, f, tq);
        for (int k = 0; k < 3; ++k) T[3 * B + k] += tq[k];
        if (mag) { mag[2 * B] += fl; mag[2 * B + 1] += sqrt(dot3(cb, cb)) * fl; }
        cross3(ca, mf, tq);
        for (int k = 0; k < 3; ++k) T[3 * A + k] += tq[k];
        if (mag) { mag[2 * A] += fl; mag[2 * A + 1] += sqrt(dot3(ca, ca)) * fl; }
    }
    for (long long c = 0; c < nw; ++c) {
        const int s = ws[c], k0 = ww[c];
        const int A = owner[s], js = tsph[s];
        const orc_wall* wl = m->walls + k0;
        double nwv[3], nrm[3], f[3], ca[3], cb[3], zero[3] = {0.0, 0.0, 0.0};
        const double dist = orc_wall_distance(wl, t, xs + 3 * (long long)s, nwv);
        for (int k = 0; k < 3; ++k) nrm[k] = -nwv[k];
        const double rs = m->tpl_rad[js];
        active += orc_contact(m, m->tpl_mat[js], wl->material, xs + 3 * (long long)s, NULL,
                              pos + 3 * A, NULL, vel + 3 * A, angvel + 3 * A, wl->vel, zero,
                              rs, 0.0, m->tpl_mass[tpl[A]], 0.0, nrm, rs - dist, uw + 3 * c, f,
                              ca, cb);
        double tq[3], mf[3] = {-f[0], -f[1], -f[2]};
        for (int k = 0; k < 3; ++k) F[3 * A + k] -= f[k];
        cross3(ca, mf, tq);
        for (int k = 0; k < 3; ++k) T[3 * A + k] += tq[k];
        if (mag) {
            mag[2 * A] += sqrt(dot3(f, f));
            mag[2 * A + 1] += sqrt(dot3(ca, ca)) * sqrt(dot3(f, f));
        }
        if (Fw) for (int k = 0; k < 3; ++k) Fw[3 * k0 + k] += f[k];
        if (Tw) {
            /* moment of f about the wall's reference point at time t */
            double arm[3], tw[3];
            for (int k = 0; k < 3; ++k)
                arm[k] = (pos[3 * A + k] + ca[k]) - (wl->p[k] + wl->vel[k] * t);
            cross3(arm, f, tw);
            for (int k = 0; k < 3; ++k) Tw[3 * k0 + k] += tw[k];
        }
    }
    free(xs);
    free(owner);
    free(tsph);
    return active;
}

/* ------------------------------------------------------------------ */
/* equations of motion, Eq. (5a), (5b) with A4, A9                      */
/* ------------------------------------------------------------------ */
void orc_integrate(const orc_model* m, int n, const int* tpl, double* pos, double* quat,
                   double* vel, double* angvel, const double* F, const double* T) {
    const double h = m->h;
    for (int c = 0; c < n; ++c) {
        const double mass = m->tpl_mass[tpl[c]];
        const double* I = m->tpl_inertia + 3 * tpl[c];
        double* q = quat + 4 * c;
        /* Eq. (5a): m dv/dt = m g + sum F */
        for (int k = 0; k < 3; ++k) {
            vel[3 * c + k] += h * (F[3 * c + k] / mass + m->g[k]);
            pos[3 * c + k] += h * vel[3 * c + k];
        }
        /* Eq. (5b) in the principal body frame, with the gyroscopic term */
        double wb[3], tb[3], Iw[3], gy[3];
        rotate_t(q, angvel + 3 * c, wb);
        rotate_t(q, T + 3 * c, tb);
        for (int k = 0; k < 3; ++k) Iw[k] = I[k] * wb[k];
        cross3(wb, Iw, gy);
        for (int k = 0; k < 3; ++k) wb[k] += h * (tb[k] - gy[k]) / I[k];
        /* orientation: q <- q * exp(h wb / 2), renormalised */
        const double wl = sqrt(dot3(wb, wb));
        double dq[4] = {1.0, 0.0, 0.0, 0.0};
        if (wl > 0.0) {
            const double th = 0.5 * h * wl;
            const double sc = sin(th) / wl;
            dq[0] = cos(th);
            for (int k = 0; k < 3; ++k) dq[k + 1] = sc * wb[k];
        }
        double qn[4];
        qmul(q, dq, qn);
        const double ql = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int k = 0; k < 4; ++k) q[k] = qn[k] / ql;
        rotate(q, wb, angvel + 3 * c);
    }
}

/* ------------------------------------------------------------------ */
/* simulation driver: list rebuilt every K steps (section 2.2)          */
/* ------------------------------------------------------------------ */
struct orc_sim {
    orc_model m;
    int n;
    int* tpl;
    double *pos, *quat, *vel, *angvel, *F, *T;
    long long ns;
    double* margin;
    double margin_value;
    int every;
    long long step;
    int since;
    long long np, nw, active;
    int *pa, *pb, *ws, *ww;
    double *up, *uw;
};

static void* dup(const void* p, size_t bytes) {
    void* q = malloc(bytes ? bytes : 1);
    if (bytes) memcpy(q, p, bytes);
    return q;
}

orc_sim* orc_sim_create(const orc_model* m, int n, const int* tpl, const double* pos,
                        const double* quat, const double* vel, const double* angvel,
                        double margin, int rebuild_every) {
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->m = *m; /* the caller keeps the model arrays alive */
    s->n = n;
    s->tpl = (int*)dup(tpl, sizeof(int) * (size_t)n);
    s->pos = (double*)dup(pos, sizeof(double) * 3 * (size_t)n);
    s->quat = (double*)dup(quat, sizeof(double) * 4 * (size_t)n);
    s->vel = (double*)dup(vel, sizeof(double) * 3 * (size_t)n);
    s->angvel = (double*)dup(angvel, sizeof(double) * 3 * (size_t)n);
    s->F = (double*)calloc(3 * (size_t)n + 1, sizeof(double));
    s->T = (double*)calloc(3 * (size_t)n + 1, sizeof(double));
    s->ns = orc_num_spheres(m, n, tpl);
    s->margin = (double*)malloc(sizeof(double) * (size_t)(s->ns + 1));
    for (long long i = 0; i < s->ns; ++i) s->margin[i] = margin;
    s->margin_value = margin;
    s->every = rebuild_every < 1 ? 1 : rebuild_every;
    s->pa = s->pb = s->ws = s->ww = NULL;
    s->up = s->uw = NULL;
    return s;
}

/* Rebuild both lists at the current state and carry the tangential history
 * of every pair present before and after (Eq. (3) history persists). */
static void sim_rebuild(orc_sim* s) {
    const orc_model* m = &s->m;
    const long long ns = s->ns;
    const double t = (double)s->step * m->h;
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(ns + 1));
    int* owner = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    int* tsph = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    long long* qc = (long long*)malloc(sizeof(long long) * 3 * (size_t)(ns + 1));
    long long* rho = (long long*)malloc(sizeof(long long) * (size_t)(ns + 1));
    orc_sphere_centres(m, s->n, s->tpl, s->pos, s->quat, xs, owner, tsph);
    orc_detect_coords(m, ns, xs, tsph, s->margin, qc, rho);
    const long long np = orc_pairs_binned(m, ns, owner, qc, rho, 0, NULL, NULL);
    int* pa = (int*)malloc(sizeof(int) * (size_t)(np + 1));
    int* pb = (int*)malloc(sizeof(int) * (size_t)(np + 1));
    orc_pairs_binned(m, ns, owner, qc, rho, np, pa, pb);
    double* up = (double*)calloc(3 * (size_t)np + 1, sizeof(double));
    long long j = 0;
    for (long long i = 0; i < np; ++i) {
        while (j < s->np && (s->pa[j] < pa[i] || (s->pa[j] == pa[i] && s->pb[j] < pb[i]))) ++j;
        if (j < s->np && s->pa[j] == pa[i] && s->pb[j] == pb[i])
            for (int k = 0; k < 3; ++k) up[3 * i + k] = s->up[3 * j + k];
    }
    const double travel = (double)s->every * m->h;
    const long long nw = orc_wall_candidates(m, ns, xs, tsph, s->margin, t, travel, 0, NULL, NULL);
    int* ws = (int*)malloc(sizeof(int) * (size_t)(nw + 1));
    int* ww = (int*)malloc(sizeof(int) * (size_t)(nw + 1));
    orc_wall_candidates(m, ns, xs, tsph, s->margin, t, travel, nw, ws, ww);
    double* uw = (double*)calloc(3 * (size_t)nw + 1, sizeof(double));
    j = 0;
    for (long long i = 0; i < nw; ++i) {
        while (j < s->nw && (s->ws[j] < ws[i] || (s->ws[j] == ws[i] && s->ww[j] < ww[i]))) ++j;
        if (j < s->nw && s->ws[j] == ws[i] && s->ww[j] == ww[i])
            for (int k = 0; k < 3; ++k) uw[3 * i + k] = s->uw[3 * j + k];
    }
    free(s->pa); free(s->pb); free(s->up); free(s->ws); free(s->ww); free(s->uw);
    s->pa = pa; s->pb = pb; s->up = up; s->np = np;
    s->ws = ws; s->ww = ww; s->uw = uw; s->nw = nw;
    free(xs); free(owner); free(tsph); free(qc); free(rho);
}

/* Count touching contacts (delta_n > 0 in FP64) that are not in the list. */
static long long sim_audit(const orc_sim* s) {
    const orc_model* m = &s->m;
    const long long ns = s->ns;
    const double t = (double)s->step * m->h;
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)(ns + 1));
    int* owner = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    int* tsph = (int*)malloc(sizeof(int) * (size_t)(ns + 1));
    long long* qc = (long long*)malloc(sizeof(long long) * 3 * (size_t)(ns + 1));
    long long* rho = (long long*)malloc(sizeof(long long) * (size_t)(ns + 1));
    double* zero = (double*)calloc((size_t)ns + 1, sizeof(double));
    orc_sphere_centres(m, s->n, s->tpl, s->pos, s->quat, xs, owner, tsph);
    orc_detect_coords(m, ns, xs, tsph, zero, qc, rho);
    const long long np = orc_pairs_binned(m, ns, owner, qc, rho, 0, NULL, NULL);
    int* pa = (int*)malloc(sizeof(int) * (size_t)(np + 1));
    int* pb = (int*)malloc(sizeof(int) * (size_t)(np + 1));
    orc_pairs_binned(m, ns, owner, qc, rho, np, pa, pb);
    long long miss = 0, j = 0;
    for (long long i = 0; i < np; ++i) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = xs[3 * (long long)pb[i] + k] - xs[3 * (long long)pa[i] + k];
        const double gap = sqrt(dot3(d, d)) - (m->tpl_rad[tsph[pa[i]]] + m->tpl_rad[tsph[pb[i]]]);
        if (!(gap < 0.0)) continue;
        while (j < s->np && (s->pa[j] < pa[i] || (s->pa[j] == pa[i] && s->pb[j] < pb[i]))) ++j;
        if (!(j < s->np && s->pa[j] == pa[i] && s->pb[j] == pb[i])) ++miss;
    }
    j = 0;
    for (long long i = 0; i < ns; ++i)
        for (int k = 0; k < m->n_walls; ++k) {
            double nw[3];
            if (!(orc_wall_distance(m->walls + k, t, xs + 3 * i, nw) < m->tpl_rad[tsph[i]])) continue;
            while (j < s->nw && (s->ws[j] < i || (s->ws[j] == i && s->ww[j] < k))) ++j;
            if (!(j < s->nw && s->ws[j] == i && s->ww[j] == k)) ++miss;
        }
    free(xs); free(owner); free(tsph); free(qc); free(rho); free(zero); free(pa); free(pb);
    return miss;
}

long long orc_sim_step(orc_sim* s, int nsteps, int audit) {
    long long misses = 0;
    for (int it = 0; it < nsteps; ++it) {
        if (s->step == 0 || s->since >= s->every || s->pa == NULL) {
            sim_rebuild(s);
            s->since = 0;
        }
        if (audit) misses += sim_audit(s);
        const double t = (double)s->step * s->m.h;
        s->active = orc_forces(&s->m, s->n, s->tpl, s->pos, s->quat, s->vel, s->angvel, t,
                               s->np, s->pa, s->pb, s->up, s->nw, s->ws, s->ww, s->uw, s->F,
                               s->T, NULL, NULL, NULL);
        orc_integrate(&s->m, s->n, s->tpl, s->pos, s->quat, s->vel, s->angvel, s->F, s->T);
        s->step += 1;
        s->since += 1;
    }
    return misses;
}

void orc_sim_get_state(const orc_sim* s, double* pos, double* quat, double* vel,
                       double* angvel) {
    memcpy(pos, s->pos, sizeof(double) * 3 * (size_t)s->n);
    memcpy(quat, s->quat, sizeof(double) * 4 * (size_t)s->n);
    memcpy(vel, s->vel, sizeof(double) * 3 * (size_t)s->n);
    memcpy(angvel, s->angvel, sizeof(double) * 3 * (size_t)s->n);
}

long long orc_sim_num_contacts(const orc_sim* s, long long* n_wall) {
    if (n_wall) *n_wall = s->nw;
    return s->np;
}

void orc_sim_get_contacts(const orc_sim* s, int* a, int* b, double* u, int* ws, int* ww,
                          double* uw) {
    if (a) memcpy(a, s->pa, sizeof(int) * (size_t)s->np);
    if (b) memcpy(b, s->pb, sizeof(int) * (size_t)s->np);
    if (u) memcpy(u, s->up, sizeof(double) * 3 * (size_t)s->np);
    if (ws) memcpy(ws, s->ws, sizeof(int) * (size_t)s->nw);
    if (ww) memcpy(ww, s->ww, sizeof(int) * (size_t)s->nw);
    if (uw) memcpy(uw, s->uw, sizeof(double) * 3 * (size_t)s->nw);
}

void orc_sim_last_forces(const orc_sim* s, double* F, double* T) {
    memcpy(F, s->F, sizeof(double) * 3 * (size_t)s->n);
    memcpy(T, s->T, sizeof(double) * 3 * (size_t)s->n);
}

double orc_sim_time(const orc_sim* s) { return (double)s->step * s->m.h; }
long long orc_sim_active(const orc_sim* s) { return s->active; }

void orc_sim_destroy(orc_sim* s) {
    if (!s) return;
    free(s->tpl); free(s->pos); free(s->quat); free(s->vel); free(s->angvel);
    free(s->F); free(s->T); free(s->margin);
    free(s->pa); free(s->pb); free(s->up); free(s->ws); free(s->ww); free(s->uw);
    free(s);
}

/* ------------------------------------------------------------------ */
/* learned lifetime regressor: plain dense layers, ReLU, MSE, Adam       */
/* ------------------------------------------------------------------ */
#define MLP_L 4
static const int mlp_in[MLP_L] = {ORC_MLP_IN, ORC_MLP_H, ORC_MLP_H, ORC_MLP_H};
static const int mlp_out[MLP_L] = {ORC_MLP_H, ORC_MLP_H, ORC_MLP_H, 1};

int orc_mlp_num_params(void) {
    int n = 0;
    for (int l = 0; l < MLP_L; ++l) n += mlp_out[l] * mlp_in[l] + mlp_out[l];
    return n;
}

/* Forward pass of one sample, keeping every layer's activations. */
static double mlp_sample(const double* p, const double* x, double act[MLP_L + 1][ORC_MLP_H],
                         double pre[MLP_L][ORC_MLP_H]) {
    for (int i = 0; i < ORC_MLP_IN; ++i) act[0][i] = x[i];
    const double* w = p;
    for (int l = 0; l < MLP_L; ++l) {
        const double* b = w + mlp_out[l] * mlp_in[l];
        for (int o = 0; o < mlp_out[l]; ++o) {
            double s = b[o];
            for (int i = 0; i < mlp_in[l]; ++i) s += w[o * mlp_in[l] + i] * act[l][i];
            pre[l][o] = s;
            act[l + 1][o] = (l < MLP_L - 1) ? (s > 0.0 ? s : 0.0) : s;
        }
        w = b + mlp_out[l];
    }
    return act[MLP_L][0];
}

void orc_mlp_forward(const double* params, long long n, const double* x, double* y) {
    double act[MLP_L + 1][ORC_MLP_H], pre[MLP_L][ORC_MLP_H];
    for (long long k = 0; k < n; ++k) y[k] = mlp_sample(params, x + ORC_MLP_IN * k, act, pre);
}

/* The nearest bfloat16 (8 significant bits), ties to even. */
static double round_bf16(double v) {
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    const double m = frexp(v, &e);           /* v = m 2^e, 0.5 <= |m| < 1 */
    return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* The forward pass with every layer's input (the features and the three
 * hidden activations after ReLU) rounded to bfloat16 before its products, the
 * sums kept in double: the arithmetic of a tensor-core pass with bfloat16
 * operands and wide accumulation.  The caller rounds the weights. */
void orc_mlp_forward_bf16act(const double* params, long long n, const double* x, double* y) {
    for (long long k = 0; k < n; ++k) {
        double in[ORC_MLP_H], out[ORC_MLP_H];
        for (int i = 0; i < ORC_MLP_IN; ++i) in[i] = round_bf16(x[ORC_MLP_IN * k + i]);
        const double* w = params;
        for (int l = 0; l < MLP_L; ++l) {
            const double* b = w + mlp_out[l] * mlp_in[l];
            for (int o = 0; o < mlp_out[l]; ++o) {
                double s = b[o];
                for (int i = 0; i < mlp_in[l]; ++i) s += w[o * mlp_in[l] + i] * in[i];
                out[o] = (l < MLP_L - 1) ? round_bf16(s > 0.0 ? s : 0.0) : s;
            }
            for (int o = 0; o < mlp_out[l]; ++o) in[o] = out[o];
            w = b + mlp_out[l];
        }
        y[k] = in[0];
    }
}

double orc_mlp_loss_grad(const double* params, long long n, const double* x, const double* t,
                         double* grad) {
    const int np = orc_mlp_num_params();
    if (grad) for (int i = 0; i < np; ++i) grad[i] = 0.0;
    double loss = 0.0;
    double act[MLP_L + 1][ORC_MLP_H], pre[MLP_L][ORC_MLP_H], delta[ORC_MLP_H], nd[ORC_MLP_H];
    int off[MLP_L];
    off[0] = 0;
    for (int l = 1; l < MLP_L; ++l) off[l] = off[l - 1] + mlp_out[l - 1] * mlp_in[l - 1] + mlp_out[l - 1];
    for (long long k = 0; k < n; ++k) {
        const double y = mlp_sample(params, x + ORC_MLP_IN * k, act, pre);
        const double e = y - t[k];
        loss += e * e;
        if (!grad) continue;
        /* dL/dy for L = (1/n) sum e^2 */
        delta[0] = 2.0 * e / (double)n;
        for (int l = MLP_L - 1; l >= 0; --l) {
            const double* w = params + off[l];
            double* gw = grad + off[l];
            double* gb = gw + mlp_out[l] * mlp_in[l];
            for (int o = 0; o < mlp_out[l]; ++o) {
                gb[o] += delta[o];
                for (int i = 0; i < mlp_in[l]; ++i) gw[o * mlp_in[l] + i] += delta[o] * act[l][i];
            }
            if (l == 0) break;
            /* back through W and the ReLU of the layer below */
            for (int i = 0; i < mlp_in[l]; ++i) {
                double s = 0.0;
                for (int o = 0; o < mlp_out[l]; ++o) s += w[o * mlp_in[l] + i] * delta[o];
                nd[i] = pre[l - 1][i] > 0.0 ? s : 0.0;
            }
            for (int i = 0; i < mlp_in[l]; ++i) delta[i] = nd[i];
        }
    }
    return loss / (double)n;
}

void orc_mlp_adam(double* params, double* m, double* v, const double* grad, int step, double lr,
                  double beta1, double beta2, double eps) {
    const int np = orc_mlp_num_params();
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (int i = 0; i < np; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
