// dem_detect.cu -- contact detection with an enlarged geometry (section 2.2).
//
// Every sphere, enlarged by the safety margin, is quantised onto the 2^-24 m
// detection lattice and registered in every bin its enlarged box touches
// (multi-bin registration).  The registrations are grouped by bin key with a
// counting sort (an LSD radix sort whose single digit is the whole key: count
// per bin, exclusive scan, scatter into slots); each bin's members are then
// tested pairwise, across clumps, with the exact integer predicate
// |qa - qb|^2 <= (rho_a + rho_b)^2, keeping a pair only in the bin that holds
// the per-axis maximum of the two boxes' lower corners, so each pair is found
// once.  The output is a canonical list sorted by (a, b), one row per sphere,
// onto which the tangential history of the previous list is carried.
#include <cfloat>

#include "dem_dev.cuh"
#include "dem_prims.cuh"
#include "dem_walls.cuh"

namespace dem {

namespace {

__device__ __forceinline__ void clump_com(const DevState& d, int c, const SceneGrid& g,
                                          double X[3]) {
  if (d.prec == 0) {
    const double4_32a p = d.cpos[c];
    X[0] = p.x; X[1] = p.y; X[2] = p.z;
  } else {
    const int4 v = d.cvox[c];
    const float4 o = d.coff[c];
    // exact for positions on the 2^-44 m grid (see dem_set_state)
    X[0] = __dadd_rn(g.lo[0], __dadd_rn(__dmul_rn((double)v.x, kVoxel), (double)o.x));
    X[1] = __dadd_rn(g.lo[1], __dadd_rn(__dmul_rn((double)v.y, kVoxel), (double)o.y));
    X[2] = __dadd_rn(g.lo[2], __dadd_rn(__dmul_rn((double)v.z, kVoxel), (double)o.z));
  }
}

// Float estimate of the same distance; |error| is far below wall_slack().
// A facet's distance is at least its plane distance, so once that exceeds
// `cut` (the caller's threshold + slack: the pair is no candidate either way)
// it is returned without the region and edge work.
__device__ float wall_distance_est(const WallDev& w, float t, const float x[3], float cut) {
  float dd[3], n[3];
  for (int k = 0; k < 3; ++k) {
    dd[k] = x[k] - (w.pf[k] + w.vf[k] * t);
    n[k] = w.nh[k];
  }
  const float ax = dd[0] * n[0] + dd[1] * n[1] + dd[2] * n[2];
  if (w.type == 0) return ax;
  if (w.type == 3) {
    if (ax > cut) return ax;
    const float* e1 = w.e1h;
    const float* e2 = w.e2h;
    const float d00 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const float d01 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const float d11 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const float b0 = dd[0] * e1[0] + dd[1] * e1[1] + dd[2] * e1[2];
    const float b1 = dd[0] * e2[0] + dd[1] * e2[1] + dd[2] * e2[2];
    const float den = d00 * d11 - d01 * d01;
    const float u = (d11 * b0 - d01 * b1) / den, v = (d00 * b1 - d01 * b0) / den;
    if (u >= 0.f && v >= 0.f && u + v <= 1.f) return ax;
    float best = 3.4e38f;
    for (int j = 0; j < 3; ++j) {
      float r[3], e[3];
      for (int k = 0; k < 3; ++k) {
        r[k] = j == 2 ? dd[k] - e1[k] : dd[k];
        e[k] = j == 0 ? e1[k] : (j == 1 ? e2[k] : e2[k] - e1[k]);
      }
      float t = (r[0] * e[0] + r[1] * e[1] + r[2] * e[2]) / (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      t = fminf(fmaxf(t, 0.f), 1.f);
      const float q0 = r[0] - t * e[0], q1 = r[1] - t * e[1], q2 = r[2] - t * e[2];
      best = fminf(best, sqrtf(q0 * q0 + q1 * q1 + q2 * q2));
    }
    return best;
  }
  float rv[3] = {dd[0] - ax * n[0], dd[1] - ax * n[1], dd[2] - ax * n[2]};
  const float rho = sqrtf(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
  if (w.type == 1) return w.radf - rho;
  const float H = w.heightf, Rb = w.rbf;
  float tl = (rho * Rb + ax * H) / (Rb * Rb + H * H);
  tl = fminf(fmaxf(tl, 0.f), 1.f);
  const float dl = sqrtf((rho - tl * Rb) * (rho - tl * Rb) + (ax - tl * H) * (ax - tl * H));
  float tb = fminf(fmaxf(rho / Rb, 0.f), 1.f);
  const float db = sqrtf((rho - tb * Rb) * (rho - tb * Rb) + (ax - H) * (ax - H));
  const bool inside = (ax >= 0.f && ax <= H && rho * H <= ax * Rb);
  const float dm = fminf(dl, db);
  return inside ? -dm : dm;
}

__device__ __forceinline__ float wall_slack(const WallDev& w, const float x[3]) {
  float m = fabsf(w.pf[0]) + fabsf(w.pf[1]) + fabsf(w.pf[2]) +
            fabsf(x[0]) + fabsf(x[1]) + fabsf(x[2]) + 1.f;
  return 4e-6f * m;
}

// Lattice coordinates of a sphere centre.  The exact value is the double
// formula det_centre() rounded to the nearest lattice point; the pose record
// written by the last update kernel carries the same centre with a known
// error bound (FP32_VOXEL: within 2 fixed-point units of 2^-44 m; FP64:
// within 2^-20 lattice units), so the formula is evaluated only when that
// approximation lies too close to a rounding boundary to decide it.
__device__ __forceinline__ bool lattice_from_pose(const DevState& d, long long s, const SceneGrid& g,
                                                  long long qc[3], float xf[3]) {
  bool exact = true;
  if (d.prec == 1) {
    long long P[3];
    sphere_fix(d, s, d.sinfo[s].x, P);
    for (int k = 0; k < 3; ++k) {
      const long long half = 1ll << (kFixBits - kDetBits - 1);
      const long long rem = P[k] & ((1ll << (kFixBits - kDetBits)) - 1);
      if (rem - half <= 2 && half - rem <= 2) exact = false;
      qc[k] = (P[k] + half) >> (kFixBits - kDetBits);
      xf[k] = g.lof[k] + ff_to_float(fix_to_ff(P[k]));
    }
  } else {
    const SphA64 A = d.sa64[s];
    const double P[3] = {A.x, A.y, A.z};
    for (int k = 0; k < 3; ++k) {
      const double u = (P[k] - g.lo[k]) * kDetScale;
      const double f = u - floor(u);
      if (fabs(f - 0.5) < 0x1p-20) exact = false;
      qc[k] = __double2ll_rn(u);
      xf[k] = (float)P[k];
    }
  }
  return exact;
}

// The bins an enlarged box {q - rho, q + rho} touches (clamped to the grid),
// walked with x fastest; mask() is the owning-bin mask of the current bin.
struct BinWalk {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int x = 0, y = 0, z = 0;
  long long n = 0;  // bins touched
  uint32_t d0 = 0, d01 = 0, base = 0;
  __device__ void init(const SceneGrid& g, const int4 q) {
    const int qq[3] = {q.x, q.y, q.z};
    for (int k = 0; k < 3; ++k) {
      lo[k] = clampi(floordiv_bin((long long)qq[k] - q.w, g.L, g.invL), g.dims[k] - 1);
      hi[k] = clampi(floordiv_bin((long long)qq[k] + q.w, g.L, g.invL), g.dims[k] - 1);
    }
    x = lo[0]; y = lo[1]; z = lo[2];
    n = (long long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    d0 = (uint32_t)g.dims[0];
    d01 = d0 * (uint32_t)g.dims[1];
    base = g.key_base;
  }
  __device__ uint32_t key() const { return base + (uint32_t)z * d01 + (uint32_t)y * d0 + (uint32_t)x; }
  __device__ uint32_t mask() const {
    return (x == lo[0] ? 1u : 0u) | (y == lo[1] ? 2u : 0u) | (z == lo[2] ? 4u : 0u);
  }
  __device__ void next() {
    if (++x > hi[0]) {
      x = lo[0];
      if (++y > hi[1]) { y = lo[1]; ++z; }
    }
  }
};

// ceil((r + m) 2^24) + 1 with r + m rounded to double (the scaling by 2^24 is exact).
__device__ __forceinline__ long long tpl_rho(double r, double m) {
  return ceil_pos_d2ll(__dmul_rn(__dadd_rn(r, m), kDetScale)) + 1;
}

__global__ void k_tpl_rho(DevState d, double margin, int n, int* __restrict__ trho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) trho[i] = (int)tpl_rho(d.tp64[i].w, margin);
}

// The exact detection centre of sphere s (owner c, template sphere ts) and
// its float estimate, computed on first use.
struct SphereCentre {
  const DevState& d;
  long long s;
  int c, ts;
  const SceneGrid& g;
  double x[3];
  bool have = false;
  __device__ SphereCentre(const DevState& dd, long long ss, int cc, int tt, const SceneGrid& gg)
      : d(dd), s(ss), c(cc), ts(tt), g(gg) {}
  __device__ const double* exact() {
    if (!have) {
      double X[3];
      clump_com(d, c, g, X);
      const double4_32a q4 = d.cq[c];
      const double4_32a tp = d.tp64[ts];
      const double q[4] = {q4.x, q4.y, q4.z, q4.w};
      const double p[3] = {tp.x, tp.y, tp.z};
      det_centre(q, p, X, x);
      have = true;
    }
    return x;
  }
};

// Is wall w a candidate of the sphere (section 2.2's enlarged geometry: the
// distance from its centre to the wall at time t within r + m plus the
// wall's travel over the list's lifetime)?  A float estimate decides when it
// is clear of the threshold by more than its error bound; otherwise the
// double distance from the exact centre, as the oracle evaluates it.
__device__ __forceinline__ bool wall_candidate(const WallDev& w, float tf, float ttf,
                                               const float xf[3], float rmf, double t,
                                               double travel_time, double r, double m,
                                               SphereCentre& ctr) {
  const float thrf = rmf + w.speed * ttf;
  const float slack = wall_slack(w, xf);
  bool exact = false;
  if (w.type == 3) {
    // a facet is one-sided: clearly behind its plane, no candidate; within
    // the estimate's error of the plane, the side is decided exactly
    float ax = 0.f;
    for (int k = 0; k < 3; ++k) ax += (xf[k] - (w.pf[k] + w.vf[k] * tf)) * w.nh[k];
    if (ax < -slack) return false;
    exact = ax <= slack;
  }
  if (!exact) {
    const float est = wall_distance_est(w, tf, xf, thrf + slack);
    if (est > thrf + slack) return false;
    if (est < thrf - slack) return true;
  }
  double nw[3];
  const double thr = __dadd_rn(__dadd_rn(r, m), __dmul_rn(w.speed_d, travel_time));
  return wall_distance64(w, t, ctr.exact(), nw) <= thr;
}

// One thread per sphere: detection coordinates, analytic wall candidates, and
// the counting pass of the bin sort (one count per bin the enlarged box
// touches).  Mesh facets are found through the bins (k_facet_narrow).
// Lattice point of sphere s (clamped) and its enlarged lattice radius, with
// the float estimate xf of its centre.
__device__ __forceinline__ void sphere_lattice(const DevState& d, const DetectOut& o, long long s,
                                               int2 si, const SceneGrid& g, double m,
                                               SphereCentre& ctr, long long qc[3], float xf[3],
                                               long long& rho) {
  if (!lattice_from_pose(d, s, g, qc, xf)) {
    const double* x = ctr.exact();
    for (int k = 0; k < 3; ++k) qc[k] = __double2ll_rn(__dmul_rn(__dsub_rn(x[k], g.lo[k]), kDetScale));
  }
  for (int k = 0; k < 3; ++k) {
    // a sphere more than 64 m outside its domain is clamped (it only meets
    // the boundary bins, where it can still be found); the clamped range
    // keeps every coordinate difference inside 32 bits
    constexpr long long kQ = (1ll << 30) - 1;
    qc[k] = qc[k] < -kQ ? -kQ : (qc[k] > kQ ? kQ : qc[k]);
  }
  // enlarged lattice radius ceil((r + m) 2^24) + 1: from the per template
  // sphere table when every clump has the same margin
  rho = o.trho ? (long long)o.trho[si.y] : tpl_rho(d.tp64[si.y].w, m);
}

__global__ void k_detect(DevState d, DetectOut o, double margin, const double* __restrict__ smargin,
                         double t, double travel_time) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns) return;
  const int2 si = d.sinfo[s];
  const int2 ci = d.cinfo[si.x];
  const float ttf = d2f(travel_time);
  const SceneGrid g = d.grids[ci.y];
  SphereCentre ctr(d, s, si.x, si.y, g);
  const double m = smargin ? smargin[s] : (d.cmargin ? f2d(d.cmargin[si.x]) : margin);
  long long qc[3], rho;
  float xf[3];
  sphere_lattice(d, o, s, si, g, m, ctr, qc, xf, rho);
  const float tf = d2f(t);
  const double mw = m + o.wall_extra;  // the wall candidates' margin
  const float rmf = d.tp32[si.y].w + d2f(mw);  // r + m for the estimates
  const int4 dq = make_int4((int)qc[0], (int)qc[1], (int)qc[2], (int)rho);
  o.det[s] = dq;
  {
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = clampi(floordiv_bin(qc[k] - rho, g.L, g.invL), g.dims[k] - 1);
      hi[k] = clampi(floordiv_bin(qc[k] + rho, g.L, g.invL), g.dims[k] - 1);
    }
    const uint32_t d0 = (uint32_t)g.dims[0], d01 = d0 * (uint32_t)g.dims[1];
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
      for (int by = lo[1]; by <= hi[1]; ++by)
        for (int bx = lo[0]; bx <= hi[0]; ++bx)
          atomicAdd(&o.bin_size[g.key_base + (uint32_t)bz * d01 + (uint32_t)by * d0 + (uint32_t)bx], 1u);
  }
  // analytic wall candidates: distance within radius + margin + wall travel
  uint32_t mask = 0;
  for (int i = 0; i < g.wall_count; ++i) {
    const WallDev& w = d.walls[d.wall_idx[g.wall_start + i]];
    if (wall_candidate(w, tf, ttf, xf, rmf, t, travel_time, d.tp64[si.y].w, mw, ctr)) mask |= 1u << i;
  }
  o.wall_mask[s] = mask;
  o.wall_cnt[s] = __popc(mask);
}

// Scatter pass of the bin sort: every registration takes a slot of its bin
// (counting the bin's size down to zero) and stores there the record the
// narrow phase tests (lattice centre, enlarged radius, owner, sphere id,
// owning-bin mask).  The order inside a bin is whatever the atomics give;
// nothing downstream depends on it.  A slot request past the counted size (a
// broken invariant) is dropped and flagged.
__global__ void k_bin_scatter(DevState d, DetectOut o) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns) return;
  const int4 q = o.det[s];
  const int owner = d.sinfo[s].x;
  BinWalk w;
  w.init(d.grids[d.cinfo[owner].y], q);
  for (long long r = 0; r < w.n; ++r, w.next()) {
    const uint32_t key = w.key();
    const uint32_t left = atomicSub(&o.bin_size[key], 1u);
    if (left == 0u) {  // more registrations than counted: a broken invariant
      atomicAdd(&o.bin_size[key], 1u);
      atomicOr(d.flags, kFlagBounds);
      continue;
    }
    EntryRec rec;
    rec.qx = q.x; rec.qy = q.y; rec.qz = q.z; rec.rho = q.w;
    rec.owner = owner;
    rec.id = (uint32_t)s;
    rec.mask = w.mask();
    rec.pad = 0u;
    o.rec[o.bin_start[key] + left - 1u] = rec;
  }
}

// ---------------------------------------------------------------------------
// mesh facets in the bins
// ---------------------------------------------------------------------------
// A facet is registered, like a sphere, in every bin its enlarged box touches:
// the box of its three vertices at time t, widened by the distance it
// travels over the list's lifetime and by two lattice units for the
// roundings.  A sphere within reach of the facet (centre within r + m + that
// travel of a point of the facet) has an enlarged box [q - rho, q + rho]
// that meets the facet's box, so the two share a bin; the pair is tested
// only in the bin of the per-axis max of the two boxes' lower corners (the
// owning-bin rule of the sphere pairs), so it is found once.
__device__ __forceinline__ void facet_box(const DevState& d, const WallDev& w, const SceneGrid& g,
                                          double t, double travel_time, long long lo[3],
                                          long long hi[3]) {
  const double reach = __dmul_rn(w.speed_d, travel_time);
  for (int k = 0; k < 3; ++k) {
    const double a = w.p[k] + w.vel[k] * t;
    const double mn = fmin(a, fmin(a + w.e1[k], a + w.e2[k])) - reach;
    const double mx = fmax(a, fmax(a + w.e1[k], a + w.e2[k])) + reach;
    constexpr double kQ = (double)((1ll << 30) - 1);
    const double l = fmin(fmax(floor((mn - g.lo[k]) * kDetScale) - 2.0, -kQ), kQ);
    const double h = fmin(fmax(ceil((mx - g.lo[k]) * kDetScale) + 2.0, -kQ), kQ);
    lo[k] = (long long)l;
    hi[k] = (long long)h;
  }
}

// The bins of a facet's enlarged box (clamped to its scene's grid).
struct FacetBins {
  int b0[3], b1[3];
  uint32_t d0, d01, base;
  long long n;
  __device__ FacetBins(const DevState& d, const DetectOut& o, int f, double t, double travel_time) {
    const int w = d.facet_idx[f];
    const SceneGrid g = d.grids[d.wall_scene[w]];
    long long lo[3], hi[3];
    facet_box(d, d.walls[w], g, t, travel_time, lo, hi);
    for (int k = 0; k < 3; ++k) {
      b0[k] = clampi(floordiv_ll(lo[k], g.L), g.dims[k] - 1);
      b1[k] = clampi(floordiv_ll(hi[k], g.L), g.dims[k] - 1);
    }
    d0 = (uint32_t)g.dims[0];
    d01 = d0 * (uint32_t)g.dims[1];
    base = g.key_base;
    n = (long long)(b1[0] - b0[0] + 1) * (b1[1] - b0[1] + 1) * (b1[2] - b0[2] + 1);
  }
  // the j-th bin (x fastest): key and owning-bin mask
  __device__ uint32_t key(long long j, uint32_t& mask) const {
    const long long nx = b1[0] - b0[0] + 1, ny = b1[1] - b0[1] + 1;
    const int bx = b0[0] + (int)(j % nx), by = b0[1] + (int)((j / nx) % ny),
              bz = b0[2] + (int)(j / (nx * ny));
    mask = (bx == b0[0] ? 1u : 0u) | (by == b0[1] ? 2u : 0u) | (bz == b0[2] ? 4u : 0u);
    return base + (uint32_t)bz * d01 + (uint32_t)by * d0 + (uint32_t)bx;
  }
};

// One block per facet, its threads over the facet's bins (a facet of a box
// face spans a whole layer of bins): counts its registrations (o.fbin_size).
__global__ void k_facet_count(DevState d, DetectOut o, double t, double travel_time) {
  const FacetBins fb(d, o, blockIdx.x, t, travel_time);
  for (long long j = threadIdx.x; j < fb.n; j += blockDim.x) {
    uint32_t mask;
    atomicAdd(&o.fbin_size[fb.key(j, mask)], 1u);
  }
}

// Scatter pass: every facet registration takes a slot of its bin and stores
// the bin key, the wall id and the facet's owning-bin mask in that bin.
__global__ void k_facet_scatter(DevState d, DetectOut o, double t, double travel_time) {
  const FacetBins fb(d, o, blockIdx.x, t, travel_time);
  const uint32_t w = (uint32_t)d.facet_idx[blockIdx.x];
  for (long long j = threadIdx.x; j < fb.n; j += blockDim.x) {
    uint32_t mask;
    const uint32_t key = fb.key(j, mask);
    const uint32_t left = atomicSub(&o.fbin_size[key], 1u);
    if (left == 0u) {  // more registrations than counted: a broken invariant
      atomicAdd(&o.fbin_size[key], 1u);
      atomicOr(d.flags, kFlagBounds);
      continue;
    }
    o.frec[o.fbin_start[key] + left - 1u] = make_uint4(key, w, mask, 0u);
  }
}

// Facet narrow phase: one warp per facet registration, its lanes over the
// sphere registrations of the same bin.  A (sphere, facet) pair owned by the
// bin is a candidate when the sphere is within reach (wall_candidate); it
// goes to o.fcand and counts in o.fcnt[sphere].  Candidates past o.fcap are
// counted but not written (the caller grows the buffer and runs again).
__global__ void k_facet_narrow(DevState d, DetectOut o, double margin,
                               const double* __restrict__ smargin, double t, double travel_time) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const float tf = d2f(t), ttf = d2f(travel_time);
  for (long long e = warp; e < o.nfreg; e += nwarps) {
    const uint4 fr = o.frec[e];
    const uint32_t key = fr.x;
    const WallDev& w = d.walls[fr.y];
    const uint32_t b0 = o.bin_start[key], b1 = o.bin_start[key + 1];
    for (uint32_t j = b0 + lane; j < b1; j += 32) {
      const EntryRec r = o.rec[j];
      if ((r.mask | fr.z) != 7u) continue;  // another bin owns the pair
      const int2 si = d.sinfo[r.id];
      const SceneGrid g = d.grids[d.cinfo[si.x].y];
      const double m = (smargin ? smargin[r.id] : (d.cmargin ? f2d(d.cmargin[si.x]) : margin)) +
                       o.wall_extra;
      // float centre from the lattice point (within 2^-25 m, far below the slack)
      const float xf[3] = {g.lof[0] + (float)r.qx * (1.f / 16777216.f),
                           g.lof[1] + (float)r.qy * (1.f / 16777216.f),
                           g.lof[2] + (float)r.qz * (1.f / 16777216.f)};
      const float rmf = d.tp32[si.y].w + d2f(m);
      SphereCentre ctr(d, r.id, si.x, si.y, g);
      if (!wall_candidate(w, tf, ttf, xf, rmf, t, travel_time, d.tp64[si.y].w, m, ctr)) continue;
      const unsigned long long slot = atomicAdd(o.d_nf, 1ull);
      if (slot < o.fcap) o.fcand[slot] = make_uint2(r.id, fr.y);
      atomicAdd(&o.fcnt[r.id], 1u);
    }
  }
}

// After k_wall_emit: each facet candidate takes a slot after its sphere's
// analytic walls (o.fcnt, zeroed again, counts the slots taken), then every
// row that got facets is sorted by wall id (rows are short: insertion sort).
__global__ void k_facet_emit(DevState d, DetectOut o, long long nf, int* __restrict__ ws,
                             uint32_t* __restrict__ ww) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const uint2 c = o.fcand[i];
  const uint32_t k = atomicAdd(&o.fcnt[c.x], 1u);
  const uint32_t at = o.wall_off[c.x] + __popc(o.wall_mask[c.x]) + k;
  ws[at] = (int)c.x;
  ww[at] = c.y;
}

__global__ void k_sort_wall_rows(DevState d, DetectOut o, uint32_t* __restrict__ ww) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns || o.fcnt[s] == 0u) return;
  const uint32_t r0 = o.wall_off[s], r1 = o.wall_off[s + 1];
  for (uint32_t i = r0 + 1; i < r1; ++i) {
    const uint32_t v = ww[i];
    uint32_t j = i;
    while (j > r0 && ww[j - 1] > v) {
      ww[j] = ww[j - 1];
      --j;
    }
    ww[j] = v;
  }
}

// wall_cnt[s] += fcnt[s] (analytic walls plus facets per sphere), and fcnt
// cleared for k_facet_emit's slots; rows with facets are flagged in fcnt by
// k_facet_emit again.
__global__ void k_add_facet_counts(long long ns, DetectOut o) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  o.wall_cnt[s] += o.fcnt[s];
  o.fcnt[s] = 0u;
}

// ---------------------------------------------------------------------------
// inner lists filtered from an outer list
// ---------------------------------------------------------------------------
// An outer list holds the pairs and wall candidates of a detection with a
// wider margin m_out, from the lattice points q0 and enlarged radii rho' of
// its time.  While every sphere's lattice point stays within rho' - rho of
// q0 (rho the enlarged radius at the list's own margin m), every pair that
// meets the exact predicate |q_a - q_b|^2 <= (rho_a + rho_b)^2 now met the
// wider one then (|q0_a - q0_b| <= |q_a - q_b| + |dq_a| + |dq_b| <= rho'_a +
// rho'_b), so filtering the outer list with the predicate gives exactly the
// list a fresh detection would give, in the same (a, b) order.  Wall
// candidates likewise (the outer list's wall threshold covers the travel of
// the walls over its lifetime and a little more than m_out - m of
// displacement), each kept by the fresh detection's own test.

// Lattice points and radii at the list's margin (o.det), and the count of
// spheres that left their allowance around q0 (*bad).
__global__ void k_lattice_check(DevState d, DetectOut o, double margin, const int4* __restrict__ q0,
                                unsigned long long* bad) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns) return;
  const int2 si = d.sinfo[s];
  const SceneGrid g = d.grids[d.cinfo[si.x].y];
  SphereCentre ctr(d, s, si.x, si.y, g);
  long long qc[3], rho;
  float xf[3];
  sphere_lattice(d, o, s, si, g, margin, ctr, qc, xf, rho);
  o.det[s] = make_int4((int)qc[0], (int)qc[1], (int)qc[2], (int)rho);
  const int4 r0 = q0[s];
  const long long lim = (long long)r0.w - rho;
  const long long dx = qc[0] - r0.x, dy = qc[1] - r0.y, dz = qc[2] - r0.z;
  if (lim < 0 || dx * dx + dy * dy + dz * dz > lim * lim) atomicAdd(bad, 1ull);
}

// The narrow phase's predicate on two lattice points (box test first, so
// that the sum of the squares fits 63 bits).
__device__ __forceinline__ bool lattice_pair(int4 qa, int4 qb) {
  const long long rr = (long long)qa.w + qb.w;
  const long long dx = (long long)qb.x - qa.x, dy = (long long)qb.y - qa.y, dz = (long long)qb.z - qa.z;
  if (dx > rr || -dx > rr || dy > rr || -dy > rr || dz > rr || -dz > rr) return false;
  return dx * dx + dy * dy + dz * dz <= rr * rr;
}

// EMIT = false: per sphere a, the partners of its outer row that pass (into
// o.pair_cnt, each decision into o.fkeep); EMIT = true: writes the kept ones
// into the inner rows (o.pair_off), from the recorded decisions.
template <bool EMIT>
__global__ void k_filter_pairs(DevState d, DetectOut o, ContactList outer, ContactList inner) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.ns) return;
  uint32_t k = EMIT ? o.pair_off[a] : 0u;
  const uint32_t j0 = outer.row[a], j1 = outer.row[a + 1];
  if (EMIT) {
    for (uint32_t j = j0; j < j1; ++j) {
      if (!o.fkeep[j]) continue;
      inner.pa[k] = (int)a;
      inner.pb[k] = outer.pb[j] & ~kHistFlag;
      ++k;
    }
    return;
  }
  if (j0 == j1) {
    o.pair_cnt[a] = 0u;
    return;
  }
  const int4 qa = o.det[a];
  for (uint32_t j = j0; j < j1; ++j) {
    const uint32_t b = outer.pb[j] & ~kHistFlag;
    const bool keep = lattice_pair(qa, o.det[b]);
    o.fkeep[j] = keep ? 1 : 0;
    k += keep ? 1u : 0u;
  }
  o.pair_cnt[a] = k;
}

// The same for each sphere's wall candidates (into o.wall_cnt, then the
// inner wall rows at o.wall_off).
template <bool EMIT>
__global__ void k_filter_walls(DevState d, DetectOut o, ContactList outer, ContactList inner,
                               double margin, double t, double travel_time) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns) return;
  const uint32_t j0 = outer.wrow[s], j1 = outer.wrow[s + 1];
  uint32_t k = EMIT ? o.wall_off[s] : 0u;
  if (EMIT && j1 - j0 <= 32u) {  // the decisions recorded by the count pass
    const uint32_t keep = j0 < j1 ? o.wkeep[s] : 0u;
    for (uint32_t j = j0; j < j1; ++j) {
      if (!((keep >> (j - j0)) & 1u)) continue;
      inner.ws[k] = (int)s;
      inner.ww[k] = outer.ww[j] & ~kHistFlag;
      ++k;
    }
    return;
  }
  uint32_t keep = 0u;
  if (j0 < j1) {
    const int2 si = d.sinfo[s];
    const SceneGrid g = d.grids[d.cinfo[si.x].y];
    SphereCentre ctr(d, s, si.x, si.y, g);
    long long qc[3];
    float xf[3];
    lattice_from_pose(d, s, g, qc, xf);
    const float tf = d2f(t), ttf = d2f(travel_time);
    const float rmf = d.tp32[si.y].w + d2f(margin);
    for (uint32_t j = j0; j < j1; ++j) {
      const uint32_t w = outer.ww[j] & ~kHistFlag;
      if (!wall_candidate(d.walls[w], tf, ttf, xf, rmf, t, travel_time, d.tp64[si.y].w, margin, ctr))
        continue;
      if (j - j0 < 32u) keep |= 1u << (j - j0);
      if (EMIT) {
        inner.ws[k] = (int)s;
        inner.ww[k] = w;
      }
      ++k;
    }
  }
  if (!EMIT) {
    o.wall_cnt[s] = k;
    if (j0 < j1) o.wkeep[s] = keep;
  }
}

// The sphere id of every registration (inspection).
__global__ void k_rec_ids(const EntryRec* __restrict__ rec, long long n, uint32_t* __restrict__ ids) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ids[i] = rec[i].id;
}

// Narrow phase, one warp per bin (persistent warps striding over the bins).
// The bin's registrations (in any order) are taken 32 at a time: lane l
// holds registration i; the registrations of the same tile are paired by
// rotation, and every later tile is staged in shared memory and tested by all
// lanes at once, so the loops are uniform across the warp.  A pair
// (a = min id < b = max id) is kept when the spheres belong to different
// clumps, the bin owns the pair (owning-bin masks) and the enlarged spheres
// overlap on the 2^-24 m lattice: |q_b - q_a|^2 <= (rho_a + rho_b)^2, exact
// in integers.
//
// Kept pairs are appended, unordered, to o.upairs through a per-warp buffer
// in shared memory that is flushed 32 pairs at a time (one global atomic per
// flush); pairs past o.ucap are counted but not written, so the caller can
// grow the buffer and run the pass again.  o.pair_cnt[a] counts the partners
// of every sphere a.
constexpr int kNarrowWarps = 8;
constexpr int kBinChunk = 8;  // bins a warp claims at a time, unless o.chunk says otherwise

__device__ __forceinline__ void flush_pairs(const DetectOut& o, uint2* buf, int n, int lane) {
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(o.d_np, (unsigned long long)n);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (lane < n && base + (unsigned long long)lane < o.ucap) o.upairs[base + lane] = buf[lane];
}

// The pair test of two registrations of one bin (A held by the lane, B from
// shared memory): different clumps, the bin owns the pair, enlarged spheres
// overlap.  Coordinates lie in [-(2^30 - 1), 2^30 - 1] and rr < 2^30 + 2, so
// the differences fit in 32 bits and -rr <= d <= rr is one unsigned
// comparison of d + rr (a wrapped sum lands above 2 rr); past it every
// |d| <= rr and the sum of the squares fits in 63 bits.
//
// The operands are pre-shifted so that an axis costs one subtraction and one
// comparison: B is staged as (q_b + rho_b, 2 rho_b), the lane holds
// (q_a - rho_a, 2 rho_a), and t = (q_b + rho_b) - (q_a - rho_a) = d + rr
// (mod 2^32) lies in [0, 2 rr] exactly when |d| <= rr.  Every predicate is
// evaluated and combined without branches (the 64-bit sum wraps harmlessly on
// lanes whose box test failed).
struct NarrowA {
  uint32_t x, y, z;  // q_a - rho_a (two's complement)
  uint32_t r2;       // 2 rho_a
  int owner;
  uint32_t mask;
};

__device__ __forceinline__ NarrowA narrow_a(const EntryRec& A) {
  return {(uint32_t)A.qx - (uint32_t)A.rho, (uint32_t)A.qy - (uint32_t)A.rho,
          (uint32_t)A.qz - (uint32_t)A.rho, 2u * (uint32_t)A.rho, A.owner, A.mask};
}

__device__ __forceinline__ int4 narrow_b(const EntryRec& R) {
  return make_int4((int)((uint32_t)R.qx + (uint32_t)R.rho), (int)((uint32_t)R.qy + (uint32_t)R.rho),
                   (int)((uint32_t)R.qz + (uint32_t)R.rho), (int)(2u * (uint32_t)R.rho));
}

__device__ __forceinline__ bool narrow_test(const NarrowA& A, const int4 q, const int4 mm) {
  const uint32_t rr2 = A.r2 + (uint32_t)q.w;
  const uint32_t tx = (uint32_t)q.x - A.x, ty = (uint32_t)q.y - A.y, tz = (uint32_t)q.z - A.z;
  const bool box = (tx <= rr2) & (ty <= rr2) & (tz <= rr2);
  const uint32_t rr = rr2 >> 1;
  const int dx = (int)(tx - rr), dy = (int)(ty - rr), dz = (int)(tz - rr);
  const unsigned long long d2 = (unsigned long long)((long long)dx * dx) +
                                (unsigned long long)((long long)dy * dy) +
                                (unsigned long long)((long long)dz * dz);
  const bool sph = d2 <= (unsigned long long)rr * rr;
  return box & sph & (mm.x != A.owner) & ((A.mask | (uint32_t)mm.z) == 7u);
}

__global__ void __launch_bounds__(32 * kNarrowWarps) k_narrow_bins(DetectOut o) {
  __shared__ int4 sq[kNarrowWarps][32];   // q + rho (x, y, z), 2 rho
  __shared__ int4 sm[kNarrowWarps][32];   // owner, id, mask
  __shared__ uint2 sbuf[kNarrowWarps][64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint2* buf = sbuf[wib];
  int nbuf = 0;  // warp-uniform
  // appends the kept pairs of one warp-wide test to the warp's buffer as
  // (lower id, higher id) and counts a partner of the lower id
  auto emit = [&](bool hit, uint32_t a, uint32_t b) {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (!m) return;
    if (hit) {
      const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
      atomicAdd(&o.pair_cnt[lo], 1u);
      buf[nbuf + __popc(m & lt)] = make_uint2(lo, hi);
    }
    nbuf += __popc(m);
    if (nbuf >= 32) {
      __syncwarp();
      flush_pairs(o, buf, 32, lane);
      __syncwarp();
      const int rem = nbuf - 32;  // < 32: move them to the front
      uint2 v = make_uint2(0u, 0u);
      if (lane < rem) v = buf[32 + lane];
      __syncwarp();
      if (lane < rem) buf[lane] = v;
      __syncwarp();
      nbuf = rem;
    }
  };
  auto stage = [&](uint32_t j0, uint32_t e) {
    const uint32_t jl = j0 + (uint32_t)lane;
    if (jl < e) {
      const EntryRec R = o.rec[jl];
      sq[wib][lane] = narrow_b(R);
      sm[wib][lane] = make_int4(R.owner, (int)R.id, (int)R.mask, 0);
    }
    __syncwarp();
  };
  // every warp claims chunks of consecutive bins from a global counter until
  // none are left, so bins of uneven size do not leave warps idle at the end
  const unsigned long long chunk = (unsigned long long)(o.chunk > 0 ? o.chunk : kBinChunk);
  unsigned long long bin = 0, b1 = 0;  // the warp's current chunk [bin, b1)
  for (;; ++bin) {
    if (bin >= b1) {
      unsigned long long b0 = 0;
      if (lane == 0) b0 = atomicAdd(o.next_bin, chunk);
      bin = __shfl_sync(0xffffffffu, b0, 0);
      if (bin >= (unsigned long long)o.nbins) break;
      b1 = bin + chunk < o.nbins ? bin + chunk : o.nbins;
    }
    const uint32_t s = o.bin_start[bin], e = o.bin_start[bin + 1];
    if (e <= s + 1u) continue;  // fewer than two registrations
    for (uint32_t i0 = s; i0 < e; i0 += 32u) {
      const uint32_t i = i0 + (uint32_t)lane;
      const bool vi = i < e;
      EntryRec A{};
      if (vi) A = o.rec[i];
      const NarrowA na = narrow_a(A);
      const int nt = (int)min(32u, e - i0);
      // pairs inside the lane's own tile, by rotation: at offset t lane l
      // meets (l + t) mod nt, so every unordered pair comes up once for
      // t < nt / 2 (and at t = nt / 2 from the lower half of the lanes)
      stage(i0, e);
      for (int t = 1; 2 * t <= nt; ++t) {
        int pj = lane + t;
        if (pj >= nt) pj -= nt;
        const bool valid = lane < nt && (2 * t < nt || lane < t);
        const int4 q = sq[wib][pj];
        const int4 mm = sm[wib][pj];
        const bool hit = valid & narrow_test(na, q, mm);
        emit(hit, A.id, (uint32_t)mm.y);
      }
      __syncwarp();
      // later tiles of the bin, staged one at a time and met by every lane
      for (uint32_t j0 = i0 + 32u; j0 < e; j0 += 32u) {
        stage(j0, e);
        const int jn = (int)min(32u, e - j0);
#pragma unroll 2
        for (int jj = 0; jj < jn; ++jj) {
          const int4 q = sq[wib][jj];
          const int4 mm = sm[wib][jj];
          const bool hit = vi & narrow_test(na, q, mm);
          emit(hit, A.id, (uint32_t)mm.y);
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (nbuf > 0) flush_pairs(o, buf, nbuf, lane);
}

// Places every unordered pair into the row of its sphere a (slots taken from
// the partner counts, which this consumes); rows are then sorted by b.
__global__ void k_scatter_pairs(DetectOut o, long long np, uint32_t* __restrict__ pb,
                                int* __restrict__ flags) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const uint2 p = o.upairs[k];
  const uint32_t left = atomicSub(&o.pair_cnt[p.x], 1u);
  if (left == 0u) {  // a broken invariant: never write outside the row
    atomicAdd(&o.pair_cnt[p.x], 1u);
    atomicOr(flags, kFlagBounds);
    return;
  }
  pb[o.pair_off[p.x] + left - 1u] = p.y;
}

// Sorts every row of the new list by b and fills in the row owner a.  A row
// of up to kRowRegs partners (nearly all of them) is loaded at once into
// registers and sorted there by odd-even transposition (kRowRegs rounds of
// compare-exchanges with fixed indices); a longer row is insertion-sorted in
// place.
constexpr int kRowRegs = 8;

__global__ void k_sort_rows(long long ns, const uint32_t* __restrict__ row, int* __restrict__ pa,
                            uint32_t* __restrict__ pb) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ns) return;
  const uint32_t r0 = row[a], r1 = row[a + 1];
  const uint32_t n = r1 - r0;
  if (n == 0) return;
  if (n <= (uint32_t)kRowRegs) {
    uint32_t v[kRowRegs];
#pragma unroll
    for (int k = 0; k < kRowRegs; ++k) v[k] = (uint32_t)k < n ? pb[r0 + k] : 0xffffffffu;
#pragma unroll
    for (int p = 0; p < kRowRegs; ++p) {
#pragma unroll
      for (int k = p & 1; k + 1 < kRowRegs; k += 2) {
        const uint32_t lo = min(v[k], v[k + 1]), hi = max(v[k], v[k + 1]);
        v[k] = lo;
        v[k + 1] = hi;
      }
    }
#pragma unroll
    for (int k = 0; k < kRowRegs; ++k) {
      if ((uint32_t)k < n) {
        pb[r0 + k] = v[k];
        pa[r0 + k] = (int)a;
      }
    }
    return;
  }
  for (uint32_t i = r0 + 1; i < r1; ++i) {
    const uint32_t v = pb[i];
    uint32_t j = i;
    while (j > r0 && pb[j - 1] > v) {
      pb[j] = pb[j - 1];
      --j;
    }
    pb[j] = v;
  }
  for (uint32_t i = r0; i < r1; ++i) pa[i] = (int)a;
}

// The owner clumps and radii of both sides of every pair and its row of the
// pair-material table, so that the force kernel issues all of a pair's pose
// loads at once and reads no per-sphere table.
__global__ void k_pair_owners(DevState d, ContactList l) {
  const long long n = l.dn[0];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int2 sa = d.sinfo[l.pa[i]], sb = d.sinfo[l.pb[i] & ~kHistFlag];
    const float2 ra = d.trm[sa.y], rb = d.trm[sb.y];
    l.pown[i] = make_int4(sa.x, sb.x, __float_as_int(ra.x), __float_as_int(rb.x));
    l.ppm[i] = __float_as_int(ra.y) * d.nmat + __float_as_int(rb.y);
  }
}

// Carries the tangential history of every (a, b) present in the old list
// (binary search of b in the old row of a, which is sorted by b).
__global__ void k_hist_pairs(ContactList oldl, ContactList newl, long long old_ns) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= newl.n) return;
  const int a = newl.pa[i];
  const uint32_t b = newl.pb[i] & ~kHistFlag;
  if (a >= old_ns || oldl.n == 0) return;
  uint32_t lo = oldl.row[a], hi = oldl.row[a + 1];
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((oldl.pb[mid] & ~kHistFlag) < b) lo = mid + 1; else hi = mid;
  }
  if (lo < oldl.row[a + 1]) {
    const uint32_t ob = oldl.pb[lo];
    if ((ob & ~kHistFlag) == b && (ob & kHistFlag)) {
      newl.u[i] = oldl.u[lo];
      newl.u[newl.cap + i] = oldl.u[oldl.cap + lo];
      newl.u[2 * newl.cap + i] = oldl.u[2 * oldl.cap + lo];
      newl.pb[i] = b | kHistFlag;
    }
  }
}

__global__ void k_wall_emit(DevState d, DetectOut o, int* __restrict__ ws, uint32_t* __restrict__ ww) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.ns) return;
  uint32_t mask = o.wall_mask[s];
  if (!mask) return;
  const SceneGrid g = d.grids[d.cinfo[d.sinfo[s].x].y];
  uint32_t off = o.wall_off[s];
  while (mask) {
    const int i = __ffs(mask) - 1;
    mask &= mask - 1;
    ws[off] = (int)s;
    ww[off] = (uint32_t)d.wall_idx[g.wall_start + i];
    ++off;
  }
}

__global__ void k_hist_walls(ContactList oldl, ContactList newl, long long old_ns) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= newl.nw) return;
  const int s = newl.ws[i];
  const uint32_t w = newl.ww[i] & ~kHistFlag;
  if (s >= old_ns || oldl.nw == 0) return;
  for (uint32_t j = oldl.wrow[s]; j < oldl.wrow[s + 1]; ++j) {
    const uint32_t ow = oldl.ww[j];
    if ((ow & ~kHistFlag) == w) {
      if (ow & kHistFlag) {
        newl.uw[i] = oldl.uw[j];
        newl.uw[newl.capw + i] = oldl.uw[oldl.capw + j];
        newl.uw[2 * newl.capw + i] = oldl.uw[2 * oldl.capw + j];
        newl.ww[i] = w | kHistFlag;
      }
      break;
    }
  }
}

// Row pointers of the wall list from the per-sphere offsets.
// Exact missed-contact check: each touching pair of a fresh zero-margin list
// must be present in the current list.
__global__ void k_audit_pairs(DevState d, ContactList cur, long long nf, const int* __restrict__ fa,
                              const uint32_t* __restrict__ fb, unsigned long long* missed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const int a = fa[i];
  const uint32_t b = fb[i] & ~kHistFlag;
  double xa[3], xb[3];
  for (int side = 0; side < 2; ++side) {
    const long long s = side ? (long long)b : (long long)a;
    const int2 si = d.sinfo[s];
    const SceneGrid g = d.grids[d.cinfo[si.x].y];
    double X[3];
    clump_com(d, si.x, g, X);
    const double4_32a q4 = d.cq[si.x];
    const double q[4] = {q4.x, q4.y, q4.z, q4.w};
    const double4_32a tp = d.tp64[si.y];
    const double p[3] = {tp.x, tp.y, tp.z};
    det_centre(q, p, X, side ? xb : xa);
  }
  const double ra = d.tp64[d.sinfo[a].y].w, rb = d.tp64[d.sinfo[b].y].w;
  double dd[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
  const double gap = __dsub_rn(__dsqrt_rn(dot3d(dd, dd)), __dadd_rn(ra, rb));
  if (!(gap < 0.0)) return;
  uint32_t lo = cur.row[a], hi = cur.row[a + 1];
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((cur.pb[mid] & ~kHistFlag) < b) lo = mid + 1; else hi = mid;
  }
  if (!(lo < cur.row[a + 1] && (cur.pb[lo] & ~kHistFlag) == b)) atomicAdd(missed, 1ull);
}

__global__ void k_audit_walls(DevState d, ContactList cur, long long nf, const int* __restrict__ fs,
                              const uint32_t* __restrict__ fw, double t,
                              unsigned long long* missed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const int s = fs[i];
  const uint32_t w = fw[i] & ~kHistFlag;
  const int2 si = d.sinfo[s];
  const SceneGrid g = d.grids[d.cinfo[si.x].y];
  double X[3], x[3], nw[3];
  clump_com(d, si.x, g, X);
  const double4_32a q4 = d.cq[si.x];
  const double q[4] = {q4.x, q4.y, q4.z, q4.w};
  const double4_32a tp = d.tp64[si.y];
  const double p[3] = {tp.x, tp.y, tp.z};
  det_centre(q, p, X, x);
  if (!(wall_distance64(d.walls[w], t, x, nw) < tp.w)) return;
  for (uint32_t j = cur.wrow[s]; j < cur.wrow[s + 1]; ++j)
    if ((cur.ww[j] & ~kHistFlag) == w) return;
  atomicAdd(missed, 1ull);
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_detect(const DevState& d, const DetectOut& o, double margin, const double* smargin,
                   double t, double travel_time, cudaStream_t st) {
  if (d.ns == 0) return;
  if (o.trho) {
    k_tpl_rho<<<(o.n_tsph + 127) / 128, 128, 0, st>>>(d, margin, o.n_tsph, o.trho);
    count_launch();
  }
  { k_detect<<<nblk(d.ns, 128), 128, 0, st>>>(d, o, margin, smargin, t, travel_time); count_launch(); }
}

void launch_rec_ids(const EntryRec* rec, long long n, uint32_t* ids, cudaStream_t st) {
  if (n == 0) return;
  k_rec_ids<<<nblk(n, 256), 256, 0, st>>>(rec, n, ids);
  count_launch();
}

void launch_bin_scatter(const DevState& d, const DetectOut& o, cudaStream_t st) {
  if (d.ns == 0) return;
  { k_bin_scatter<<<nblk(d.ns, 128), 128, 0, st>>>(d, o); count_launch(); }
}

void launch_narrow(const DevState& d, const DetectOut& o, cudaStream_t st) {
  if (d.ns == 0 || o.nbins == 0) return;
  // resident blocks only: the warps take their bins from the counter
  static int occ = 0;
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_narrow_bins, 32 * kNarrowWarps, 0) !=
            cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 4;
    }
  }
  const long long per_block = (long long)kNarrowWarps * (o.chunk > 0 ? o.chunk : kBinChunk);
  const long long want = ((long long)o.nbins + per_block - 1) / per_block;
  const long long cap = (long long)device_sms() * occ;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_narrow_bins<<<grid, 32 * kNarrowWarps, 0, st>>>(o);
  count_launch();
}

void launch_list_rows(const DevState& d, const DetectOut& o, const ContactList& newl,
                      const ContactList* oldl, long long old_ns, cudaStream_t st) {
  if (d.ns == 0) return;
  if (o.np > 0) {
    k_scatter_pairs<<<nblk(o.np, 256), 256, 0, st>>>(o, o.np, newl.pb, d.flags);
    count_launch();
  }
  k_sort_rows<<<nblk(d.ns, 256), 256, 0, st>>>(d.ns, newl.row, newl.pa, newl.pb);
  count_launch();
  if (oldl && oldl->n > 0 && o.np > 0) {
    k_hist_pairs<<<nblk(o.np, 256), 256, 0, st>>>(*oldl, newl, old_ns);
    count_launch();
  }
}

void launch_wall_emit(const DevState& d, const DetectOut& o, int* ws, uint32_t* ww,
                      cudaStream_t st) {
  if (d.ns == 0) return;
  { k_wall_emit<<<nblk(d.ns, 128), 128, 0, st>>>(d, o, ws, ww); count_launch(); }
}

void launch_facet_count(const DevState& d, const DetectOut& o, double t, double travel_time,
                        cudaStream_t st) {
  if (d.nfacets == 0) return;
  k_facet_count<<<(unsigned)d.nfacets, 128, 0, st>>>(d, o, t, travel_time);
  count_launch();
}

void launch_facet_scatter(const DevState& d, const DetectOut& o, double t, double travel_time,
                          cudaStream_t st) {
  if (d.nfacets == 0) return;
  k_facet_scatter<<<(unsigned)d.nfacets, 128, 0, st>>>(d, o, t, travel_time);
  count_launch();
}

void launch_facet_narrow(const DevState& d, const DetectOut& o, double margin, const double* smargin,
                         double t, double travel_time, cudaStream_t st) {
  if (o.nfreg == 0) return;
  const long long warps = o.nfreg;
  const long long cap = (long long)device_sms() * 8;  // 8 blocks of 8 warps per SM
  const long long blocks = std::min((warps + 7) / 8, cap);
  k_facet_narrow<<<(unsigned)blocks, 256, 0, st>>>(d, o, margin, smargin, t, travel_time);
  count_launch();
}

void launch_facet_finish(const DevState& d, const DetectOut& o, long long nf, int* ws, uint32_t* ww,
                         cudaStream_t st) {
  if (nf == 0) return;
  k_facet_emit<<<nblk(nf, 256), 256, 0, st>>>(d, o, nf, ws, ww);
  count_launch();
  k_sort_wall_rows<<<nblk(d.ns, 256), 256, 0, st>>>(d, o, ww);
  count_launch();
}

void launch_add_facet_counts(const DevState& d, const DetectOut& o, cudaStream_t st) {
  if (d.ns == 0) return;
  k_add_facet_counts<<<nblk(d.ns, 256), 256, 0, st>>>(d.ns, o);
  count_launch();
}

void launch_lattice_check(const DevState& d, const DetectOut& o, double margin, const int4* q0,
                          unsigned long long* bad, cudaStream_t st) {
  if (d.ns == 0) return;
  if (o.trho) {
    k_tpl_rho<<<(o.n_tsph + 127) / 128, 128, 0, st>>>(d, margin, o.n_tsph, o.trho);
    count_launch();
  }
  k_lattice_check<<<nblk(d.ns, 128), 128, 0, st>>>(d, o, margin, q0, bad);
  count_launch();
}

void launch_filter_count(const DevState& d, const DetectOut& o, const ContactList& outer,
                         double margin, double t, double travel_time, cudaStream_t st) {
  if (d.ns == 0) return;
  k_filter_pairs<false><<<nblk(d.ns, 128), 128, 0, st>>>(d, o, outer, outer);
  count_launch();
  k_filter_walls<false><<<nblk(d.ns, 128), 128, 0, st>>>(d, o, outer, outer, margin, t, travel_time);
  count_launch();
}

void launch_filter_emit(const DevState& d, const DetectOut& o, const ContactList& outer,
                        const ContactList& inner, double margin, double t, double travel_time,
                        cudaStream_t st) {
  if (d.ns == 0) return;
  k_filter_pairs<true><<<nblk(d.ns, 128), 128, 0, st>>>(d, o, outer, inner);
  count_launch();
  k_filter_walls<true><<<nblk(d.ns, 128), 128, 0, st>>>(d, o, outer, inner, margin, t, travel_time);
  count_launch();
}

void launch_pair_owners(const DevState& d, const ContactList& l, cudaStream_t st) {
  if (l.n > 0 && l.pown && l.ppm) {
    k_pair_owners<<<nblk(l.n, 256), 256, 0, st>>>(d, l);
    count_launch();
  }
}

void launch_hist_pairs(const ContactList& oldl, ContactList& newl, long long old_ns, cudaStream_t st) {
  if (oldl.n > 0 && newl.n > 0) {
    k_hist_pairs<<<nblk(newl.n, 256), 256, 0, st>>>(oldl, newl, old_ns);
    count_launch();
  }
}

void launch_hist_walls(const ContactList& oldl, ContactList& newl, long long old_ns,
                       cudaStream_t st) {
  if (newl.nw > 0) { k_hist_walls<<<nblk(newl.nw, 256), 256, 0, st>>>(oldl, newl, old_ns); count_launch(); }
}

void launch_audit(const DevState& d, const DetectOut& o, const ContactList& cur, long long n_fresh,
                  const int* fa, const uint32_t* fb, long long nw_fresh, const int* fws,
                  const uint32_t* fww, double t, unsigned long long* d_missed, cudaStream_t st) {
  (void)o;
  if (n_fresh > 0) { k_audit_pairs<<<nblk(n_fresh, 128), 128, 0, st>>>(d, cur, n_fresh, fa, fb, d_missed); count_launch(); }
  if (nw_fresh > 0)
    { k_audit_walls<<<nblk(nw_fresh, 128), 128, 0, st>>>(d, cur, nw_fresh, fws, fww, t, d_missed); count_launch(); }
}

}  // namespace dem
