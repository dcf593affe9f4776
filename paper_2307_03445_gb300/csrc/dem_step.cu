// dem_step.cu -- per-step kernels: contact forces and clump update.
//
// Force kernels run one thread per listed contact (grid-stride, persistent
// grid).  A listed contact whose overlap is not positive is a false positive
// of the enlarged list and contributes nothing (section 2.2); its history is
// dropped by clearing a flag bit instead of rewriting it.  Active contacts
// evaluate Eq. (2) (kinematics), Eq. (3) (history update), Eq. (1) (forces)
// and Eq. (4) (cap), and add +F to body b and -F to body a together with the
// moments of F about each centre of mass (vector reductions into float
// accumulators in FP32_VOXEL, double atomics in FP64).
//
// The update kernel integrates Eq. (5) for a block of clumps, then, with the
// new orientation held as a float-float rotation matrix in shared memory,
// recomputes the pose records of all spheres of those clumps.
//
// FP32_VOXEL specifics: the pair kernel takes each pair's owners, radii and
// pair-material row from the list's per-pair record (written at the
// rebuild) and keeps the tangential history as float-float; the update
// kernel keeps a per-clump motion bound since the last rebuild, which decides
// when the exact displacement certificate has to read that rebuild's state.
#include <algorithm>

#include "dem_dev.cuh"
#include "dem_prims.cuh"
#include "dem_walls.cuh"

namespace dem {

namespace {

template <typename T>
struct Law {
  V3<T> F;    // force on body b
  V3<T> u;    // capped: the new history; otherwise the increment to add
  bool capped;
};

// Division and square root inside the contact law.  FP64: IEEE.  FP32: the
// hardware approximations (a reciprocal times the dividend; a square root as
// x times its reciprocal square root), a few 1e-7 relative, far inside the
// float path's 1e-5 bar, without the IEEE special-case code of '/' and sqrtf.
__device__ __forceinline__ double cdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float cdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double csqrt_pos(double x) { return sqrt(x); }
__device__ __forceinline__ float csqrt_pos(float x) { return x * rsqrtf(x); }  // x > 0

// Eq. (2b)-(4) for one active contact: n from a to b, dn > 0, vrel = velocity
// of b minus velocity of a at the contact point, u the stored history.
template <typename T>
__device__ __forceinline__ Law<T> contact_law(const PairMat<T>& pm, T h, V3<T> n, T dn, V3<T> vrel,
                                              V3<T> u, T Rbar, T mbar) {
  Law<T> r;
  const T vns = dot(vrel, n);
  const V3<T> vt = vrel - vns * n;                  // Eq. (2b), (2c)
  const V3<T> up = u + h * vt;                      // Eq. (3)
  const T upn = dot(up, n);
  const V3<T> upt = up - upn * n;
  const T f = csqrt_pos(Rbar * dn);                 // Eq. (1c)
  const T sfm = csqrt_pos(f * mbar);
  const T fns = f * pm.kn * dn - pm.cn * sfm * vns; // Eq. (1a) along n
  const V3<T> Ft = (-f * pm.kt) * upt - (pm.ct * sfm) * vt;  // Eq. (1b)
  const T fn = fabs(fns), ft2 = dot(Ft, Ft);
  // Eq. (4): FP64 compares |F_t| itself (the oracle's order); float compares
  // the squares and scales with a reciprocal square root
  bool cap;
  T s;
  if constexpr (sizeof(T) == 4) {
    const T lim = pm.mu * fn;
    cap = ft2 > lim * lim;
    s = cap ? lim * rsqrtf(ft2) : T(1);
  } else {
    const T ft = sqrt(ft2);
    cap = ft > pm.mu * fn;
    s = cap && ft > T(0) ? cdiv(pm.mu * fn, ft) : T(0);
  }
  if (cap) {
    const T ul = sqrt(dot(upt, upt));
    const T us = ul > T(0) ? cdiv(cdiv(pm.mu * fn, f * pm.kt), ul) : T(0);
    r.F = fns * n + s * Ft;
    r.u = us * upt;
    r.capped = true;
  } else {
    r.F = fns * n + Ft;
    r.u = h * vt - upn * n;  // u' - u
    r.capped = false;
  }
  return r;
}

__device__ __forceinline__ void warp_count(bool active, unsigned long long* ctr) {
  const unsigned m = __activemask();
  const unsigned b = __ballot_sync(m, active);
  if ((threadIdx.x & 31) == __ffs(m) - 1 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

__device__ __forceinline__ void add_clump64(double* acc, int c, V3<double> F, V3<double> T) {
  double* p = acc + 8 * (long long)c;
  atomicAdd(p + 0, F.x); atomicAdd(p + 1, F.y); atomicAdd(p + 2, F.z);
  atomicAdd(p + 3, T.x); atomicAdd(p + 4, T.y); atomicAdd(p + 5, T.z);
}
__device__ __forceinline__ void add_clump32(float* acc, int c, V3<float> F, V3<float> T) {
  float* p = acc + 8 * (long long)c;
  red_add_v4(p, F.x, F.y, F.z, T.x);
  red_add_v2(p + 4, T.y, T.z);
}

// ---------------------------------------------------------------------------
// sphere-sphere contacts
// ---------------------------------------------------------------------------
// One side of an FP32_VOXEL sphere-wall contact: the sphere's fixed-point
// centre, radius, material, owner and the owner's voxel offset.
struct Side32 {
  long long P[3];
  float r;
  int owner, tsph;
  float4 off;
  long long rel[3];  // centre from the owner's voxel corner (the pose record)
};

// Loads of one side, in two dependent rounds: the static {owner, template
// sphere} pair and the pose record, then the owner's voxel and offset and the
// template sphere's radius.
__device__ __forceinline__ Side32 load_side32(const DevState& d, uint32_t s) {
  Side32 S;
  const int2 si = d.sinfo[s];
  const uint4 rec = d.srec32[s];
  S.owner = si.x;
  S.tsph = si.y;
  const int4 v = d.cvox[si.x];
  S.off = d.coff[si.x];
  S.r = d.tp32[si.y].w;
  unpack_rel(rec, S.rel[0], S.rel[1], S.rel[2]);
  S.P[0] = ((long long)v.x << (kFixBits - kVoxLog2)) + S.rel[0];
  S.P[1] = ((long long)v.y << (kFixBits - kVoxLog2)) + S.rel[1];
  S.P[2] = ((long long)v.z << (kFixBits - kVoxLog2)) + S.rel[2];
  return S;
}

// Lever arm R p of a side (float): its centre from the voxel corner minus the
// clump's offset in the voxel.
__device__ __forceinline__ V3<float> arm32(const Side32& S) {
  return {fix_to_float(S.rel[0]) - S.off.x, fix_to_float(S.rel[1]) - S.off.y,
          fix_to_float(S.rel[2]) - S.off.z};
}

// One side of an FP32_VOXEL sphere pair, as the pair kernel uses it: the
// owner's voxel, the centre from that voxel's corner (the pose record), the
// radius and owner.  The centre difference of two sides is
// ((voxel_b - voxel_a) << 24) + (rel_b - rel_a), in 2^-44 m.  With the owner
// and radius taken from the list's per-pair record, the two loads of a side
// depend on the pair alone and issue together.
struct PairSide32 {
  int vx, vy, vz;
  int owner;
  float r;
  long long rel[3];
};

__device__ __forceinline__ PairSide32 load_pair_side32(const DevState& d, uint32_t s, int owner,
                                                       float r) {
  PairSide32 S;
  const uint4 rec = d.srec32[s];
  S.owner = owner;
  const int4 v = d.cvox[owner];
  S.vx = v.x; S.vy = v.y; S.vz = v.z;
  S.r = r;
  unpack_rel(rec, S.rel[0], S.rel[1], S.rel[2]);
  return S;
}

__device__ __forceinline__ long long fix_diff(int va, int vb, long long ra, long long rb) {
  return (long long)(vb - va) * (1ll << (kFixBits - kVoxLog2)) + (rb - ra);
}

// Lever arm R p of a pair side: its centre from the voxel corner minus the
// owner's offset in the voxel.
__device__ __forceinline__ V3<float> arm32(const PairSide32& S, float4 off) {
  return {fix_to_float(S.rel[0]) - off.x, fix_to_float(S.rel[1]) - off.y,
          fix_to_float(S.rel[2]) - off.z};
}

// Tangential history of an FP32_VOXEL pair contact: each component a
// float-float (high, low) in the 8 bytes of its slot, the high part the
// component rounded to float.  The float increment of Eq. (3) is added
// without rounding away its low bits (TwoSum), as a double sum would.
__device__ __forceinline__ float2 hist_add(float2 u, float inc) {
  const ff s = two_sum(u.x, inc);
  const ff r = fast_two_sum(s.h, __fadd_rn(s.l, u.y));
  return make_float2(r.h, r.l);
}

// Eq. (1)-(5) for one active sphere pair of the FP32_VOXEL list: forces, the
// history update, and the force and moments added to both clumps.
__device__ __forceinline__ void pair_force32(const DevState& d, ContactList& l, long long i,
                                             uint32_t b, uint32_t bw, const PairSide32& A,
                                             const PairSide32& B, int pmi, float fx, float fy,
                                             float fz, float dist, float dn) {
    const float inv = __fdividef(1.f, dist);
    const V3<float> n = {fx * inv, fy * inv, fz * inv};
    const float4 va = d.mv32[A.owner], wa = d.mw32[A.owner];
    const float4 vb = d.mv32[B.owner], wb = d.mw32[B.owner];
    const float4 offa = d.coff[A.owner], offb = d.coff[B.owner];
    float2* uf = reinterpret_cast<float2*>(l.u);
    float2 u0 = make_float2(0.f, 0.f), u1 = u0, u2 = u0;
    if (bw & kHistFlag) {
      u0 = uf[i];
      u1 = uf[l.cap + i];
      u2 = uf[2 * l.cap + i];
    }
    const float sa = A.r - 0.5f * dn, sb = B.r - 0.5f * dn;
    const V3<float> ca = arm32(A, offa) + sa * n;
    const V3<float> cb = arm32(B, offb) - sb * n;
    const V3<float> vA = V3<float>{va.x, va.y, va.z} + cross(V3<float>{wa.x, wa.y, wa.z}, ca);
    const V3<float> vB = V3<float>{vb.x, vb.y, vb.z} + cross(V3<float>{wb.x, wb.y, wb.z}, cb);
    const PairMat<float> pm = d.pm32[pmi];
    const float Rbar = __fdividef(A.r * B.r, A.r + B.r);
    const float mbar = __fdividef(va.w * vb.w, va.w + vb.w);
    const Law<float> law = contact_law<float>(pm, d.hf, n, dn, vB - vA,
                                              V3<float>{u0.x, u1.x, u2.x}, Rbar, mbar);
    if (law.capped) {
      u0 = make_float2(law.u.x, 0.f); u1 = make_float2(law.u.y, 0.f);
      u2 = make_float2(law.u.z, 0.f);
    } else {
      u0 = hist_add(u0, law.u.x); u1 = hist_add(u1, law.u.y); u2 = hist_add(u2, law.u.z);
    }
    uf[i] = u0;
    uf[l.cap + i] = u1;
    uf[2 * l.cap + i] = u2;
    if (!(bw & kHistFlag)) l.pb[i] = b | kHistFlag;
    const V3<float> F = law.F;
    const V3<float> Ta = -1.f * cross(ca, F), Tb = cross(cb, F);
    if (d.det_off) {
      d.det_pair32[3 * i] = make_float4(F.x, F.y, F.z, 0.f);
      d.det_pair32[3 * i + 1] = make_float4(Ta.x, Ta.y, Ta.z, 0.f);
      d.det_pair32[3 * i + 2] = make_float4(Tb.x, Tb.y, Tb.z, 0.f);
    } else {
      add_clump32(d.acc32, B.owner, F, Tb);
      add_clump32(d.acc32, A.owner, -1.f * F, Ta);
    }
}

__global__ void __launch_bounds__(256) k_pairs32(DevState d, ContactList l, int count_active) {
  if (halted(d)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long ln = l.dn[0];
  // software pipeline: the ids and per-pair record of the next pair are
  // loaded one iteration ahead, so that the loads of an iteration (pose
  // records and voxels of both sides) issue together at its start.  (L2
  // prefetches of the next pair's pose records cost more load-unit requests
  // than the latency they saved.)
  long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int a_n = 0;
  uint32_t bw_n = 0;
  int4 own_n = make_int4(0, 0, 0, 0);
  int pm_n = 0;
  if (i0 < ln) { a_n = l.pa[i0]; bw_n = l.pb[i0]; own_n = l.pown[i0]; pm_n = l.ppm[i0]; }
  for (long long i = i0; i < ln; i += stride) {
    const int a = a_n;
    const uint32_t bw = bw_n;
    const uint32_t b = bw & ~kHistFlag;
    const int4 own = own_n;
    const int pmi = pm_n;
    if (i + stride < ln) {
      a_n = l.pa[i + stride]; bw_n = l.pb[i + stride]; own_n = l.pown[i + stride];
      pm_n = l.ppm[i + stride];
    }
    const PairSide32 A = load_pair_side32(d, (uint32_t)a, own.x, __int_as_float(own.z));
    const PairSide32 B = load_pair_side32(d, b, own.y, __int_as_float(own.w));
    // the centre difference b - a as exact float-float metres; its high
    // parts are the float estimate used for the cheap rejection
    const ff dx = fix_to_ff_near(fix_diff(A.vx, B.vx, A.rel[0], B.rel[0]));
    const ff dy = fix_to_ff_near(fix_diff(A.vy, B.vy, A.rel[1], B.rel[1]));
    const ff dz = fix_to_ff_near(fix_diff(A.vz, B.vz, A.rel[2], B.rel[2]));
    const float fx = dx.h, fy = dy.h, fz = dz.h;
    // cheap rejection of clear false positives
    const float s_est = fx * fx + fy * fy + fz * fz;
    const float rs = A.r + B.r;
    float dn = -1.f;
    float dist = 0.f;
    if (s_est <= rs * rs * 1.0001f) {
      // overlap rho - |d| = (rho^2 - |d|^2) / (rho + |d|), numerator in float-float
      const ff s = ff_add(ff_add(ff_mul(dx, dx), ff_mul(dy, dy)), ff_mul(dz, dz));
      const ff rho = two_sum(A.r, B.r);
      const ff diff = ff_sub(ff_mul(rho, rho), s);
      dist = csqrt_pos(s.h);
      dn = __fdividef(ff_to_float(diff), ff_to_float(rho) + dist);
    }
    const bool active = dn > 0.f;
    if (count_active) warp_count(active, d.counters);
    if (!active) {
      if (bw & kHistFlag) l.pb[i] = b;  // history reset (false positive)
      if (d.det_off) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        d.det_pair32[3 * i] = z; d.det_pair32[3 * i + 1] = z; d.det_pair32[3 * i + 2] = z;
      }
    } else {
      pair_force32(d, l, i, b, bw, A, B, pmi, fx, fy, fz, dist, dn);
    }
    // the lanes of a warp take the next pair together
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) k_pairs64(DevState d, ContactList l, int count_active) {
  if (halted(d)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long ln = l.dn[0];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ln; i += stride) {
    const int a = l.pa[i];
    const uint32_t bw = l.pb[i];
    const uint32_t b = bw & ~kHistFlag;
    const SphA64 A = d.sa64[a];
    const SphA64 B = d.sa64[b];
    const V3<double> dv = {B.x - A.x, B.y - A.y, B.z - A.z};
    const double dist = sqrt(dot(dv, dv));
    const double dn = (A.r + B.r) - dist;
    const bool active = dn > 0.0;
    if (count_active) warp_count(active, d.counters);
    if (!active) {
      if (bw & kHistFlag) l.pb[i] = b;
      if (d.det_off) {
        const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        d.det_pair64[3 * i] = z; d.det_pair64[3 * i + 1] = z; d.det_pair64[3 * i + 2] = z;
      }
      continue;
    }
    const V3<double> n = (1.0 / dist) * dv;
    const double4_32a RA = d.sb64[a], RB = d.sb64[b];
    const long long ia = __double_as_longlong(RA.w), ib = __double_as_longlong(RB.w);
    const int oa = (int)(ia & 0xffffffff), ob = (int)(ib & 0xffffffff);
    const int ma = (int)(ia >> 32), mb = (int)(ib >> 32);
    const double4_32a va = d.mv64[oa], wa = d.mw64[oa], vb = d.mv64[ob], wb = d.mw64[ob];
    const double sa = A.r - 0.5 * dn, sb = B.r - 0.5 * dn;
    const V3<double> ca = V3<double>{RA.x, RA.y, RA.z} + sa * n;
    const V3<double> cb = V3<double>{RB.x, RB.y, RB.z} - sb * n;
    const V3<double> vA = V3<double>{va.x, va.y, va.z} + cross(V3<double>{wa.x, wa.y, wa.z}, ca);
    const V3<double> vB = V3<double>{vb.x, vb.y, vb.z} + cross(V3<double>{wb.x, wb.y, wb.z}, cb);
    V3<double> u = {0.0, 0.0, 0.0};
    if (bw & kHistFlag) u = {l.u[i], l.u[l.cap + i], l.u[2 * l.cap + i]};
    const PairMat<double> pm = d.pm64[ma * d.nmat + mb];
    const double Rbar = A.r * B.r / (A.r + B.r);
    const double mbar = va.w * vb.w / (va.w + vb.w);
    const Law<double> law = contact_law<double>(pm, d.h, n, dn, vB - vA, u, Rbar, mbar);
    const V3<double> un = law.capped ? law.u : u + law.u;
    l.u[i] = un.x;
    l.u[l.cap + i] = un.y;
    l.u[2 * l.cap + i] = un.z;
    if (!(bw & kHistFlag)) l.pb[i] = b | kHistFlag;
    const V3<double> Ta = -1.0 * cross(ca, law.F), Tb = cross(cb, law.F);
    if (d.det_off) {
      d.det_pair64[3 * i] = make_double4_32a(law.F.x, law.F.y, law.F.z, 0.0);
      d.det_pair64[3 * i + 1] = make_double4_32a(Ta.x, Ta.y, Ta.z, 0.0);
      d.det_pair64[3 * i + 2] = make_double4_32a(Tb.x, Tb.y, Tb.z, 0.0);
    } else {
      add_clump64(d.acc64, ob, law.F, Tb);
      add_clump64(d.acc64, oa, -1.0 * law.F, Ta);
    }
  }
}

// ---------------------------------------------------------------------------
// sphere-wall contacts (body a = the sphere's clump, body b = the wall)
// ---------------------------------------------------------------------------
// Net force on each wall: summed per block in shared memory, then one global
// double atomic per wall component per block (all contacts of a wall would
// otherwise serialise on the same three addresses).  Walls past the first
// kMaxBlockWalls (the facets of large meshes, each touched by few spheres)
// add straight to global memory.
constexpr int kMaxBlockWalls = 256;

__device__ __forceinline__ void wall_force_flush(const DevState& d, const float* s_wf,
                                                 const float* s_wt) {
  __syncthreads();
  const int nw = d.nwalls < kMaxBlockWalls ? d.nwalls : kMaxBlockWalls;
  for (int i = threadIdx.x; i < 3 * nw; i += blockDim.x) {
    if (s_wf[i] != 0.f) atomicAdd(d.wforce + i, (double)s_wf[i]);
    if (s_wt[i] != 0.f) atomicAdd(d.wtorque + i, (double)s_wt[i]);
  }
}

__global__ void k_walls32(DevState d, ContactList l, int count_active) {
  if (halted(d)) return;
  __shared__ float s_wf[3 * kMaxBlockWalls];  // force on each wall
  __shared__ float s_wt[3 * kMaxBlockWalls];  // its moment about the wall's reference point
  for (int i = threadIdx.x; i < 3 * kMaxBlockWalls; i += blockDim.x) s_wf[i] = s_wt[i] = 0.f;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long lnw = l.dn[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < lnw; i += stride) {
    const int s = l.ws[i];
    const uint32_t wwv = l.ww[i];
    const uint32_t w = wwv & ~kHistFlag;
    const Side32 S = load_side32(d, (uint32_t)s);
    const WallDev& W = d.walls[w];
    V3<float> n;
    const float dn = wall_geom32(W, d.wfix + 3 * (long long)w, S.P[0], S.P[1], S.P[2], S.r, n);
    const bool active = dn > 0.f;
    if (count_active) warp_count(active, d.counters);
    if (!active) {
      if (wwv & kHistFlag) l.ww[i] = w;
      if (d.det_off) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        d.det_wall32[2 * i] = z; d.det_wall32[2 * i + 1] = z;
      }
      continue;
    }
    const float4 va = d.mv32[S.owner], wa = d.mw32[S.owner];
    const V3<float> ca = arm32(S) + (S.r - 0.5f * dn) * n;
    const V3<float> vA = V3<float>{va.x, va.y, va.z} + cross(V3<float>{wa.x, wa.y, wa.z}, ca);
    const V3<float> vW = {W.vf[0], W.vf[1], W.vf[2]};
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
    if (wwv & kHistFlag) {
      u0 = l.uw[i];
      u1 = l.uw[l.capw + i];
      u2 = l.uw[2 * l.capw + i];
    }
    const PairMat<float> pm = d.pm32[d.tmat[S.tsph] * d.nmat + W.material];
    const Law<float> law = contact_law<float>(pm, d.hf, n, dn, vW - vA,
                                              V3<float>{d2f(u0), d2f(u1), d2f(u2)}, S.r, va.w);
    if (law.capped) {
      u0 = f2d(law.u.x); u1 = f2d(law.u.y); u2 = f2d(law.u.z);
    } else {
      u0 += f2d(law.u.x); u1 += f2d(law.u.y); u2 += f2d(law.u.z);
    }
    l.uw[i] = u0;
    l.uw[l.capw + i] = u1;
    l.uw[2 * l.capw + i] = u2;
    if (!(wwv & kHistFlag)) l.ww[i] = w | kHistFlag;
    const V3<float> Fs = -1.f * law.F, Ts = -1.f * cross(ca, law.F);
    if (d.det_off) {
      d.det_wall32[2 * i] = make_float4(Fs.x, Fs.y, Fs.z, 0.f);
      d.det_wall32[2 * i + 1] = make_float4(Ts.x, Ts.y, Ts.z, 0.f);
    } else {
      add_clump32(d.acc32, S.owner, Fs, Ts);
    }
    // moment about the wall's reference point (fixed point, like the sphere
    // centre), the force acting at the contact point
    const long long* wf = d.wfix + 3 * (long long)w;
    const V3<float> rw = V3<float>{fix_to_float(S.P[0] - wf[0]), fix_to_float(S.P[1] - wf[1]),
                                   fix_to_float(S.P[2] - wf[2])} + (S.r - 0.5f * dn) * n;
    const V3<float> tw = cross(rw, law.F);
    if (w < (uint32_t)kMaxBlockWalls) {
      atomicAdd(&s_wf[3 * w], law.F.x);
      atomicAdd(&s_wf[3 * w + 1], law.F.y);
      atomicAdd(&s_wf[3 * w + 2], law.F.z);
      atomicAdd(&s_wt[3 * w], tw.x);
      atomicAdd(&s_wt[3 * w + 1], tw.y);
      atomicAdd(&s_wt[3 * w + 2], tw.z);
    } else {
      double* fw = d.wforce + 3 * (long long)w;
      atomicAdd(fw, (double)law.F.x);
      atomicAdd(fw + 1, (double)law.F.y);
      atomicAdd(fw + 2, (double)law.F.z);
      double* mw = d.wtorque + 3 * (long long)w;
      atomicAdd(mw, (double)tw.x);
      atomicAdd(mw + 1, (double)tw.y);
      atomicAdd(mw + 2, (double)tw.z);
    }
  }
  wall_force_flush(d, s_wf, s_wt);
}

__global__ void k_walls64(DevState d, ContactList l, int count_active) {
  if (halted(d)) return;
  const double t = (double)(*d.dstep) * d.h;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long lnw = l.dn[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < lnw; i += stride) {
    const int s = l.ws[i];
    const uint32_t wwv = l.ww[i];
    const uint32_t w = wwv & ~kHistFlag;
    const SphA64 S = d.sa64[s];
    const WallDev& W = d.walls[w];
    const double x[3] = {S.x, S.y, S.z};
    double nw[3];
    const double dist = wall_distance64(W, t, x, nw);
    const double dn = S.r - dist;
    const bool active = dn > 0.0;
    if (count_active) warp_count(active, d.counters);
    if (!active) {
      if (wwv & kHistFlag) l.ww[i] = w;
      if (d.det_off) {
        const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        d.det_wall64[2 * i] = z; d.det_wall64[2 * i + 1] = z;
      }
      continue;
    }
    const V3<double> n = {-nw[0], -nw[1], -nw[2]};
    const double4_32a RS = d.sb64[s];
    const long long is = __double_as_longlong(RS.w);
    const int os = (int)(is & 0xffffffff), ms = (int)(is >> 32);
    const double4_32a va = d.mv64[os], wa = d.mw64[os];
    const V3<double> ca = V3<double>{RS.x, RS.y, RS.z} + (S.r - 0.5 * dn) * n;
    const V3<double> vA = V3<double>{va.x, va.y, va.z} + cross(V3<double>{wa.x, wa.y, wa.z}, ca);
    const V3<double> vW = {W.vel[0], W.vel[1], W.vel[2]};
    V3<double> u = {0.0, 0.0, 0.0};
    if (wwv & kHistFlag) u = {l.uw[i], l.uw[l.capw + i], l.uw[2 * l.capw + i]};
    const PairMat<double> pm = d.pm64[ms * d.nmat + W.material];
    const Law<double> law = contact_law<double>(pm, d.h, n, dn, vW - vA, u, S.r, va.w);
    const V3<double> un = law.capped ? law.u : u + law.u;
    l.uw[i] = un.x;
    l.uw[l.capw + i] = un.y;
    l.uw[2 * l.capw + i] = un.z;
    if (!(wwv & kHistFlag)) l.ww[i] = w | kHistFlag;
    const V3<double> Fs = -1.0 * law.F, Ts = -1.0 * cross(ca, law.F);
    if (d.det_off) {
      d.det_wall64[2 * i] = make_double4_32a(Fs.x, Fs.y, Fs.z, 0.0);
      d.det_wall64[2 * i + 1] = make_double4_32a(Ts.x, Ts.y, Ts.z, 0.0);
    } else {
      add_clump64(d.acc64, os, Fs, Ts);
    }
    double* fw = d.wforce + 3 * (long long)w;
    atomicAdd(fw, law.F.x);
    atomicAdd(fw + 1, law.F.y);
    atomicAdd(fw + 2, law.F.z);
    // moment about the wall's reference point p + v t, the force acting at
    // the contact point
    const V3<double> rw = V3<double>{x[0] - (W.p[0] + W.vel[0] * t), x[1] - (W.p[1] + W.vel[1] * t),
                                     x[2] - (W.p[2] + W.vel[2] * t)} + (S.r - 0.5 * dn) * n;
    const V3<double> tw = cross(rw, law.F);
    double* mw = d.wtorque + 3 * (long long)w;
    atomicAdd(mw, tw.x);
    atomicAdd(mw + 1, tw.y);
    atomicAdd(mw + 2, tw.z);
  }
}

// ---------------------------------------------------------------------------
// clump update: Eq. (5) + sphere poses
// ---------------------------------------------------------------------------
constexpr int kUpd = 128;

__device__ __forceinline__ void quat_mul(const double a[4], const double b[4], double c[4]) {
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}
__device__ __forceinline__ void quat_mulf(const float a[4], const float b[4], float c[4]) {
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

__device__ __forceinline__ bool finite4(double4_32a v) {
  return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

// FP64 mode.
__global__ void __launch_bounds__(kUpd) k_update64(DevState d, int integrate, float margin,
                                                   int check_cert) {
  if (integrate && halted(d)) return;
  __shared__ double sR[kUpd][9];
  __shared__ double sX[kUpd][3];
  const long long c0 = (long long)blockIdx.x * kUpd;
  const long long c = c0 + threadIdx.x;
  if (c < d.ncl) {
    const int tpl = d.cinfo[c].x;
    double4_32a X = d.cpos[c], q4 = d.cq[c], v, w;
    load_vel(d.cvw + c, v, w);
    const double mass = d.tmass[tpl];
    const double I[3] = {d.tinert[3 * tpl], d.tinert[3 * tpl + 1], d.tinert[3 * tpl + 2]};
    double q[4] = {q4.x, q4.y, q4.z, q4.w};
    double R[9];
    if (integrate) {
      double* acc = d.acc64 + 8 * c;
      const V3<double> F = {acc[0], acc[1], acc[2]}, T = {acc[3], acc[4], acc[5]};
      for (int k = 0; k < 6; ++k) acc[k] = 0.0;
      const double h = d.h;
      if (d.alast) d.alast[c] = (float)(sqrt(F.x * F.x + F.y * F.y + F.z * F.z) / mass);
      // Eq. (5a), semi-implicit Euler
      v.x += h * (F.x / mass + d.g[0]);
      v.y += h * (F.y / mass + d.g[1]);
      v.z += h * (F.z / mass + d.g[2]);
      X.x += h * v.x; X.y += h * v.y; X.z += h * v.z;
      // Eq. (5b) in the principal frame with the gyroscopic term
      quat_to_mat(q[0], q[1], q[2], q[3], R);
      const V3<double> tb = mat_tmul(R, T);
      const V3<double> wb = {w.x, w.y, w.z};
      const V3<double> Iw = {I[0] * wb.x, I[1] * wb.y, I[2] * wb.z};
      const V3<double> gy = cross(wb, Iw);
      w.x += h * (tb.x - gy.x) / I[0];
      w.y += h * (tb.y - gy.y) / I[1];
      w.z += h * (tb.z - gy.z) / I[2];
      const double wl = sqrt(w.x * w.x + w.y * w.y + w.z * w.z);
      double dq[4] = {1.0, 0.0, 0.0, 0.0};
      if (wl > 0.0) {
        double sn, cs;
        sincos(0.5 * h * wl, &sn, &cs);
        const double sc = sn / wl;
        dq[0] = cs; dq[1] = sc * w.x; dq[2] = sc * w.y; dq[3] = sc * w.z;
      }
      double qn[4];
      quat_mul(q, dq, qn);
      const double ql = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
      for (int k = 0; k < 4; ++k) q[k] = qn[k] / ql;
      q4 = make_double4_32a(q[0], q[1], q[2], q[3]);
      if (!(finite4(X) && finite4(v) && finite4(w) && finite4(q4))) atomicOr(d.flags, kFlagNonFinite);
      d.cpos[c] = X; d.cq[c] = q4;
      store_vel(d.cvw + c, v, w);
      if (check_cert) {
        const double4_32a X0 = d.ref_pos[c];
        const float4 r0 = d.ref_q[c];
        const float dx = (float)(X.x - X0.x), dy = (float)(X.y - X0.y), dz = (float)(X.z - X0.z);
        // |vec(conj(q0) q)| = sin(angle / 2)
        const float a[4] = {r0.x, -r0.y, -r0.z, -r0.w};
        const float b[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
        float e[4];
        quat_mulf(a, b, e);
        const float disp = sqrtf(dx * dx + dy * dy + dz * dz) +
                           2.f * d.tpbound[tpl] * sqrtf(e[1] * e[1] + e[2] * e[2] + e[3] * e[3]);
        const float mlim = d.cmargin ? d.cmargin[c] : margin;
        if (disp * 1.00001f + 1e-12f > mlim) {
          atomicOr(d.flags, kFlagGuard);
          atomicAdd(d.counters + 1, 1ull);
          // the state of step *dstep + 1 may lack a listed contact
          if (d.halt_at) atomicMin(reinterpret_cast<unsigned long long*>(d.halt_at),
                                   (unsigned long long)(*d.dstep + 1));
        }
      }
    }
    quat_to_mat(q[0], q[1], q[2], q[3], R);
    const V3<double> ww = mat_mul(R, V3<double>{w.x, w.y, w.z});
    d.mv64[c] = make_double4_32a(v.x, v.y, v.z, mass);
    d.mw64[c] = make_double4_32a(ww.x, ww.y, ww.z, 0.0);
    for (int k = 0; k < 9; ++k) sR[threadIdx.x][k] = R[k];
    sX[threadIdx.x][0] = X.x; sX[threadIdx.x][1] = X.y; sX[threadIdx.x][2] = X.z;
  }
  __syncthreads();
  const long long c1 = c0 + kUpd < d.ncl ? c0 + kUpd : d.ncl;
  if (c0 >= c1) return;
  const long long s0 = d.csph[c0], s1 = d.csph[c1];
  for (long long s = s0 + threadIdx.x; s < s1; s += kUpd) {
    const int2 si = d.sinfo[s];
    const int lc = (int)(si.x - c0);
    const double4_32a tp = d.tp64[si.y];
    const V3<double> rel = mat_mul(sR[lc], V3<double>{tp.x, tp.y, tp.z});
    SphA64 A;
    A.x = sX[lc][0] + rel.x; A.y = sX[lc][1] + rel.y; A.z = sX[lc][2] + rel.z; A.r = tp.w;
    d.sa64[s] = A;
    const long long bits = (long long)(uint32_t)si.x | ((long long)d.tmat[si.y] << 32);
    d.sb64[s] = make_double4_32a(rel.x, rel.y, rel.z, __longlong_as_double(bits));
  }
}

// FP32_VOXEL mode, in two phases per warp of 32 clumps.  Phase 1: one thread
// per clump integrates Eq. (5) and forms its float-float rotation matrix;
// the matrix, the clump's offset in fixed point and its sphere range go to
// the warp's slice of shared memory.  Phase 2: the warp's lanes take the
// warp's spheres in order (consecutive records: coalesced 16-byte stores),
// each finding its clump by a binary search of the sphere ranges, and write
// the pose records.  Only __syncwarp between the phases; no block barrier.
// INTEG = false recomputes poses and mirrors from the state; CERT adds the
// displacement certificate.  B (64, 128 or 256 clumps per block) is a launch
// shape the tile autotuner picks.
struct WarpPoses {
  float Rh[9][32], Rl[9][32];  // rotation matrix (float-float), [entry][lane]
  int off[3][32];              // offset in the voxel, 2^-44 m units
  int s0[33];                  // first sphere of each clump; s0[n] = end of the warp's spheres
  int t0[32];                  // first template sphere of each clump's template
};

// (the register cap lets 7 blocks of 128 or 3 of 256 clumps share an SM:
// 43.75 % occupancy at 128, measured 3 % faster than the uncapped 80 registers)
template <int B, bool INTEG, bool CERT>
__global__ void __launch_bounds__(B, 896 / B) k_update32(DevState d, float margin) {
  if (INTEG && halted(d)) return;
  __shared__ WarpPoses sh[B / 32];
  const int lane = threadIdx.x & 31;
  WarpPoses& wp = sh[threadIdx.x >> 5];
  const long long cw0 = (long long)blockIdx.x * B + (threadIdx.x & ~31);  // the warp's first clump
  if (cw0 >= d.ncl) return;  // the whole warp
  const int nw = (int)(d.ncl - cw0 < 32 ? d.ncl - cw0 : 32);
  const long long c = cw0 + lane;
  if (lane < nw) {
    // every global load of the clump is issued first (one memory round trip)
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    if (INTEG) {
      a0 = *reinterpret_cast<const float4*>(d.acc32 + 8 * c);
      a1 = *reinterpret_cast<const float4*>(d.acc32 + 8 * c + 4);
    }
    const int tpl = d.cinfo[c].x;
    int4 vox = d.cvox[c];
    float4 off = d.coff[c];
    double4_32a q4 = d.cq[c], v, w;
    load_vel(d.cvw + c, v, w);
    const float2 mim = *reinterpret_cast<const float2*>(d.tmassf + 2 * tpl);  // m, 1/m
    const float mass = mim.x;
    // orientation as float-float; integrating needs only the high parts of
    // the old one (the rotation matrix is built from the new orientation)
    ff qw, qx, qy, qz;
    V3<float> wf_new;  // the new angular velocity as float (integrating)
    float vf_new[3];   // the new velocity as float (integrating)
    if (INTEG) {
      qw = {d2f(q4.x), 0.f}; qx = {d2f(q4.y), 0.f}; qy = {d2f(q4.z), 0.f}; qz = {d2f(q4.w), 0.f};
    } else {
      qw = ff_from_double(q4.x); qx = ff_from_double(q4.y); qy = ff_from_double(q4.z);
      qz = ff_from_double(q4.w);
    }
    if (INTEG) {
      float* acc = d.acc32 + 8 * c;
      *reinterpret_cast<float4*>(acc) = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(acc + 4) = make_float4(0.f, 0.f, 0.f, 0.f);
      const float hf = d.hf;
      const float im = mim.y;
      if (d.alast) d.alast[c] = sqrtf(a0.x * a0.x + a0.y * a0.y + a0.z * a0.z) * im;
      // Eq. (5a): double velocity, accumulating the float increment
      // h F/m + h g (one double addition per component)
      v.x += f2d(fmaf(hf, a0.x * im, d.hgf[0]));
      v.y += f2d(fmaf(hf, a0.y * im, d.hgf[1]));
      v.z += f2d(fmaf(hf, a0.z * im, d.hgf[2]));
      // position: the offset increment h*v carries 1e-7 relative error, far
      // below the 2^-44 m resolution of the offset itself
      const float vx_f = d2f(v.x), vy_f = d2f(v.y), vz_f = d2f(v.z);
      vf_new[0] = vx_f; vf_new[1] = vy_f; vf_new[2] = vz_f;
      float o[3] = {off.x + hf * vx_f, off.y + hf * vy_f, off.z + hf * vz_f};
      int vi[3] = {vox.x, vox.y, vox.z};
      const float kV = (float)kVoxel;
      bool carried = false;
      for (int k = 0; k < 3; ++k) {
        if (fabsf(o[k]) > 0.5f * kV) {
          const float m = rintf(o[k] * (1.f / kV));
          vi[k] += (int)m;
          o[k] -= m * kV;  // exact: m * 2^-20 and the difference are representable
          carried = true;
        }
      }
      vox = make_int4(vi[0], vi[1], vi[2], vox.w);
      // Eq. (5b): body frame, float angular acceleration, double accumulation
      float Rf[9];
      quat_to_mat(qw.h, qx.h, qy.h, qz.h, Rf);
      const V3<float> tb = mat_tmul(Rf, V3<float>{a0.w, a1.x, a1.y});
      const V3<float> wf = {d2f(w.x), d2f(w.y), d2f(w.z)};
      const float* It = d.tinertf + 6 * tpl;  // I0, I1, I2 and their inverses
      const V3<float> gy = cross(wf, V3<float>{It[0] * wf.x, It[1] * wf.y, It[2] * wf.z});
      w.x += f2d(hf * ((tb.x - gy.x) * It[3]));
      w.y += f2d(hf * ((tb.y - gy.y) * It[4]));
      w.z += f2d(hf * ((tb.z - gy.z) * It[5]));
      // orientation: q <- q * exp(h w / 2); the increment q * (dq - 1) in
      // float, accumulated in double; then |q| is restored to one with a
      // first-order correction whose size is measured in float-float
      const V3<float> wn = {d2f(w.x), d2f(w.y), d2f(w.z)};
      wf_new = wn;
      const float th = 0.5f * hf * sqrtf(dot(wn, wn));
      const float th2 = th * th;
      const float cm1 = -0.5f * th2 + th2 * th2 * (1.f / 24.f);  // cos(th) - 1
      const float sc = 0.5f * hf * (1.f - th2 * (1.f / 6.f) + th2 * th2 * (1.f / 120.f));
      float dqm[4] = {cm1, sc * wn.x, sc * wn.y, sc * wn.z};
      if (th > 1e-2f) {
        const float sn = sinf(th), cs = cosf(th);
        const float s2 = sn / (2.f * th / hf);
        dqm[0] = cs - 1.f; dqm[1] = s2 * wn.x; dqm[2] = s2 * wn.y; dqm[3] = s2 * wn.z;
      }
      const float qf[4] = {qw.h, qx.h, qy.h, qz.h};
      float inc[4];
      quat_mulf(qf, dqm, inc);
      // q + inc in float-float (the exact split of the double orientation
      // plus the float increment), its norm, and then one double addition
      // per component for the increment and the normalisation together:
      // q <- q + (inc + hs (q + inc)), hs = 1/|q + inc| - 1 to first order
      const ff a[4] = {ff_add(ff_from_double(q4.x), ff{inc[0], 0.f}),
                       ff_add(ff_from_double(q4.y), ff{inc[1], 0.f}),
                       ff_add(ff_from_double(q4.z), ff{inc[2], 0.f}),
                       ff_add(ff_from_double(q4.w), ff{inc[3], 0.f})};
      const ff n2 = ff_add(ff_add(ff_mul(a[0], a[0]), ff_mul(a[1], a[1])),
                           ff_add(ff_mul(a[2], a[2]), ff_mul(a[3], a[3])));
      const float hs = -0.5f * ff_to_float(ff_sub(n2, {1.f, 0.f}));
      double qd[4] = {q4.x + f2d(fmaf(hs, a[0].h, inc[0])), q4.y + f2d(fmaf(hs, a[1].h, inc[1])),
                      q4.z + f2d(fmaf(hs, a[2].h, inc[2])), q4.w + f2d(fmaf(hs, a[3].h, inc[3]))};
      qw = ff_add(a[0], ff_mulf(a[0], hs)); qx = ff_add(a[1], ff_mulf(a[1], hs));
      qy = ff_add(a[2], ff_mulf(a[2], hs)); qz = ff_add(a[3], ff_mulf(a[3], hs));
      q4 = make_double4_32a(qd[0], qd[1], qd[2], qd[3]);
      // motion bound since the last rebuild, in the offset record's fourth
      // word (+inf when unknown): a sphere at most b from the centre of mass
      // moved at most h |v| + b h |omega| this step, plus the rounding of the
      // offset update (below 2^-43 m); summed with upward rounding.  The
      // square roots are x rsqrt(x) (within 2^-21 of the root), which the
      // factor 1 + 2^-18 covers together with the float rounding of v
      const float bnd = d.tpbound[tpl];
      const float v2 = __fmaf_ru(vx_f, vx_f, __fmaf_ru(vy_f, vy_f, __fmaf_ru(vz_f, vz_f, 1e-30f)));
      const float w2 = __fmaf_ru(wn.x, wn.x, __fmaf_ru(wn.y, wn.y, __fmaf_ru(wn.z, wn.z, 1e-30f)));
      const float sv = __fmul_ru(v2, rsqrtf(v2)), sw = __fmul_ru(w2, rsqrtf(w2));
      const float step_b = __fmaf_ru(__fmul_ru(hf, __fmaf_ru(bnd, sw, sv)), 1.000003814697265625f,
                                     1.1368683772161603e-13f);  // (1 + 2^-18), 2^-43 m
      const float motion = __fadd_ru(off.w, step_b);
      off = make_float4(o[0], o[1], o[2], motion);
      if (!(finite_d(v.x) && finite_d(v.y) && finite_d(v.z) && finite_d(w.x) && finite_d(w.y) &&
            finite_d(w.z) && finite_d(qd[0]) && finite_d(qd[1]) && finite_d(qd[2]) &&
            finite_d(qd[3]) && isfinite(o[0]) && isfinite(o[1]) && isfinite(o[2])))
        atomicOr(d.flags, kFlagNonFinite);
      if (carried) d.cvox[c] = vox;
      d.coff[c] = off; d.cq[c] = q4;
      store_vel(d.cvw + c, v, w);
      const float mlim = CERT ? (d.cmargin ? d.cmargin[c] : margin) : 0.f;
      // The exact certificate (below) reads the 48-byte state of the last
      // rebuild.  Its computed displacement is at most the motion bound times
      // (1 + 2^-12) plus 2^-40 m plus b 2^-18 (the roundings of the offsets'
      // differences, of the float reference orientation and of the quaternion
      // product), and its test is monotone in the displacement: when that
      // bound passes the same test the exact certificate passes too.
      const float mb = __fmaf_ru(off.w, 1.000244140625f,
                                 __fmaf_ru(bnd, 3.814697265625e-6f, 9.094947017729282e-13f));
      if (CERT && mb * 1.00001f + 1e-12f > mlim) {
        const int4 v0 = d.ref_vox[c];
        const float4 o0 = d.ref_off[c];
        const float4 ref_qv = d.ref_q[c];
        const float dx = (float)(vox.x - v0.x) * kV + (off.x - o0.x);
        const float dy = (float)(vox.y - v0.y) * kV + (off.y - o0.y);
        const float dz = (float)(vox.z - v0.z) * kV + (off.z - o0.z);
        const float4 r0 = ref_qv;
        const float a[4] = {r0.x, -r0.y, -r0.z, -r0.w};
        const float b[4] = {qw.h, qx.h, qy.h, qz.h};
        float e[4];
        quat_mulf(a, b, e);
        const float disp = sqrtf(dx * dx + dy * dy + dz * dz) +
                           2.f * bnd * sqrtf(e[1] * e[1] + e[2] * e[2] + e[3] * e[3]);
        if (disp * 1.00001f + 1e-12f > mlim) {
          atomicOr(d.flags, kFlagGuard);
          atomicAdd(d.counters + 1, 1ull);
          // the state of step *dstep + 1 may lack a listed contact
          if (d.halt_at) atomicMin(reinterpret_cast<unsigned long long*>(d.halt_at),
                                   (unsigned long long)(*d.dstep + 1));
        }
      }
    }
    // rotation matrix as float-float from the double orientation
    const ff xx = ff_mul(qx, qx), yy = ff_mul(qy, qy), zz = ff_mul(qz, qz);
    const ff xy = ff_mul(qx, qy), xz = ff_mul(qx, qz), yz = ff_mul(qy, qz);
    const ff wx = ff_mul(qw, qx), wy = ff_mul(qw, qy), wz = ff_mul(qw, qz);
    const ff one = {1.f, 0.f};
    ff R[9];
    R[0] = ff_sub(one, ff_scale2(ff_add(yy, zz), 2.f));
    R[1] = ff_scale2(ff_sub(xy, wz), 2.f);
    R[2] = ff_scale2(ff_add(xz, wy), 2.f);
    R[3] = ff_scale2(ff_add(xy, wz), 2.f);
    R[4] = ff_sub(one, ff_scale2(ff_add(xx, zz), 2.f));
    R[5] = ff_scale2(ff_sub(yz, wx), 2.f);
    R[6] = ff_scale2(ff_sub(xz, wy), 2.f);
    R[7] = ff_scale2(ff_add(yz, wx), 2.f);
    R[8] = ff_sub(one, ff_scale2(ff_add(xx, yy), 2.f));
    float Rf[9];
    for (int k = 0; k < 9; ++k) Rf[k] = R[k].h;
    if (!INTEG) {
      wf_new = {d2f(w.x), d2f(w.y), d2f(w.z)};
      vf_new[0] = d2f(v.x); vf_new[1] = d2f(v.y); vf_new[2] = d2f(v.z);
      // a state set from outside: its motion since the last rebuild is
      // unknown (CERT here: a state restored with its certificate reference,
      // whose motion bound still holds)
      if (!CERT) d.coff[c] = make_float4(off.x, off.y, off.z, __int_as_float(0x7f800000));
    }
    const V3<float> ww = mat_mul(Rf, wf_new);
    d.mv32[c] = make_float4(vf_new[0], vf_new[1], vf_new[2], mass);
    d.mw32[c] = make_float4(ww.x, ww.y, ww.z, 0.f);
    for (int k = 0; k < 9; ++k) {
      wp.Rh[k][lane] = R[k].h;
      wp.Rl[k][lane] = R[k].l;
    }
    wp.off[0][lane] = __float2int_rn(off.x * kMToFix);
    wp.off[1][lane] = __float2int_rn(off.y * kMToFix);
    wp.off[2][lane] = __float2int_rn(off.z * kMToFix);
    wp.s0[lane] = d.csph[c];
    if (lane == nw - 1) wp.s0[nw] = d.csph[c + 1];
    wp.t0[lane] = d.tpl_off[tpl];
  }
  __syncwarp();
  // pose records: x_rel = round(R p .h) + round(off) + round(R p .l), each
  // term in 2^-44 m units (|off| <= 2^-21 m and |R p .l| <= 2^-31 m fit a
  // 32-bit integer): three roundings of half a unit plus the float-float
  // error of R p (a small fraction of a unit) keep the centre within 2 units
  // of the exact one, the bound the detection relies on
  const int S0 = wp.s0[0], S1 = wp.s0[nw];
  for (int j = S0 + lane; j < S1; j += 32) {
    int lo = 0, hi = nw - 1;  // the clump k of sphere j: the last k with s0[k] <= j
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wp.s0[mid] <= j) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const float4 t4 = d.tp32[wp.t0[k] + (j - wp.s0[k])];
    const float p[3] = {t4.x, t4.y, t4.z};
    long long X[3];
    for (int i = 0; i < 3; ++i) {
      // row i of R p in float-float: the three products of the high parts
      // exactly (TwoProduct), summed with TwoSum; their errors, the rounding
      // errors of the sums and the low parts' products, all below 2^-23 of
      // the result, summed in float
      const ff p0 = two_prod(wp.Rh[3 * i][k], p[0]);
      const ff p1 = two_prod(wp.Rh[3 * i + 1][k], p[1]);
      const ff p2 = two_prod(wp.Rh[3 * i + 2][k], p[2]);
      const ff s01 = two_sum(p0.h, p1.h);
      const ff s = two_sum(s01.h, p2.h);
      float lo = fmaf(wp.Rl[3 * i][k], p[0], (p0.l + p1.l) + (p2.l + (s01.l + s.l)));
      lo = fmaf(wp.Rl[3 * i + 1][k], p[1], lo);
      lo = fmaf(wp.Rl[3 * i + 2][k], p[2], lo);
      const ff acc = fast_two_sum(s.h, lo);
      X[i] = f2ll_rn_near(acc.h * kMToFix) + wp.off[i][k] + __float2int_rn(acc.l * kMToFix);
    }
    d.srec32[j] = pack_rel(X[0], X[1], X[2]);
  }
}

// ---------------------------------------------------------------------------
// deterministic reduction: per-clump lists of contribution slots, built at a
// rebuild, and the per-clump sums in list order
// ---------------------------------------------------------------------------
__global__ void k_det_count(DevState d, ContactList l, long long n, long long nw,
                            uint32_t* __restrict__ cnt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    atomicAdd(&cnt[d.sinfo[l.pa[i]].x], 1u);
    atomicAdd(&cnt[d.sinfo[l.pb[i] & ~kHistFlag].x], 1u);
  } else if (i < n + nw) {
    atomicAdd(&cnt[d.sinfo[l.ws[i - n]].x], 1u);
  }
}

__global__ void k_det_fill(DevState d, ContactList l, long long n, long long nw,
                           const uint32_t* __restrict__ off, uint32_t* __restrict__ fill,
                           uint32_t* __restrict__ ids) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int ca = d.sinfo[l.pa[i]].x, cb = d.sinfo[l.pb[i] & ~kHistFlag].x;
    ids[off[ca] + atomicAdd(&fill[ca], 1u)] = (uint32_t)(2 * i);
    ids[off[cb] + atomicAdd(&fill[cb], 1u)] = (uint32_t)(2 * i + 1);
  } else if (i < n + nw) {
    const int c = d.sinfo[l.ws[i - n]].x;
    ids[off[c] + atomicAdd(&fill[c], 1u)] = (uint32_t)(2 * n + (i - n));
  }
}

// each clump's slot ids in ascending order (insertion sort: lists are short)
__global__ void k_det_sort(long long ncl, const uint32_t* __restrict__ off, uint32_t* __restrict__ ids) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncl) return;
  const uint32_t r0 = off[c], r1 = off[c + 1];
  for (uint32_t i = r0 + 1; i < r1; ++i) {
    const uint32_t v = ids[i];
    uint32_t j = i;
    while (j > r0 && ids[j - 1] > v) {
      ids[j] = ids[j - 1];
      --j;
    }
    ids[j] = v;
  }
}

__global__ void k_det_gather(DevState d, ContactList l) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (halted(d) || c >= d.ncl) return;
  const long long n2 = 2 * l.dn[0];
  const uint32_t r0 = d.det_off[c], r1 = d.det_off[c + 1];
  if (d.prec == 0) {
    V3<double> F = {0.0, 0.0, 0.0}, T = {0.0, 0.0, 0.0};
    for (uint32_t r = r0; r < r1; ++r) {
      const long long id = d.det_ids[r];
      if (id < n2) {
        const long long k = id >> 1;
        const double4_32a f = d.det_pair64[3 * k], t = d.det_pair64[3 * k + 1 + (id & 1)];
        const double sg = (id & 1) ? 1.0 : -1.0;
        F = F + sg * V3<double>{f.x, f.y, f.z};
        T = T + V3<double>{t.x, t.y, t.z};
      } else {
        const long long j = id - n2;
        const double4_32a f = d.det_wall64[2 * j], t = d.det_wall64[2 * j + 1];
        F = F + V3<double>{f.x, f.y, f.z};
        T = T + V3<double>{t.x, t.y, t.z};
      }
    }
    double* acc = d.acc64 + 8 * c;
    acc[0] = F.x; acc[1] = F.y; acc[2] = F.z; acc[3] = T.x; acc[4] = T.y; acc[5] = T.z;
  } else {
    V3<float> F = {0.f, 0.f, 0.f}, T = {0.f, 0.f, 0.f};
    for (uint32_t r = r0; r < r1; ++r) {
      const long long id = d.det_ids[r];
      if (id < n2) {
        const long long k = id >> 1;
        const float4 f = d.det_pair32[3 * k], t = d.det_pair32[3 * k + 1 + (id & 1)];
        const float sg = (id & 1) ? 1.f : -1.f;
        F = F + sg * V3<float>{f.x, f.y, f.z};
        T = T + V3<float>{t.x, t.y, t.z};
      } else {
        const long long j = id - n2;
        const float4 f = d.det_wall32[2 * j], t = d.det_wall32[2 * j + 1];
        F = F + V3<float>{f.x, f.y, f.z};
        T = T + V3<float>{t.x, t.y, t.z};
      }
    }
    float* acc = d.acc32 + 8 * c;
    *reinterpret_cast<float4*>(acc) = make_float4(F.x, F.y, F.z, T.x);
    *reinterpret_cast<float4*>(acc + 4) = make_float4(T.y, T.z, 0.f, 0.f);
  }
}

__device__ __forceinline__ void place_walls(const DevState& d, double t) {
  for (int w = threadIdx.x; w < d.nwalls; w += blockDim.x) {
    const WallDev& W = d.walls[w];
    const SceneGrid& g = d.grids[d.wall_scene[w]];
    for (int k = 0; k < 3; ++k) {
      const double p = W.p[k] + W.vel[k] * t;
      d.wpos[3 * w + k] = p;
      d.wfix[3 * w + k] = __double2ll_rn((p - g.lo[k]) * 17592186044416.0);
    }
  }
}

// Places the walls at step `step` and sets the device step counter (one block).
__global__ void k_walls_at(DevState d, long long step) {
  place_walls(d, (double)step * d.h);
  if (threadIdx.x == 0) *d.dstep = step;
}

// After an integration: advances the device step counter and places the walls
// at the new time (one block).
__global__ void k_walls_advance(DevState d) {
  if (halted(d)) return;
  const long long next = *d.dstep + 1;
  __syncthreads();
  place_walls(d, (double)next * d.h);
  __syncthreads();
  if (threadIdx.x == 0) *d.dstep = next;
}

__global__ void k_set_ref(DevState d) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const double4_32a q = d.cq[c];
  d.ref_q[c] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
  if (d.prec == 0) {
    d.ref_pos[c] = d.cpos[c];
  } else {
    d.ref_vox[c] = d.cvox[c];
    const float4 o = d.coff[c];
    d.ref_off[c] = o;
    d.coff[c] = make_float4(o.x, o.y, o.z, 0.f);  // no motion since this state
  }
}

__global__ void k_get_state(DevState d, double* pos, double* quat, double* vel, double* angvel) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const double4_32a q = d.cq[c];
  if (pos) {
    if (d.prec == 0) {
      const double4_32a X = d.cpos[c];
      pos[3 * c] = X.x; pos[3 * c + 1] = X.y; pos[3 * c + 2] = X.z;
    } else {
      const SceneGrid g = d.grids[d.cinfo[c].y];
      const int4 v = d.cvox[c];
      const float4 o = d.coff[c];
      pos[3 * c] = g.lo[0] + ((double)v.x * kVoxel + (double)o.x);
      pos[3 * c + 1] = g.lo[1] + ((double)v.y * kVoxel + (double)o.y);
      pos[3 * c + 2] = g.lo[2] + ((double)v.z * kVoxel + (double)o.z);
    }
  }
  if (quat) {
    quat[4 * c] = q.x; quat[4 * c + 1] = q.y; quat[4 * c + 2] = q.z; quat[4 * c + 3] = q.w;
  }
  double4_32a v, w;
  load_vel(d.cvw + c, v, w);
  if (vel) {
    vel[3 * c] = v.x; vel[3 * c + 1] = v.y; vel[3 * c + 2] = v.z;
  }
  if (angvel) {
    double R[9];
    quat_to_mat(q.x, q.y, q.z, q.w, R);
    const V3<double> ww = mat_mul(R, V3<double>{w.x, w.y, w.z});
    angvel[3 * c] = ww.x; angvel[3 * c + 1] = ww.y; angvel[3 * c + 2] = ww.z;
  }
}

// Voxel split of one position coordinate relative to the scene corner:
// rel = m * 2^-20 + off with m = rint(rel * 2^20).  Both products are exact
// (powers of two) and rel - m * 2^-20 is exact (Sterbenz), so the split is the
// same whether or not the compiler contracts it.
__device__ __forceinline__ double voxel_index(double x, double lo) { return rint((x - lo) / kVoxel); }

// Validation pass over a staged state (pos 3n | quat 4n | vel 3n | angvel 3n
// doubles): bit 0 of *err for a non-finite value, bit 1 for a position too far
// from its scene corner for the int32 voxel index.  Nothing is written to the
// clump state, so a rejected call leaves it as it was.
__global__ void k_check_state(DevState d, const double* t, int* err) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const long long n = d.ncl;
  bool finite = true;
  for (int k = 0; k < 3; ++k) finite &= isfinite(t[3 * c + k]) && isfinite(t[7 * n + 3 * c + k]) &&
                                        isfinite(t[10 * n + 3 * c + k]);
  for (int k = 0; k < 4; ++k) finite &= isfinite(t[3 * n + 4 * c + k]);
  int e = finite ? 0 : 1;
  if (finite && d.prec != 0) {
    const SceneGrid g = d.grids[d.cinfo[c].y];
    for (int k = 0; k < 3; ++k)
      if (fabs(voxel_index(t[3 * c + k], g.lo[k])) > 2.0e9) e |= 2;
  }
  if (e) atomicOr(err, e);
}

// Writes a validated staged state into the clump records: quaternion and
// velocity as given, the angular velocity rotated into the body frame
// (w_body = R(q)^T w), the position as FP64 or as voxel index + float offset.
__global__ void k_set_state(DevState d, const double* t) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const long long n = d.ncl;
  const double* p = t + 3 * c;
  const double* q = t + 3 * n + 4 * c;
  const double* v = t + 7 * n + 3 * c;
  const double* w = t + 10 * n + 3 * c;
  d.cq[c] = make_double4_32a(q[0], q[1], q[2], q[3]);
  double R[9];
  quat_to_mat(q[0], q[1], q[2], q[3], R);
  const V3<double> wb = mat_tmul(R, V3<double>{w[0], w[1], w[2]});
  store_vel(d.cvw + c, make_double4_32a(v[0], v[1], v[2], 0.0),
            make_double4_32a(wb.x, wb.y, wb.z, 0.0));
  if (d.prec == 0) {
    d.cpos[c] = make_double4_32a(p[0], p[1], p[2], 0.0);
  } else {
    const SceneGrid g = d.grids[d.cinfo[c].y];
    int vox[3];
    float off[3];
    for (int k = 0; k < 3; ++k) {
      const double m = voxel_index(p[k], g.lo[k]);
      vox[k] = (int)m;
      off[k] = (float)((p[k] - g.lo[k]) - m * kVoxel);
    }
    d.cvox[c] = make_int4(vox[0], vox[1], vox[2], 0);
    d.coff[c] = make_float4(off[0], off[1], off[2], 0.f);
  }
}

__global__ void k_get_forces(DevState d, double* F, double* T) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  for (int k = 0; k < 3; ++k) {
    if (d.prec == 0) {
      F[3 * c + k] = d.acc64[8 * c + k];
      T[3 * c + k] = d.acc64[8 * c + 3 + k];
    } else {
      F[3 * c + k] = (double)d.acc32[8 * c + k];
      T[3 * c + k] = (double)d.acc32[8 * c + 3 + k];
    }
  }
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

int g_sm_count = 0;
int sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 132;
  }
  return g_sm_count;
}

}  // namespace

// The contact kernels read the list lengths from device memory and run on a
// persistent grid of fixed size, so one launch (or one captured graph) serves
// every list the buffers will hold.
void launch_force_pairs(const DevState& d, ContactList& l, bool count_active, cudaStream_t st) {
  const unsigned grid = (unsigned)sm_count() * (unsigned)(d.pairs_bpsm > 0 ? d.pairs_bpsm : 8);
  if (d.prec == 0)
    { k_pairs64<<<grid, 256, 0, st>>>(d, l, count_active ? 1 : 0); count_launch(); }
  else
    { k_pairs32<<<grid, 256, 0, st>>>(d, l, count_active ? 1 : 0); count_launch(); }
}

void launch_force_walls(const DevState& d, ContactList& l, double t, bool count_active,
                        cudaStream_t st) {
  (void)t;
  if (d.nwalls == 0) return;
  // about one wall contact per thread (the list's length at its rebuild; the
  // kernel strides over the length on the device), at most the blocks that
  // fit at once (80 registers x 128 threads: 6 per SM)
  const long long want = (l.nw + 127) / 128;
  const long long cap = (long long)sm_count() * 6;
  const unsigned grid = (unsigned)std::max(1LL, std::min(want, cap));
  if (d.prec == 0)
    { k_walls64<<<grid, 128, 0, st>>>(d, l, count_active ? 1 : 0); count_launch(); }
  else
    { k_walls32<<<grid, 128, 0, st>>>(d, l, count_active ? 1 : 0); count_launch(); }
}

template <int B>
void launch_update32(const DevState& d, bool integrate, bool cert, float margin, cudaStream_t st) {
  const unsigned g = nblk(d.ncl, B);
  // without integration, cert = true keeps the motion bounds (a state restored
  // together with its certificate reference)
  if (!integrate) {
    if (cert) k_update32<B, false, true><<<g, B, 0, st>>>(d, margin);
    else k_update32<B, false, false><<<g, B, 0, st>>>(d, margin);
  }
  else if (cert) k_update32<B, true, true><<<g, B, 0, st>>>(d, margin);
  else k_update32<B, true, false><<<g, B, 0, st>>>(d, margin);
  count_launch();
}

// integrate: one explicit step of every clump, then the device step counter
// advances and the walls move to the new time.  Otherwise the sphere poses
// and mirrors are recomputed from the state and the walls are placed at
// `step` (which also sets the device step counter).
void launch_update(const DevState& d, bool integrate, long long step, double margin,
                   bool check_cert, cudaStream_t st) {
  if (d.ncl > 0) {
    if (d.prec == 0)
      { k_update64<<<nblk(d.ncl, kUpd), kUpd, 0, st>>>(d, integrate ? 1 : 0, (float)margin,
                                                      check_cert ? 1 : 0); count_launch(); }
    else if (d.upd_block == 64)
      launch_update32<64>(d, integrate, check_cert, (float)margin, st);
    else if (d.upd_block == 256)
      launch_update32<256>(d, integrate, check_cert, (float)margin, st);
    else
      launch_update32<128>(d, integrate, check_cert, (float)margin, st);
  }
  if (integrate) {
    k_walls_advance<<<1, 256, 0, st>>>(d);
    count_launch();
  } else {
    launch_walls_at(d, step, st);
  }
}

void launch_walls_at(const DevState& d, long long step, cudaStream_t st) {
  k_walls_at<<<1, 256, 0, st>>>(d, step);
  count_launch();
}

void launch_det_lists(const DevState& d, const ContactList& l, long long n, long long nw,
                      uint32_t* cnt, uint32_t* fill, uint32_t* off, uint32_t* ids, void* scan_scratch,
                      unsigned long long* d_total, cudaStream_t st) {
  if (d.ncl == 0) return;
  const long long m = n + nw;
  if (m > 0) { k_det_count<<<nblk(m, 256), 256, 0, st>>>(d, l, n, nw, cnt); count_launch(); }
  exclusive_scan_u32(cnt, off, d.ncl + 1, scan_scratch, d_total, st);
  if (m > 0) { k_det_fill<<<nblk(m, 256), 256, 0, st>>>(d, l, n, nw, off, fill, ids); count_launch(); }
  k_det_sort<<<nblk(d.ncl, 256), 256, 0, st>>>(d.ncl, off, ids);
  count_launch();
}

void launch_det_gather(const DevState& d, const ContactList& l, cudaStream_t st) {
  if (d.ncl == 0) return;
  k_det_gather<<<nblk(d.ncl, 256), 256, 0, st>>>(d, l);
  count_launch();
}

void launch_set_cert_ref(const DevState& d, cudaStream_t st) {
  if (d.ncl > 0) { k_set_ref<<<nblk(d.ncl, 256), 256, 0, st>>>(d); count_launch(); }
}

void launch_get_state(const DevState& d, double* pos, double* quat, double* vel, double* angvel,
                      cudaStream_t st) {
  if (d.ncl > 0) { k_get_state<<<nblk(d.ncl, 256), 256, 0, st>>>(d, pos, quat, vel, angvel); count_launch(); }
}

void launch_check_state(const DevState& d, const double* staged, int* err, cudaStream_t st) {
  if (d.ncl > 0) { k_check_state<<<nblk(d.ncl, 256), 256, 0, st>>>(d, staged, err); count_launch(); }
}

void launch_set_state(const DevState& d, const double* staged, cudaStream_t st) {
  if (d.ncl > 0) { k_set_state<<<nblk(d.ncl, 256), 256, 0, st>>>(d, staged); count_launch(); }
}

void launch_get_forces(const DevState& d, double* F, double* T, cudaStream_t st) {
  if (d.ncl > 0) { k_get_forces<<<nblk(d.ncl, 256), 256, 0, st>>>(d, F, T); count_launch(); }
}

}  // namespace dem
