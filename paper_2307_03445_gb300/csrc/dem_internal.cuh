// dem_internal.cuh -- device layouts and helpers shared by the DEM kernels.
//
// Two precision modes (the C ABI's DEM_FP64 and DEM_FP32_VOXEL):
//   FP64        every quantity in double; used for small reference runs.
//   FP32_VOXEL  clump position = int voxel index (voxel edge 2^-20 m) + float
//               offset; forces, torques and contact kinematics in float;
//               double only for the velocity / angular velocity / orientation
//               state of the integrator and the tangential-history sums.
//               Where a float difference would cancel catastrophically (the
//               overlap delta_n = r_a + r_b - |x_b - x_a| of Eq. (1)), sphere
//               centres are carried as int64 fixed point (2^-44 m) and the
//               overlap is formed with float-float error-free transforms
//               (Knuth's TwoSum, FMA-based TwoProduct), not with double.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dem {

constexpr int kDetBits = 24;   // detection lattice: 2^-24 m
constexpr int kFixBits = 44;   // fixed-point sphere centres: 2^-44 m
constexpr int kVoxLog2 = 20;   // voxel edge 2^-20 m (FP32_VOXEL positions)
constexpr double kDetScale = 16777216.0;          // 2^24
constexpr double kVoxel = 1.0 / 1048576.0;        // 2^-20
constexpr float kFixToM = 5.684341886080802e-14f; // 2^-44
constexpr float kMToFix = 17592186044416.0f;      // 2^44
constexpr uint32_t kHistFlag = 0x80000000u;       // in pb / ww: history is non-zero

// A clump's velocity and body-frame angular velocity (FP64, both precision
// modes): 48 bytes, moved as three 16-byte vectors.
struct alignas(16) VelRec {
  double vx, vy, vz, wx, wy, wz;
};

__device__ __forceinline__ void load_vel(const VelRec* p, double4_32a& v, double4_32a& w) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = q[0], b = q[1], c = q[2];
  v = make_double4_32a(a.x, a.y, b.x, 0.0);
  w = make_double4_32a(b.y, c.x, c.y, 0.0);
}

__device__ __forceinline__ void store_vel(VelRec* p, const double4_32a& v, const double4_32a& w) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, w.x);
  q[2] = make_double2(w.y, w.z);
}

// Pair material coefficients (section 2.1: derived from E, nu, CoR and mu).
// kn = 4/3 E*, kt = 8 G*, mu; the damping terms of Eq. (1a), (1b) are
//   f gamma_n m = cn sqrt(f m),  f gamma_t m = ct sqrt(f m)
// with cn = -2 sqrt(5/6) beta sqrt(2 E*), ct = -2 sqrt(5/6) beta sqrt(8 G*).
template <typename T>
struct PairMat {
  T kn, kt, mu, cn, ct, pad0, pad1, pad2;
};

// Per-scene detection grid.
struct SceneGrid {
  double lo[3];      // domain corner (also the voxel origin in FP32_VOXEL)
  long long L;       // bin edge in lattice units (2^-24 m)
  int dims[3];       // bins per axis
  uint32_t key_base; // first bin key of this scene
  int wall_start;    // this scene's walls: wall_idx[wall_start .. wall_start+wall_count)
  int wall_count;
  float lof[3];      // lo as float (estimates only)
  float invL;        // 1 / L as float (division estimates only)
};

// Wall description on the device (both precisions).  For FP32_VOXEL the
// geometric constants are also kept as float-float pairs.
struct WallDev {
  int type, material;
  double p[3], n[3], vel[3];
  double radius, half_angle, height;
  double rb;          // cone base radius = height * tan(half_angle)
  float nh[3], nl[3]; // unit normal / axis as float-float
  float rh, rl;       // cylinder radius as float-float
  float ch, cl, sh, sl; // cone cos / sin of the half angle as float-float
  float hh, hl;       // cone height as float-float
  float rbh, rbl;     // cone base radius as float-float
  float speed;        // |vel|
  double speed_d;     // |vel| = sqrt((vx^2 + vy^2) + vz^2), evaluated on the host
  float pf[3], vf[3]; // reference point and velocity as float (estimates, wall speed)
  float radf, heightf, rbf;
  // mesh facet: edge vectors from the first vertex p (translation invariant)
  double e1[3], e2[3];      // b - p, c - p
  float e1h[3], e1l[3];     // as float-float
  float e2h[3], e2l[3];
};

// Sphere pose record of FP32_VOXEL (written every step by the update kernel,
// 16 bytes): the sphere centre relative to its clump's voxel corner,
// x_rel = off + R(q) p, in fixed point (2^-44 m), as three signed 40-bit
// fields packed into a uint4 (x in bits 0-39, y in 40-79, z in 80-119; the
// top 8 bits are zero).  The centre relative to the scene corner is
// (voxel << 24) + x_rel.  40 bits hold |x_rel| < 2^39 units = 2^-5 m, so
// template sphere centres must lie within 2^-5 m - 2^-20 m of the clump's
// centre of mass (checked when the templates are loaded).  The radius,
// material and owner come from the static per-sphere and template tables.
constexpr long long kRelLimit = 1ll << 39;
__device__ __forceinline__ uint4 pack_rel(long long x, long long y, long long z) {
  const unsigned long long m = (1ull << 40) - 1ull;
  const unsigned long long ux = (unsigned long long)x & m, uy = (unsigned long long)y & m,
                           uz = (unsigned long long)z & m;
  const unsigned long long lo = ux | (uy << 40), hi = (uy >> 24) | (uz << 16);
  return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
}
__device__ __forceinline__ void unpack_rel(uint4 r, long long& x, long long& y, long long& z) {
  const unsigned long long lo = (unsigned long long)r.x | ((unsigned long long)r.y << 32);
  const unsigned long long hi = (unsigned long long)r.z | ((unsigned long long)r.w << 32);
  x = (long long)(lo << 24) >> 24;
  y = (long long)(((lo >> 40) | (hi << 24)) << 24) >> 24;
  z = (long long)(hi << 8) >> 24;
}
struct alignas(32) SphA64 {  // FP64 pose record: centre and radius
  double x, y, z, r;
};

// ---------------------------------------------------------------------------
// IEEE-754 binary32 <-> binary64 conversions on the integer pipe.  On this GPU
// the hardware conversions issue at the (low) double-precision rate; these
// produce the same results from the bit patterns with integer operations only,
// for every input class (zero, subnormal, infinite and NaN included), so that
// no branch the compiler may predicate brings a hardware conversion back.
// ---------------------------------------------------------------------------
static __device__ __noinline__ double f2d_rare(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  unsigned long long bits = (unsigned long long)(u >> 31) << 63;
  if (e == 0xffu) {  // infinity, or NaN made quiet
    bits |= 0x7ff0000000000000ull | ((unsigned long long)m << 29) |
            (m ? 0x0008000000000000ull : 0ull);
  } else if (e != 0u) {
    bits |= ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)m << 29);
  } else if (m != 0u) {  // subnormal float m * 2^-149: a normal double
    const int p = 31 - __clz((int)m);  // position of the leading one, 0..22
    bits |= ((unsigned long long)(p + 874) << 52) |
            (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
  }
  return __longlong_as_double((long long)bits);
}
// double -> float, rounded to nearest, ties to even.
static __device__ __noinline__ float d2f_rare(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int ed = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (ed == 0x7ff)  // infinity, or NaN made quiet
    return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u));
  const int e = ed - 1023 + 127;
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);  // overflows to infinity
  if (e > 0) {
    uint32_t r = ((uint32_t)e << 23) | (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);
    // a carry out of the mantissa correctly moves to the next binade (or infinity)
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r += 1u;
    return __uint_as_float(r | sign);
  }
  // float subnormal or zero: the value in units of 2^-149 is M * 2^-sh
  const int sh = 926 - ed;  // >= 30 here
  if (ed == 0 || sh >= 64) return __uint_as_float(sign);
  const unsigned long long M = m | 0x10000000000000ull;
  uint32_t q = (uint32_t)(M >> sh);
  const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1u))) q += 1u;  // may reach the smallest normal
  return __uint_as_float(sign | q);
}
// Normal numbers and zeros inline; the other classes out of line, so that the
// compiler does not predicate their code into every call.
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (e - 1u < 254u)
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
  if ((u << 1) == 0u) return __longlong_as_double((long long)sign);
  return f2d_rare(f);
}
__device__ __forceinline__ float d2f(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  if ((unsigned)(e - 1) < 254u) {
    const unsigned long long m = b & 0xfffffffffffffull;
    uint32_t r = ((uint32_t)e << 23) | (uint32_t)(m >> 29);
    const uint32_t rem = (uint32_t)(m & 0x1fffffffu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r += 1u;
    return __uint_as_float(r | sign);
  }
  if ((b << 1) == 0ull) return __uint_as_float(sign);
  return d2f_rare(d);
}
// Integer -> float for |v| < 2^22, exact: the float 1.5 * 2^23 has a unit
// last place, so adding v to its bit pattern and subtracting it is exact.
__device__ __forceinline__ float small_i2f(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
// float -> nearest integer (ties to even) for |x| < 2^22, same trick.
__device__ __forceinline__ int small_f2i(float x) {
  return __float_as_int(x + 12582912.0f) - 0x4B400000;
}
// int64 -> float-float (exact for |v| < 2^44), integer pipe only.
__device__ __forceinline__ void ll_split(long long v, float& hi, float& lo) {
  const int h = (int)(v >> 22);                 // |h| < 2^22
  const int l = (int)(v & ((1ll << 22) - 1));   // 0 <= l < 2^22
  hi = small_i2f(h) * 4194304.0f;               // exact: times 2^22
  lo = small_i2f(l);
}
// float -> nearest int64 (ties to even), integer pipe; exact for |x| < 2^62.
__device__ __forceinline__ long long f2ll_rn(float x) {
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu) - 127;
  if (e < 22) return (long long)small_f2i(x);
  const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
  long long v;
  if (e >= 23) {
    v = m << (e - 23);
  } else {  // e == 22: one fractional bit
    v = m >> 1;
    if ((m & 1) && (v & 1)) ++v;
  }
  return (u >> 31) ? -v : v;
}

// float -> nearest int64 (ties to even) for |x| < 2^43, without branches: with
// a = x / 2^22 rounded to an integer, b = x - a 2^22 is exact (|b| <= 2^21 and
// a multiple of x's last place), and the rounding of b decides the rounding of
// x (a 2^22 is even).  Equal to f2ll_rn on that range.
__device__ __forceinline__ long long f2ll_rn_near(float x) {
  const float t = fmaf(x, 2.38418579101562500e-7f, 12582912.0f);  // x / 2^22 + 1.5 2^23
  const int a = __float_as_int(t) - 0x4B400000;
  const float b = fmaf(t - 12582912.0f, -4194304.0f, x);
  return (long long)a * 4194304ll + (long long)small_f2i(b);
}

// ceil(d) for finite 0 <= d < 2^62, integer pipe.
__device__ __forceinline__ long long ceil_pos_d2ll(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  if (e < 0) return (b << 1) != 0ull ? 1ll : 0ll;  // 0 < d < 1 -> 1; +-0 -> 0
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  if (e >= 52) return (long long)(m << (e - 52));
  const int sh = 52 - e;
  const long long v = (long long)(m >> sh);
  return (m & ((1ull << sh) - 1ull)) ? v + 1 : v;
}

// Finite test on the bit pattern (integer pipe).
__device__ __forceinline__ bool finite_d(double d) {
  return ((unsigned long long)__double_as_longlong(d) & 0x7ff0000000000000ull) !=
         0x7ff0000000000000ull;
}

// ---------------------------------------------------------------------------
// float-float arithmetic (error-free transforms)
// ---------------------------------------------------------------------------
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.h, b.h);
  float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
  return fast_two_sum(p.h, e);
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  ff p = two_prod(a.h, b);
  float e = __fmaf_rn(a.l, b, p.l);
  return fast_two_sum(p.h, e);
}
__device__ __forceinline__ ff ff_scale2(ff a, float pow2) { return {a.h * pow2, a.l * pow2}; }
// d as float-float: h = d rounded to float, l = (d - h) rounded to float, on
// the integer pipe.  The residual d - h is exact in double; it is formed from
// the significands.  For |d| outside [2^-96, 2^127) (and non-finite d) the low
// part is dropped.
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = d2f(d);
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ed = (int)((b >> 52) & 0x7ffu);
  if (ed < 1023 - 96 || ed >= 1023 + 127) return {h, 0.f};
  const long long M = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  const uint32_t hu = __float_as_uint(h);
  const int eh = (int)((hu >> 23) & 0xffu);
  const long long Mh = (long long)((hu & 0x7fffffu) | 0x800000u) << (29 + (eh - 127) - (ed - 1023));
  const long long diff = M - Mh;  // |diff| <= 2^28, in units of 2^(ed - 1075)
  // one rounding of the exact sum of two exactly represented parts
  float l = __fadd_rn(small_i2f((int)(diff >> 7)) * 128.f, small_i2f((int)(diff & 127)));
  const int k = ed - 1075;  // -148 .. 75
  if (k >= -126) {
    l *= __int_as_float((k + 127) << 23);
  } else {
    l = (l * 5.42101086242752217e-20f) * __int_as_float((k + 64 + 127) << 23);  // 2^-64 * 2^(k+64)
  }
  return {h, (b >> 63) ? -l : l};
}
__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.h, a.l); }
// sqrt of a non-negative float-float to float-float accuracy: Dekker's
// double-length square root (T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971, procedure
// sqrt2): s = sqrt(a.h), then one Newton correction (a - s^2) / (2 s) with
// s^2 formed exactly by TwoProduct, added to s by FastTwoSum.
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.h > 0.f)) return {0.f, 0.f};
  float s = sqrtf(a.h);
  ff s2 = two_prod(s, s);
  float corr = __fdiv_rn(__fadd_rn(__fsub_rn(a.h, s2.h), __fsub_rn(a.l, s2.l)), 2.f * s);
  return fast_two_sum(s, corr);
}
// int64 fixed-point value (2^-44 m) -> float-float metres, integer pipe: the
// value is cut into three exact 22-bit pieces and summed without error.
__device__ __forceinline__ ff fix_to_ff(long long v) {
  const long long v1 = v >> 22;
  const float c0 = small_i2f((int)(v & 0x3fffff));
  const float c1 = small_i2f((int)(v1 & 0x3fffff)) * 4194304.0f;        // 2^22
  const float c2 = small_i2f((int)(v1 >> 22)) * 17592186044416.0f;      // 2^44
  ff s = two_sum(c2, c1);
  s = ff_add(s, {c0, 0.f});
  return {s.h * kFixToM, s.l * kFixToM};
}
// The same for |v| < 2^44 (neighbour differences): v = h 2^22 + l with both
// pieces exact floats, so TwoSum of them is the exact float-float of v (the
// same pair as fix_to_ff, whose high part is fix_to_float(v)).
__device__ __forceinline__ ff fix_to_ff_near(long long v) {
  const float h = small_i2f((int)(v >> 22)) * 4194304.0f;  // exact: |v >> 22| <= 2^22
  const float l = small_i2f((int)(v & 0x3fffff));
  const ff s = two_sum(h, l);
  return {s.h * kFixToM, s.l * kFixToM};
}
// Float estimate of a fixed-point value with |v| < 2^44 (neighbour differences).
__device__ __forceinline__ float fix_to_float(long long v) {
  return fmaf(small_i2f((int)(v >> 22)), 4194304.0f, small_i2f((int)(v & 0x3fffff))) * kFixToM;
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> v3(T x, T y, T z) { return {x, y, z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Rotation matrix of a unit quaternion (w, x, y, z), rows r[0..8].
template <typename T>
__device__ __forceinline__ void quat_to_mat(T w, T x, T y, T z, T r[9]) {
  T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  T wx = w * x, wy = w * y, wz = w * z;
  r[0] = T(1) - T(2) * (yy + zz); r[1] = T(2) * (xy - wz); r[2] = T(2) * (xz + wy);
  r[3] = T(2) * (xy + wz); r[4] = T(1) - T(2) * (xx + zz); r[5] = T(2) * (yz - wx);
  r[6] = T(2) * (xz - wy); r[7] = T(2) * (yz + wx); r[8] = T(1) - T(2) * (xx + yy);
}
template <typename T>
__device__ __forceinline__ V3<T> mat_mul(const T r[9], V3<T> p) {
  return {(r[0] * p.x + r[1] * p.y) + r[2] * p.z, (r[3] * p.x + r[4] * p.y) + r[5] * p.z,
          (r[6] * p.x + r[7] * p.y) + r[8] * p.z};
}
template <typename T>
__device__ __forceinline__ V3<T> mat_tmul(const T r[9], V3<T> p) {
  return {(r[0] * p.x + r[3] * p.y) + r[6] * p.z, (r[1] * p.x + r[4] * p.y) + r[7] * p.z,
          (r[2] * p.x + r[5] * p.y) + r[8] * p.z};
}

// The detection centre x = X + R(q) p evaluated with exactly one IEEE double
// rounding per operation in a fixed order (no contraction into FMA): the
// detection lattice coordinates are integers decided by this value, and the
// definition is the same wherever it is evaluated.
__device__ __forceinline__ void det_centre(const double q[4], const double p[3], const double X[3],
                                           double x[3]) {
  const double w = q[0], qx = q[1], qy = q[2], qz = q[3];
  const double xx = __dmul_rn(qx, qx), yy = __dmul_rn(qy, qy), zz = __dmul_rn(qz, qz);
  const double xy = __dmul_rn(qx, qy), xz = __dmul_rn(qx, qz), yz = __dmul_rn(qy, qz);
  const double wx = __dmul_rn(w, qx), wy = __dmul_rn(w, qy), wz = __dmul_rn(w, qz);
  double r[9];
  r[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
  r[1] = __dmul_rn(2.0, __dsub_rn(xy, wz));
  r[2] = __dmul_rn(2.0, __dadd_rn(xz, wy));
  r[3] = __dmul_rn(2.0, __dadd_rn(xy, wz));
  r[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
  r[5] = __dmul_rn(2.0, __dsub_rn(yz, wx));
  r[6] = __dmul_rn(2.0, __dsub_rn(xz, wy));
  r[7] = __dmul_rn(2.0, __dadd_rn(yz, wx));
  r[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
  for (int k = 0; k < 3; ++k) {
    const double rp = __dadd_rn(__dadd_rn(__dmul_rn(r[3 * k], p[0]), __dmul_rn(r[3 * k + 1], p[1])),
                                __dmul_rn(r[3 * k + 2], p[2]));
    x[k] = __dadd_rn(X[k], rp);
  }
}

__device__ __forceinline__ long long floordiv_ll(long long a, long long b) {
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}
// floor(a / L) for |a| < 2^31: a float reciprocal estimate, corrected by one
// integer step.  With L >= 1024 and the bin index below 2^21 the estimate is
// off by at most one; smaller L takes the integer division.
__device__ __forceinline__ long long floordiv_bin(long long a, long long L, float invL) {
  if (L < 1024) return floordiv_ll(a, L);
  long long q = (long long)__float2int_rd(__int2float_rn((int)a) * invL);
  const long long r = a - q * L;
  if (r < 0) --q;
  else if (r >= L) ++q;
  return q;
}
__device__ __forceinline__ int clampi(long long v, int hi) {
  return v < 0 ? 0 : (v > hi ? hi : (int)v);
}

// Vector reductions into global float memory (sm_90+).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// Error flags written by kernels, read by the host after each call.
enum : int {
  kFlagNonFinite = 1,
  kFlagCapacity = 2,
  kFlagGuard = 4,
  kFlagTimeout = 8,
  kFlagBounds = 16,
};

}  // namespace dem
