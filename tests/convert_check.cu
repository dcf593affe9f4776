// Test program: the integer-pipe conversions of the library (f32<->f64,
// f32->int64, ceil of a double, int64->float-float, double->float-float) against the hardware
// conversions, on random bit patterns and edge cases.
// Prints "mismatches <n> checked <m>" and exits 0 when n == 0.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#include "../paper_2307_03445_gb300/csrc/dem_internal.cuh"

__device__ uint64_t mix(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
  return x;
}

__global__ void k_check(unsigned long long n, unsigned long long* bad) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = mix(i + 12345);
  // doubles spread over all binades near the float range, plus raw patterns
  double dv;
  if (i % 3 == 0) {
    dv = __longlong_as_double((long long)r);
  } else {
    const int e = (int)(r % 300) - 150;  // exponents around the float range
    dv = ldexp(1.0 + (double)(r >> 12) * 0x1p-52, e) * ((r & 1) ? -1.0 : 1.0);
  }
  const float hw = __double2float_rn(dv), sw = dem::d2f(dv);
  const bool same_f = (__float_as_uint(hw) == __float_as_uint(sw)) || (hw != hw && sw != sw);
  const float fv = __uint_as_float((uint32_t)(r >> 17));
  const double hwd = (double)fv, swd = dem::f2d(fv);
  const bool same_d = (__double_as_longlong(hwd) == __double_as_longlong(swd)) ||
                      (hwd != hwd && swd != swd);
  // float -> int64 (nearest, ties to even) for |x| < 2^62
  const float fx = ldexpf(1.0f + (float)(r >> 41) * 0x1p-23f, (int)((r >> 5) % 62) - 2) *
                   ((r & 2) ? -1.0f : 1.0f);
  const bool same_ll = dem::f2ll_rn(fx) == __float2ll_rn(fx);
  // ceil of a non-negative double below 2^62
  const double cd = (i % 5 == 0) ? (double)(r >> 40) : fabs(dv);
  const bool same_c = !(cd < 0x1p62) || dem::ceil_pos_d2ll(cd) == (long long)ceil(cd);
  // int64 -> float-float is exact below 2^44
  const long long v = (long long)(r >> 21) - (1ll << 42);
  float hi, lo;
  dem::ll_split(v, hi, lo);
  const bool same_s = (long long)hi + (long long)lo == v;
  // double -> float-float against its definition with hardware arithmetic
  bool same_ff = true;
  if (fabs(dv) >= 0x1p-96 && fabs(dv) < 0x1p127) {
    const dem::ff p = dem::ff_from_double(dv);
    const float h0 = __double2float_rn(dv);
    const float l0 = __double2float_rn(dv - (double)h0);
    same_ff = __float_as_uint(p.h) == __float_as_uint(h0) && p.l == l0;
  }
  if (!same_f || !same_d || !same_ll || !same_c || !same_s || !same_ff) atomicAdd(bad, 1ull);
}

int main() {
  unsigned long long* bad;
  cudaMalloc(&bad, sizeof(unsigned long long));
  cudaMemset(bad, 0, sizeof(unsigned long long));
  const unsigned long long n = 1ull << 26;
  k_check<<<(unsigned)((n + 255) / 256), 256>>>(n, bad);
  unsigned long long h = 0;
  cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  cudaError_t e = cudaGetLastError();
  printf("mismatches %llu checked %llu %s\n", h, n, cudaGetErrorString(e));
  cudaFree(bad);
  return (h == 0 && e == cudaSuccess) ? 0 : 1;
}
