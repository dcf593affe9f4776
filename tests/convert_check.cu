// Test program: the integer-pipe f32<->f64 conversions of the library against
// the hardware conversions, on random bit patterns and edge cases.
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
  if (!same_f || !same_d) atomicAdd(bad, 1ull);
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
