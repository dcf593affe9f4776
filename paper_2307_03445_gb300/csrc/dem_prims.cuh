// dem_prims.cuh -- device-wide scan and radix sort used by the binning.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace dem {

// Kernels launched by this library in this process (reported in dem_stats).
extern long long g_kernel_launches;
inline void count_launch(int n = 1) { g_kernel_launches += n; }

// Multiprocessors of the current device (read once).
int device_sms();

// Scratch bytes needed by exclusive_scan_u32 for n elements.
size_t scan_scratch_bytes(long long n);
// out[i] = sum of in[0..i-1] (32-bit); *d_total (device) = the 64-bit sum of all
// n inputs, so the caller can detect a total that does not fit 32 bits.
// in and out may alias.
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* scratch,
                        unsigned long long* d_total, cudaStream_t st);

// Scratch bytes needed by radix_sort_pairs for n elements.
size_t radix_scratch_bytes(long long n);
// Stable sort of (key, value) pairs by the low key_bits bits of the key.
// Returns 0 if the result is in keys/vals, 1 if it is in keys_alt/vals_alt.
int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                     long long n, int key_bits, void* scratch, unsigned long long* d_total,
                     cudaStream_t st);

}  // namespace dem
