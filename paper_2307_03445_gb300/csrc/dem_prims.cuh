// dem_prims.cuh -- device-wide scan used by the binning and the list build.
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

}  // namespace dem
