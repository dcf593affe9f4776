// dem_prims.cu -- device-wide exclusive scan.
//
// Reduce-then-scan over tiles of 4096 counts (uint32 in, uint32 out, a uint64
// grand total so that an overflow of the 32-bit offsets is detected).
#include "dem_prims.cuh"

namespace dem {

namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Exclusive block scan of one value per thread (blockDim.x a multiple of 32).
__device__ void block_excl_scan(unsigned long long v, unsigned long long* out_excl) {
  __shared__ unsigned long long warp_tot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned long long inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long t = lane < nwarps ? warp_tot[lane] : 0ull;
    unsigned long long ti = warp_incl_scan(t);
    if (lane < nwarps) warp_tot[lane] = ti - t;
  }
  __syncthreads();
  *out_excl = warp_tot[warp] + inc - v;
  __syncthreads();
}

__global__ void k_tile_sums(const uint32_t* __restrict__ in, long long n,
                            unsigned long long* __restrict__ tile_sums) {
  const long long base = (long long)blockIdx.x * kScanTile;
  unsigned long long s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    long long idx = base + (long long)i * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  // block reduce
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ unsigned long long ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long t = threadIdx.x < (kScanThreads >> 5) ? ws[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the tile sums in place, grand total to *total.
__global__ void k_scan_tile_sums(unsigned long long* __restrict__ sums, long long ntiles,
                                 unsigned long long* __restrict__ total) {
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < ntiles; base += blockDim.x) {
    long long i = base + threadIdx.x;
    unsigned long long v = i < ntiles ? sums[i] : 0ull;
    unsigned long long ex;
    block_excl_scan(v, &ex);
    unsigned long long c = carry;
    if (i < ntiles) sums[i] = c + ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c + ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, long long n,
                             const unsigned long long* __restrict__ tile_off) {
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  unsigned long long s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    long long idx = base + i;
    v[i] = idx < n ? in[idx] : 0u;
    s += v[i];
  }
  unsigned long long ex;
  block_excl_scan(s, &ex);
  unsigned long long run = tile_off[blockIdx.x] + ex;
  for (int i = 0; i < kScanItems; ++i) {
    long long idx = base + i;
    if (idx < n) out[idx] = (uint32_t)run;
    run += v[i];
  }
}
}  // namespace

size_t scan_scratch_bytes(long long n) {
  long long ntiles = (n + kScanTile - 1) / kScanTile;
  return sizeof(unsigned long long) * (size_t)(ntiles + 2);
}

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, long long n, void* scratch,
                        unsigned long long* d_total, cudaStream_t st) {
  long long ntiles = (n + kScanTile - 1) / kScanTile;
  unsigned long long* sums = (unsigned long long*)scratch;
  if (ntiles == 0) {
    cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), st);
    return;
  }
  k_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums);
  k_scan_tile_sums<<<1, 1024, 0, st>>>(sums, ntiles, d_total);
  k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, n, sums);
  count_launch(3);
}

long long g_kernel_launches = 0;

int device_sms() {
  static int n = 0;
  if (n <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 148;
    }
  }
  return n;
}

}  // namespace dem
