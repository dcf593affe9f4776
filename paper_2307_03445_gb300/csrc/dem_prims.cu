// dem_prims.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Scan: reduce-then-scan over tiles of 4096 counts (uint32 in, uint32 out, a
// uint64 grand total so that an overflow of the 32-bit offsets is detected).
// Sort: 8-bit digits; per pass a per-tile digit histogram, a scan of the
// (digit-major, tile-minor) histogram matrix, and a scatter in which every
// tile ranks its keys stably with warp match/ballot and shared counters.
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

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
namespace {
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, long long n, int shift,
                             long long ntiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
  for (int i = 0; i < kSortItems; ++i) {
    long long idx = base + (long long)i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                long long n, int shift, long long ntiles,
                                const uint32_t* __restrict__ offs, uint32_t* __restrict__ okeys,
                                uint32_t* __restrict__ ovals) {
  __shared__ uint32_t s_cnt[kSortWarps][256];
  __shared__ uint32_t s_pre[kSortWarps][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_goff[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int w = 0; w < kSortWarps; ++w) s_cnt[w][tid] = 0;
  s_run[tid] = 0;
  s_goff[tid] = offs[(long long)tid * ntiles + blockIdx.x];
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  const long long base = (long long)blockIdx.x * kSortTile;
  for (int it = 0; it < kSortItems; ++it) {
    const long long idx = base + (long long)it * kSortThreads + tid;
    const bool valid = idx < n;
    uint32_t key = valid ? keys[idx] : 0u;
    uint32_t val = valid ? vals[idx] : 0u;
    // invalid lanes use digit 256 (never matches a real digit)
    const uint32_t digit = valid ? ((key >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const uint32_t rank = __popc(peers & lt_mask);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) s_cnt[warp][digit] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = s_run[tid];
      for (int w = 0; w < kSortWarps; ++w) {
        s_pre[w][tid] = run;
        run += s_cnt[w][tid];
        s_cnt[w][tid] = 0;
      }
      s_run[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t dst = s_goff[digit] + s_pre[warp][digit] + rank;
      okeys[dst] = key;
      ovals[dst] = val;
    }
    __syncthreads();
  }
}
}  // namespace

size_t radix_scratch_bytes(long long n) {
  long long ntiles = (n + kSortTile - 1) / kSortTile;
  size_t hist = sizeof(uint32_t) * 256 * (size_t)(ntiles > 0 ? ntiles : 1);
  return 2 * hist + scan_scratch_bytes(256 * (ntiles > 0 ? ntiles : 1)) + 64;
}

int radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                     long long n, int key_bits, void* scratch, unsigned long long* d_total,
                     cudaStream_t st) {
  if (n <= 1) return 0;
  const long long ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* hist = (uint32_t*)scratch;
  uint32_t* offs = hist + 256 * ntiles;
  void* sscr = (void*)(offs + 256 * ntiles);
  // align the scan scratch to 16 bytes
  sscr = (void*)(((uintptr_t)sscr + 15) & ~(uintptr_t)15);
  int passes = (key_bits + 7) / 8;
  if (passes < 1) passes = 1;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ki, n, shift, ntiles, hist);
    exclusive_scan_u32(hist, offs, 256 * ntiles, sscr, d_total, st);
    k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ki, vi, n, shift, ntiles, offs, ko,
                                                                 vo);
    count_launch(2);
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  return passes & 1;  // 1: the sorted data is in the *_alt buffers
}

}  // namespace dem
