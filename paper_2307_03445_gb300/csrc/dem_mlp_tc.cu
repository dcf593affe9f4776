// dem_mlp_tc.cu -- forward pass of the list-lifetime regressor on the tensor
// cores (tcgen05).  The network (6 -> 64 -> 64 -> 64 -> 1, ReLU) is three
// dense contractions per row: each persistent block takes tiles of 128 rows,
// keeps the three hidden-layer weight matrices resident in shared memory as
// bfloat16, and runs each layer as tcgen05.mma instructions (M = 128, N = 64,
// K = 16 per instruction) accumulating in FP32 in tensor memory.  Between
// layers every thread reads its row of the accumulator (tcgen05.ld), adds the
// bias, applies ReLU and writes the bfloat16 result back as the next layer's
// operand; the 64 -> 1 output layer runs on the CUDA cores in FP32.
//
// Operand tiles are K-major with the 128-byte swizzle: a row of 64 bfloat16
// values is 128 bytes, and its 16-byte chunk c is stored at chunk c ^ (row & 7).
// Waits on the MMA-completion barrier are bounded; a wait that runs out sets
// an error flag and the block stops issuing work; it frees its tensor memory
// only after a second bounded wait has seen the outstanding MMAs complete.
#include <cuda_bf16.h>

#include <cstdint>

#include "../../include/dem.h"
#include "dem_internal.cuh"
#include "dem_mlp.cuh"
#include "dem_prims.cuh"

namespace dem {

namespace {

constexpr int kRows = 128;        // rows per tile = the MMA's M
constexpr int kH = kMlpHidden;    // 64: the MMA's N and the K of layers 2 and 3
constexpr int kIn = kMlpIn;       // 6, padded to one K step of 16
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH;
constexpr int kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH;

// shared memory, from a 1024-byte aligned base (the swizzle atom)
constexpr uint32_t kSmA = 0;                         // 128 x 64 bf16 activations
constexpr uint32_t kSmW1 = kSmA + kRows * 128;       // 64 x 64 bf16 per weight matrix
constexpr uint32_t kSmW2 = kSmW1 + kH * 128;
constexpr uint32_t kSmW3 = kSmW2 + kH * 128;
constexpr uint32_t kSmF = kSmW3 + kH * 128;          // b1, b2, b3, w4 (64 floats each), b4
constexpr uint32_t kSmBar = kSmF + (4 * kH + 2) * 4; // MMA-completion barrier (8 bytes)
constexpr uint32_t kSmTmem = kSmBar + 8;             // tensor-memory address from tcgen05.alloc
constexpr uint32_t kSmBytes = kSmTmem + 8;
constexpr uint32_t kSmLaunch = kSmBytes + 1024;      // room to align the base
static_assert(kSmBar % 8 == 0, "barrier alignment");
constexpr uint32_t kTmemCols = 64;                   // one 128 x 64 FP32 accumulator

// Instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in
// bfloat16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 in bits 17-22, M / 16 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);

// Byte offset of element (row, k < 64) in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  return (uint32_t)row * 128u + ((uint32_t)(((k >> 3) ^ row) & 7) << 4) + ((uint32_t)(k & 7) << 1);
}

// Shared-memory matrix descriptor of a 128-byte-swizzled K-major tile: start
// address / 16 (bits 0-13), leading offset unused for this layout (1), stride
// between 8-row groups 1024 bytes (bits 32-45, in 16-byte units), descriptor
// version 1 (bits 46-47), swizzle mode 128 bytes (bits 61-63 = 2).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

// Bounded wait (`tries` polls) for the barrier's phase with the given parity.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, int tries = 1 << 20) {
  for (int i = 0; i < tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void st_bf16(unsigned char* sm, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(sm + off) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(kRows) k_mlp_forward_tc(const __nv_bfloat16* __restrict__ w,
                                                          const float* __restrict__ x, long long n,
                                                          float* __restrict__ y, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023u) & ~static_cast<uintptr_t>(1023u));
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
  const int t = threadIdx.x, warp = t >> 5;
  float* sf = reinterpret_cast<float*>(sm + kSmF);
  // weights: the three hidden matrices as swizzled bf16 tiles (W1 zero past
  // its 6 inputs), the biases and the output row as float
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int i = t; i < kH * 64; i += kRows) {
    const int r = i >> 6, k = i & 63;
    *reinterpret_cast<__nv_bfloat16*>(sm + kSmW1 + sw128(r, k)) = k < kIn ? w[kOffW1 + r * kIn + k] : zero;
    *reinterpret_cast<__nv_bfloat16*>(sm + kSmW2 + sw128(r, k)) = w[kOffW2 + r * kH + k];
    *reinterpret_cast<__nv_bfloat16*>(sm + kSmW3 + sw128(r, k)) = w[kOffW3 + r * kH + k];
  }
  for (int i = t; i < kH; i += kRows) {
    sf[i] = __bfloat162float(w[kOffB1 + i]);
    sf[kH + i] = __bfloat162float(w[kOffB2 + i]);
    sf[2 * kH + i] = __bfloat162float(w[kOffB3 + i]);
    sf[3 * kH + i] = __bfloat162float(w[kOffW4 + i]);
  }
  if (t == 0) sf[4 * kH] = __bfloat162float(w[kOffB4]);
  const uint32_t bar = sbase + kSmBar;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sbase + kSmTmem),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + kSmTmem);
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  uint32_t parity = 0;
  bool ok = true;
  const long long ntiles = (n + kRows - 1) / kRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r = tile * kRows + t;
    // layer-1 operand: this row's features, zero-padded to one K step
#pragma unroll
    for (int k = 0; k < 16; ++k)
      st_bf16(sm, kSmA + sw128(t, k), (k < kIn && r < n) ? x[r * kIn + k] : 0.f);
    for (int layer = 0; layer < 3; ++layer) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (t == 0) {
        const uint32_t wt = sbase + (layer == 0 ? kSmW1 : (layer == 1 ? kSmW2 : kSmW3));
        const int ksteps = layer == 0 ? 1 : kH / 16;
        for (int s = 0; s < ksteps; ++s)
          mma_bf16(tmem, sdesc(sbase + kSmA + 32u * s), sdesc(wt + 32u * s), s > 0 ? 1u : 0u);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
      }
      // every thread waits; the block goes on only if all of them saw the
      // phase complete, so that nothing is issued after a wait ran out
      ok = __syncthreads_and(bar_wait(bar, parity) ? 1 : 0) != 0;
      if (!ok) break;
      parity ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint32_t c[4][16];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(tlane + 16u * q, c[q]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const float* bias = sf + layer * kH;
      if (layer < 2) {
        // the next layer's operand: ReLU(acc + b) in bf16 (the MMA that read
        // the previous operand has completed)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < 16; ++j)
            st_bf16(sm, kSmA + sw128(t, 16 * q + j),
                    fmaxf(__uint_as_float(c[q][j]) + bias[16 * q + j], 0.f));
      } else {
        float s = sf[4 * kH];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int j = 0; j < 16; ++j)
            s = fmaf(sf[3 * kH + 16 * q + j], fmaxf(__uint_as_float(c[q][j]) + bias[16 * q + j], 0.f), s);
        if (r < n) y[r] = s;
      }
    }
    if (!ok) break;  // a wait ran out: stop this block
  }
  bool drained = true;
  if (!ok) {
    if (t == 0 && err) atomicOr(err, kFlagTimeout);
    // the MMAs of the phase that did not complete may still write the
    // accumulator: wait for that phase once more, 16 times longer, and give
    // the tensor memory back only if it completed (freeing columns that an
    // MMA still writes would hand them to the next block on this SM)
    drained = __syncthreads_and(bar_wait(bar, parity, 1 << 24) ? 1 : 0) != 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

void mlp_forward_tc_dev(const __nv_bfloat16* w, const float* x, long long n, float* y, int* err,
                        cudaStream_t st) {
  if (n <= 0) return;
  const long long tiles = (n + kRows - 1) / kRows;
  const long long cap = (long long)device_sms() * 4;
  k_mlp_forward_tc<<<(unsigned)(tiles < cap ? tiles : cap), kRows, kSmLaunch, st>>>(w, x, n, y, err);
  count_launch();
}

}  // namespace dem
