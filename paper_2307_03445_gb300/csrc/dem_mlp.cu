// dem_mlp.cu -- the learned contact-list lifetime regressor (an extension: the
// paper uses a fixed, velocity-bound margin).  6 inputs -> 3 hidden ReLU layers
// of 64 -> 1 output; BF16 weights, FP32 accumulation.  Forward, mean-squared-
// error gradient and Adam run as hand-written kernels; the parameter layout is
// one flat vector, layer by layer, W row-major [out][in] then b.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/dem.h"
#include "dem_mlp.cuh"
#include "dem_prims.cuh"

namespace dem {

namespace {

constexpr int kIn = kMlpIn, kH = kMlpHidden;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH;
constexpr int kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH;
static_assert(kOffB4 + 1 == kMlpParams, "parameter layout");

// Weights (BF16 in global memory) widened to float in shared memory.
__device__ __forceinline__ void stage_weights(const __nv_bfloat16* __restrict__ w, float* sw) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
  __syncthreads();
}

// Dense layer out = relu?(W in + b), W row-major [NOUT][NIN] in shared memory.
template <int NIN, int NOUT, bool RELU>
__device__ __forceinline__ void dense(const float* __restrict__ sw, int offW, int offB,
                                      const float (&in)[NIN], float (&out)[NOUT]) {
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    float s = sw[offB + o];
#pragma unroll
    for (int i = 0; i < NIN; ++i) s = fmaf(sw[offW + o * NIN + i], in[i], s);
    out[o] = RELU ? fmaxf(s, 0.f) : s;
  }
}

__global__ void __launch_bounds__(128) k_mlp_forward(const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ x, long long n,
                                                     float* __restrict__ y) {
  extern __shared__ float sw[];
  stage_weights(w, sw);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    float h0[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) h0[i] = x[k * kIn + i];
    float h1[kH], h2[kH];
    dense<kIn, kH, true>(sw, kOffW1, kOffB1, h0, h1);
    dense<kH, kH, true>(sw, kOffW2, kOffB2, h1, h2);
    dense<kH, kH, true>(sw, kOffW3, kOffB3, h2, h1);
    float out[1];
    dense<kH, 1, false>(sw, kOffW4, kOffB4, h1, out);
    y[k] = out[0];
  }
}

// Gradient of (1/n) sum (y - t)^2, accumulated per block in shared memory and
// added to g (global, zeroed by the caller); the loss sum goes to *loss.
__global__ void __launch_bounds__(64) k_mlp_grad(const __nv_bfloat16* __restrict__ w,
                                                 const float* __restrict__ x,
                                                 const float* __restrict__ t, long long n,
                                                 float inv_n, float* __restrict__ g,
                                                 double* __restrict__ loss) {
  extern __shared__ float smem[];
  float* sw = smem;
  float* sg = smem + kMlpParams;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sg[i] = 0.f;
  stage_weights(w, sw);
  float lsum = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    float h0[kIn], h1[kH], h2[kH], h3[kH], out[1];
#pragma unroll
    for (int i = 0; i < kIn; ++i) h0[i] = x[k * kIn + i];
    dense<kIn, kH, true>(sw, kOffW1, kOffB1, h0, h1);
    dense<kH, kH, true>(sw, kOffW2, kOffB2, h1, h2);
    dense<kH, kH, true>(sw, kOffW3, kOffB3, h2, h3);
    dense<kH, 1, false>(sw, kOffW4, kOffB4, h3, out);
    const float e = out[0] - t[k];
    lsum += e * e;
    const float dy = 2.f * e * inv_n;
    // output layer
    atomicAdd(&sg[kOffB4], dy);
    float d3[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) {
      atomicAdd(&sg[kOffW4 + i], dy * h3[i]);
      d3[i] = h3[i] > 0.f ? sw[kOffW4 + i] * dy : 0.f;
    }
    // hidden layer 3: W3 [kH][kH], input h2
    float d2[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) d2[i] = 0.f;
    for (int o = 0; o < kH; ++o) {
      const float dv = d3[o];
      if (dv == 0.f) continue;
      atomicAdd(&sg[kOffB3 + o], dv);
#pragma unroll
      for (int i = 0; i < kH; ++i) {
        atomicAdd(&sg[kOffW3 + o * kH + i], dv * h2[i]);
        d2[i] = fmaf(sw[kOffW3 + o * kH + i], dv, d2[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < kH; ++i) d2[i] = h2[i] > 0.f ? d2[i] : 0.f;
    // hidden layer 2: W2, input h1
    float d1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) d1[i] = 0.f;
    for (int o = 0; o < kH; ++o) {
      const float dv = d2[o];
      if (dv == 0.f) continue;
      atomicAdd(&sg[kOffB2 + o], dv);
#pragma unroll
      for (int i = 0; i < kH; ++i) {
        atomicAdd(&sg[kOffW2 + o * kH + i], dv * h1[i]);
        d1[i] = fmaf(sw[kOffW2 + o * kH + i], dv, d1[i]);
      }
    }
    // hidden layer 1: W1 [kH][kIn], input h0
    for (int o = 0; o < kH; ++o) {
      const float dv = h1[o] > 0.f ? d1[o] : 0.f;
      if (dv == 0.f) continue;
      atomicAdd(&sg[kOffB1 + o], dv);
#pragma unroll
      for (int i = 0; i < kIn; ++i) atomicAdd(&sg[kOffW1 + o * kIn + i], dv * h0[i]);
    }
  }
  // block loss and gradient to global
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
    if (sg[i] != 0.f) atomicAdd(&g[i], sg[i]);
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wq, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  wq[i] = __float2bfloat16_rn(pi);
}

__global__ void k_gather_rows(const long long* __restrict__ idx, long long b,
                              const float* __restrict__ x, const float* __restrict__ t,
                              float* __restrict__ bx, float* __restrict__ bt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b) return;
  const long long r = idx[i];
  for (int k = 0; k < kIn; ++k) bx[i * kIn + k] = x[r * kIn + k];
  bt[i] = t[r];
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpParams) wq[i] = __float2bfloat16_rn(p[i]);
}

int g_sms = 0;
int sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 132;
  }
  return g_sms;
}

}  // namespace

namespace {

// The dynamic shared-memory limit of a kernel is a per-device setting: it is
// raised once on every device the library launches the kernel on (a flag per
// device and kernel, set only when the call succeeded).
constexpr int kAttrMaxDevices = 64;
std::mutex g_attr_mu;

template <typename K>
bool smem_attr_once(K kernel, int slot, size_t smem) {
  static bool done[2][kAttrMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrMaxDevices) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (done[slot][dev]) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done[slot][dev] = true;
  return true;
}

}  // namespace

int mlp_forward_dev(const __nv_bfloat16* w, const float* x, long long n, float* y, cudaStream_t st) {
  if (n <= 0) return DEM_OK;
  const size_t smem = sizeof(float) * kMlpParams;
  if (!smem_attr_once(k_mlp_forward, 0, smem)) return DEM_ERR_CUDA;
  const long long want = (n + 127) / 128;
  const long long cap = (long long)sms() * 4;
  k_mlp_forward<<<(unsigned)(want < cap ? want : cap), 128, smem, st>>>(w, x, n, y);
  count_launch();
  return DEM_OK;
}

}  // namespace dem

using namespace dem;

struct dem_mlp {
  int device = 0;
  cudaStream_t st = nullptr;
  float* p = nullptr;   // fp32 master parameters
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  __nv_bfloat16* wq = nullptr;
  double* loss = nullptr;
  int adam_step = 0;
  std::string err;
};

namespace {
int mlp_fail(dem_mlp* m, int code, const char* msg) {
  if (m) m->err = msg;
  return code;
}

// Host data -> device scratch of the mlp (grown on demand).
struct Staging {
  void* p = nullptr;
  size_t bytes = 0;
};
thread_local Staging g_stage;
void* stage(size_t bytes, cudaStream_t st) {
  if (g_stage.bytes < bytes) {
    if (g_stage.p) cudaFreeAsync(g_stage.p, st);
    g_stage.p = nullptr;
    if (cudaMallocAsync(&g_stage.p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      g_stage.bytes = 0;
      return nullptr;
    }
    g_stage.bytes = bytes;
  }
  return g_stage.p;
}

int grad_pass(dem_mlp* M, long long n, const float* dx, const float* dt, double* loss_out) {
  cudaMemsetAsync(M->g, 0, sizeof(float) * kMlpParams, M->st);
  cudaMemsetAsync(M->loss, 0, sizeof(double), M->st);
  const size_t smem = 2 * sizeof(float) * kMlpParams;
  if (!smem_attr_once(k_mlp_grad, 1, smem)) return mlp_fail(M, DEM_ERR_CUDA, "gradient kernel attribute");
  const long long want = (n + 63) / 64;
  const long long cap = (long long)sms() * 2;
  k_mlp_grad<<<(unsigned)(want < cap ? want : cap), 64, smem, M->st>>>(M->wq, dx, dt, n,
                                                                        1.f / (float)n, M->g, M->loss);
  count_launch();
  if (loss_out) {
    double h = 0;
    if (cudaMemcpyAsync(&h, M->loss, sizeof(double), cudaMemcpyDeviceToHost, M->st) != cudaSuccess ||
        cudaStreamSynchronize(M->st) != cudaSuccess) {
      cudaGetLastError();
      return mlp_fail(M, DEM_ERR_CUDA, "gradient pass");
    }
    *loss_out = h / (double)n;
  }
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}
}  // namespace

extern "C" {

int dem_mlp_num_params(void) { return kMlpParams; }

int dem_mlp_create(int device, dem_mlp** out) {
  if (!out) return DEM_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return DEM_ERR_CUDA;
  }
  dem_mlp* M = new dem_mlp();
  M->device = device;
  if (cudaStreamCreateWithFlags(&M->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete M;
    return DEM_ERR_CUDA;
  }
  const size_t pb = sizeof(float) * kMlpParams;
  if (cudaMalloc(&M->p, pb) != cudaSuccess || cudaMalloc(&M->m, pb) != cudaSuccess ||
      cudaMalloc(&M->v, pb) != cudaSuccess || cudaMalloc(&M->g, pb) != cudaSuccess ||
      cudaMalloc(&M->wq, sizeof(__nv_bfloat16) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&M->loss, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    dem_mlp_destroy(M);
    return DEM_ERR_OOM;
  }
  // He-style initialisation from a fixed seed
  std::vector<float> h(kMlpParams, 0.f);
  std::mt19937_64 rng(0x5eed);
  auto fill = [&](int off, int nout, int nin) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)nin));
    for (int i = 0; i < nout * nin; ++i) h[off + i] = nd(rng);
  };
  fill(kOffW1, kH, kIn);
  fill(kOffW2, kH, kH);
  fill(kOffW3, kH, kH);
  fill(kOffW4, 1, kH);
  int rc = dem_mlp_set_params(M, h.data());
  if (rc) {
    dem_mlp_destroy(M);
    return rc;
  }
  *out = M;
  return DEM_OK;
}

void dem_mlp_destroy(dem_mlp* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  cudaFree(M->p); cudaFree(M->m); cudaFree(M->v); cudaFree(M->g); cudaFree(M->wq); cudaFree(M->loss);
  if (M->st) cudaStreamDestroy(M->st);
  delete M;
}

int dem_mlp_set_params(dem_mlp* M, const float* params) {
  if (!M || !params) return DEM_ERR_INVALID_ARG;
  for (int i = 0; i < kMlpParams; ++i)
    if (!std::isfinite(params[i])) return mlp_fail(M, DEM_ERR_NONFINITE, "non-finite parameter");
  cudaSetDevice(M->device);
  cudaMemcpyAsync(M->p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, M->st);
  cudaMemsetAsync(M->m, 0, sizeof(float) * kMlpParams, M->st);
  cudaMemsetAsync(M->v, 0, sizeof(float) * kMlpParams, M->st);
  k_to_bf16<<<(kMlpParams + 255) / 256, 256, 0, M->st>>>(M->p, M->wq);
  count_launch();
  M->adam_step = 0;
  cudaStreamSynchronize(M->st);
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}

int dem_mlp_get_params(dem_mlp* M, float* params) {
  if (!M || !params) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(M->device);
  cudaMemcpyAsync(params, M->p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, M->st);
  cudaStreamSynchronize(M->st);
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}

int dem_mlp_forward(dem_mlp* M, long long n, const float* x, float* y) {
  if (!M || n < 0 || (n > 0 && (!x || !y))) return DEM_ERR_INVALID_ARG;
  if (n == 0) return DEM_OK;
  cudaSetDevice(M->device);
  char* buf = (char*)stage(sizeof(float) * (size_t)n * (kIn + 1), M->st);
  if (!buf) return mlp_fail(M, DEM_ERR_OOM, "staging");
  float* dx = (float*)buf;
  float* dy = dx + (size_t)n * kIn;
  cudaMemcpyAsync(dx, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, M->st);
  if (mlp_forward_dev(M->wq, dx, n, dy, M->st) != DEM_OK)
    return mlp_fail(M, DEM_ERR_CUDA, "forward kernel attribute");
  cudaMemcpyAsync(y, dy, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, M->st);
  cudaStreamSynchronize(M->st);
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}

int dem_mlp_forward_tc(dem_mlp* M, long long n, const float* x, float* y) {
  if (!M || n < 0 || (n > 0 && (!x || !y))) return DEM_ERR_INVALID_ARG;
  if (n == 0) return DEM_OK;
  cudaSetDevice(M->device);
  // rows, outputs and the timeout flag in one staging buffer
  char* buf = (char*)stage(sizeof(float) * (size_t)n * (kIn + 1) + 16, M->st);
  if (!buf) return mlp_fail(M, DEM_ERR_OOM, "staging");
  float* dx = (float*)buf;
  float* dy = dx + (size_t)n * kIn;
  int* dflag = (int*)(dy + n);
  cudaMemsetAsync(dflag, 0, sizeof(int), M->st);
  cudaMemcpyAsync(dx, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, M->st);
  mlp_forward_tc_dev(M->wq, dx, n, dy, dflag, M->st);
  int flag = 0;
  cudaMemcpyAsync(y, dy, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, M->st);
  cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, M->st);
  cudaStreamSynchronize(M->st);
  if (cudaGetLastError() != cudaSuccess) return DEM_ERR_CUDA;
  if (flag) return mlp_fail(M, DEM_ERR_TIMEOUT, "tensor-core forward: a barrier wait ran out");
  return DEM_OK;
}

int dem_mlp_loss_grad(dem_mlp* M, long long n, const float* x, const float* t, double* loss,
                      float* grad) {
  if (!M || n <= 0 || !x || !t) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(M->device);
  char* buf = (char*)stage(sizeof(float) * (size_t)n * (kIn + 1), M->st);
  if (!buf) return mlp_fail(M, DEM_ERR_OOM, "staging");
  float* dx = (float*)buf;
  float* dt = dx + (size_t)n * kIn;
  cudaMemcpyAsync(dx, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, M->st);
  cudaMemcpyAsync(dt, t, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, M->st);
  int rc = grad_pass(M, n, dx, dt, loss);
  if (grad) {
    cudaMemcpyAsync(grad, M->g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, M->st);
    cudaStreamSynchronize(M->st);
  }
  return rc;
}

int dem_mlp_train(dem_mlp* M, long long n, const float* x, const float* t, int steps, int batch,
                  float lr, unsigned long long seed, double* final_loss) {
  if (!M || n <= 0 || !x || !t || steps < 0 || batch <= 0 || !(lr > 0)) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(M->device);
  const long long b = batch < n ? batch : n;
  char* buf = (char*)stage(sizeof(float) * (size_t)(n + b) * (kIn + 1), M->st);
  if (!buf) return mlp_fail(M, DEM_ERR_OOM, "staging");
  float* dx = (float*)buf;
  float* dt = dx + (size_t)n * kIn;
  float* bx = dt + (size_t)n;
  float* bt = bx + (size_t)b * kIn;
  cudaMemcpyAsync(dx, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, M->st);
  cudaMemcpyAsync(dt, t, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, M->st);
  std::mt19937_64 rng(seed);
  std::vector<long long> order(n);
  for (long long i = 0; i < n; ++i) order[i] = i;
  long long* dorder = nullptr;
  if (b < n && cudaMallocAsync((void**)&dorder, sizeof(long long) * (size_t)n, M->st) != cudaSuccess) {
    cudaGetLastError();
    return mlp_fail(M, DEM_ERR_OOM, "permutation");
  }
  long long pos = n;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int s = 0; s < steps; ++s) {
    const float* mx = dx;
    const float* mt = dt;
    long long nb = n;
    if (b < n) {
      // minibatches are consecutive slices of a shuffled permutation (one per epoch)
      if (pos + b > n) {
        std::shuffle(order.begin(), order.end(), rng);
        cudaMemcpyAsync(dorder, order.data(), sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice,
                        M->st);
        cudaStreamSynchronize(M->st);
        pos = 0;
      }
      k_gather_rows<<<(unsigned)((b + 255) / 256), 256, 0, M->st>>>(dorder + pos, b, dx, dt, bx, bt);
      count_launch();
      mx = bx;
      mt = bt;
      nb = b;
      pos += b;
    }
    int rc = grad_pass(M, nb, mx, mt, nullptr);
    if (rc) return rc;
    ++M->adam_step;
    const float c1 = 1.f - std::pow(b1, (float)M->adam_step);
    const float c2 = 1.f - std::pow(b2, (float)M->adam_step);
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, M->st>>>(M->p, M->m, M->v, M->g, M->wq, lr, b1, b2,
                                                        eps, c1, c2);
    count_launch();
  }
  if (dorder) cudaFreeAsync(dorder, M->st);
  double l = 0.0;
  int rc = grad_pass(M, n, dx, dt, &l);
  if (final_loss) *final_loss = l;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Loss and gradient without allocation.  dem_mlp_loss_grad stages its inputs
// in a buffer that grows with cudaMallocAsync / cudaFreeAsync.  Some callers
// cannot take that: a process whose device memory is held in full by another
// allocator (a framework's caching allocator sized to the whole GPU), where
// the allocation fails, and a host loop that must not wait on the implicit
// device-wide synchronisation of a free.  This variant runs the same gradient
// kernel on one fixed scratch array that is part of the library's module
// image: the rows, the targets and the two accumulators.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNaLossOff = 0;                                   // double loss sum
constexpr size_t kNaGradOff = 256;                                 // kMlpParams floats
constexpr size_t kNaGradBytes = (sizeof(float) * kMlpParams + 255) / 256 * 256;
constexpr size_t kNaXOff = kNaGradOff + kNaGradBytes;              // rows, 6 floats each
constexpr size_t kNaTOff = kNaXOff + sizeof(float) * kIn * DEM_MLP_NOALLOC_MAX_ROWS;
constexpr size_t kNaBytes = kNaTOff + sizeof(float) * DEM_MLP_NOALLOC_MAX_ROWS;
static_assert(kNaXOff % 256 == 0 && kNaTOff % 256 == 0, "scratch alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the scratch array, looked up once per device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_addr[kNaMaxDevices] = {};

int noalloc_scratch(dem_mlp* M, unsigned char** out) {
  if (M->device < 0 || M->device >= kNaMaxDevices)
    return mlp_fail(M, DEM_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[M->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return mlp_fail(M, DEM_ERR_CUDA, "scratch symbol address");
    }
    g_na_addr[M->device] = p;
  }
  if (!smem_attr_once(k_mlp_grad, 1, 2 * sizeof(float) * kMlpParams))
    return mlp_fail(M, DEM_ERR_CUDA, "gradient kernel attribute");
  *out = (unsigned char*)g_na_addr[M->device];
  return DEM_OK;
}

}  // namespace

extern "C" int dem_mlp_loss_grad_noalloc(dem_mlp* M, long long n, const float* x, const float* t,
                                         double* loss, float* grad) {
  if (!M || n <= 0 || !x || !t) return DEM_ERR_INVALID_ARG;
  if (n > DEM_MLP_NOALLOC_MAX_ROWS)
    return mlp_fail(M, DEM_ERR_CAPACITY, "more rows than the fixed scratch holds");
  if (cudaSetDevice(M->device) != cudaSuccess) {
    cudaGetLastError();
    return DEM_ERR_CUDA;
  }
  unsigned char* s = nullptr;
  int rc = noalloc_scratch(M, &s);
  if (rc) return rc;
  double* d_loss = (double*)(s + kNaLossOff);
  float* d_grad = (float*)(s + kNaGradOff);
  float* d_x = (float*)(s + kNaXOff);
  float* d_t = (float*)(s + kNaTOff);
  // the two accumulators start at zero on every call; rows and targets are
  // overwritten up to n
  if (cudaMemsetAsync(s, 0, kNaXOff, M->st) != cudaSuccess ||
      cudaMemcpyAsync(d_x, x, sizeof(float) * (size_t)n * kIn, cudaMemcpyHostToDevice, M->st) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_t, t, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, M->st) != cudaSuccess) {
    cudaGetLastError();
    return mlp_fail(M, DEM_ERR_CUDA, "staging the rows into the fixed scratch");
  }
  const long long want = (n + 63) / 64;
  const long long cap = (long long)sms() * 2;
  k_mlp_grad<<<(unsigned)(want < cap ? want : cap), 64, 2 * sizeof(float) * kMlpParams, M->st>>>(
      M->wq, d_x, d_t, n, 1.f / (float)n, d_grad, d_loss);
  count_launch();
  double h = 0.0;
  cudaError_t e = cudaMemcpyAsync(&h, d_loss, sizeof(double), cudaMemcpyDeviceToHost, M->st);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, d_grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, M->st);
  // the host buffers must outlive their copies: wait even when one failed to enqueue
  const cudaError_t es = cudaStreamSynchronize(M->st);
  if (e != cudaSuccess || es != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return mlp_fail(M, DEM_ERR_CUDA, "gradient pass on the fixed scratch");
  }
  if (loss) *loss = h / (double)n;
  return DEM_OK;
}

namespace dem {
const __nv_bfloat16* mlp_weights(const dem_mlp* M) { return M ? M->wq : nullptr; }
}  // namespace dem
