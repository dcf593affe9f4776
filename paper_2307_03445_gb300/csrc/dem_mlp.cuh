// dem_mlp.cuh -- shapes of the lifetime regressor and its device entry points.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

struct dem_mlp;

namespace dem {

constexpr int kMlpIn = 6;       // per-bin features
constexpr int kMlpHidden = 64;  // width of the three hidden layers
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + 2 * (kMlpHidden * kMlpHidden + kMlpHidden) +
                           kMlpHidden + 1;

// y[k] = f(x[k * kMlpIn .. +kMlpIn]) for k < n (device pointers, BF16 weights).
int mlp_forward_dev(const __nv_bfloat16* w, const float* x, long long n, float* y, cudaStream_t st);
// The same on the tensor cores (tcgen05): every layer's input rounded to
// bfloat16, FP32 accumulation.  A bounded wait that runs out ors
// kFlagTimeout into *err (device, may be NULL).
void mlp_forward_tc_dev(const __nv_bfloat16* w, const float* x, long long n, float* y, int* err,
                        cudaStream_t st);
const __nv_bfloat16* mlp_weights(const dem_mlp* m);

}  // namespace dem
