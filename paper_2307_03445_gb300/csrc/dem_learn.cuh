// dem_learn.cuh -- buffers and launchers of the learned rebuild rule and traces.
#pragma once
#include "dem_dev.cuh"

namespace dem {

// Per-bin statistics of the clumps whose centre of mass lies in the bin.
struct BinStats {
  uint32_t* chome;  // per clump: home bin key
  uint32_t* cnt;    // per bin: number of clumps
  int* vmax;        // per bin: largest speed bound (float bits)
  float* vsum;      // per bin: sum of speed bounds
  int* amax;        // per bin: largest acceleration (float bits)
};

struct FeatureScales {
  float h;      // time step
  float rmean;  // mean sphere radius
  float gmag;   // |g|
};

// Reference state of a trace window.
struct TraceRef {
  int4* vox;
  float4* off;
  double4_32a* pos;
  float4* q;
};

void launch_clump_home(const DevState& d, const BinStats& bs, cudaStream_t st);
void launch_bin_compact(const uint32_t* cnt, long long nbins, uint32_t* occ, uint32_t* n_occ,
                        cudaStream_t st);
void launch_bin_features(const BinStats& bs, const uint32_t* occ, long long n_occ, int nc,
                         const float* cand, const FeatureScales& fs, float* x, cudaStream_t st);
void launch_choose_margin(const uint32_t* occ, long long n_occ, int nc, const float* cand,
                          const float* y, float ln_need, float* bin_margin, cudaStream_t st);
void launch_clump_margin(const DevState& d, const uint32_t* chome, const float* bin_margin,
                         float floor_scale, float* cmargin, cudaStream_t st);
void launch_trace_ref(const DevState& d, const TraceRef& tr, cudaStream_t st);
void launch_trace_step(const DevState& d, const TraceRef& tr, const uint32_t* chome, int* dmax,
                       const uint32_t* occ, long long n_occ, int nc, const float* cand, int* T,
                       int step, cudaStream_t st);
// Writes the window's rows (features, log lifetime) to rows base.. of x / t,
// dropping those at or past cap.
void launch_trace_emit(long long n_rows, const float* xw, const int* T, int window, float* x,
                       float* t, long long base, long long cap, cudaStream_t st);

}  // namespace dem
