// dem_learn.cu -- kernels of the learned rebuild rule and of its training traces
// (an extension; the paper's margin is fixed by the maximum velocity).
//
// Every clump belongs to the detection bin holding its centre of mass (its
// home bin).  Per occupied bin the features of the regressor are built from
// the number of clumps, their largest and mean speed bound, their largest
// acceleration of the last step, the candidate margin, the mean sphere
// radius and gravity; the same displacement bound as the per-step
// certificate defines the lifetime labels of the traces.
#include "dem_dev.cuh"
#include "dem_learn.cuh"
#include "dem_mlp.cuh"
#include "dem_prims.cuh"

namespace dem {

namespace {

__device__ __forceinline__ float clump_speed_bound(const DevState& d, long long c, int tpl) {
  if (d.prec == 1) {
    const float4 v = d.mv32[c], w = d.mw32[c];
    return sqrtf(v.x * v.x + v.y * v.y + v.z * v.z) +
           sqrtf(w.x * w.x + w.y * w.y + w.z * w.z) * d.tpbound[tpl];
  }
  const double4_32a v = d.mv64[c], w = d.mw64[c];
  return (float)(sqrt(v.x * v.x + v.y * v.y + v.z * v.z) +
                 sqrt(w.x * w.x + w.y * w.y + w.z * w.z) * d.tpbound[tpl]);
}

// Home bin key of a clump (float arithmetic: a feature, not a contact decision).
__device__ __forceinline__ uint32_t clump_home(const DevState& d, long long c, const SceneGrid& g) {
  float x[3];
  if (d.prec == 1) {
    const int4 v = d.cvox[c];
    const float4 o = d.coff[c];
    const float kV = (float)kVoxel;
    x[0] = (float)v.x * kV + o.x; x[1] = (float)v.y * kV + o.y; x[2] = (float)v.z * kV + o.z;
  } else {
    const double4_32a p = d.cpos[c];
    x[0] = (float)(p.x - g.lo[0]); x[1] = (float)(p.y - g.lo[1]); x[2] = (float)(p.z - g.lo[2]);
  }
  const float Lm = (float)g.L * (float)(1.0 / kDetScale);
  int b[3];
  for (int k = 0; k < 3; ++k) {
    int v = (int)floorf(x[k] / Lm);
    b[k] = v < 0 ? 0 : (v > g.dims[k] - 1 ? g.dims[k] - 1 : v);
  }
  return g.key_base + (uint32_t)((b[2] * g.dims[1] + b[1]) * g.dims[0] + b[0]);
}

__global__ void k_clump_home(DevState d, BinStats bs) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const int2 ci = d.cinfo[c];
  const SceneGrid g = d.grids[ci.y];
  const uint32_t key = clump_home(d, c, g);
  bs.chome[c] = key;
  const float sp = clump_speed_bound(d, c, ci.x);
  const float ac = d.alast ? d.alast[c] : 0.f;
  atomicAdd(&bs.cnt[key], 1u);
  atomicMax(&bs.vmax[key], __float_as_int(sp));  // non-negative floats order as ints
  atomicAdd(&bs.vsum[key], sp);
  atomicMax(&bs.amax[key], __float_as_int(ac));
}

__global__ void k_bin_compact(const uint32_t* __restrict__ cnt, long long nbins,
                              uint32_t* __restrict__ occ, uint32_t* __restrict__ n_occ) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbins) return;
  if (cnt[k] > 0) occ[atomicAdd(n_occ, 1u)] = (uint32_t)k;
}

__global__ void k_bin_features(BinStats bs, const uint32_t* __restrict__ occ, long long n_occ,
                               int nc, const float* __restrict__ cand, FeatureScales fs,
                               float* __restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_occ * nc) return;
  const long long b = i / nc;
  const int j = (int)(i - b * nc);
  const uint32_t key = occ[b];
  const float n = (float)bs.cnt[key];
  const float vmax = __int_as_float(bs.vmax[key]);
  const float vmean = bs.vsum[key] / n;
  const float amax = __int_as_float(bs.amax[key]);
  const float m = cand[j];
  const float tiny = 1e-30f;
  float* f = x + i * kMlpIn;
  f[0] = logf(1.f + n);
  f[1] = logf(fmaxf(fs.h * vmax / m, tiny));
  f[2] = logf(fmaxf(fs.h * vmean / m, tiny));
  f[3] = logf(fmaxf(fs.h * fs.h * amax / m, tiny));
  f[4] = logf(m / fs.rmean);
  f[5] = logf(fmaxf(fs.h * fs.h * fs.gmag / m, tiny));
}

// Smallest candidate whose predicted ln(lifetime) reaches ln_need.
__global__ void k_choose_margin(const uint32_t* __restrict__ occ, long long n_occ, int nc,
                                const float* __restrict__ cand, const float* __restrict__ y,
                                float ln_need, float* __restrict__ bin_margin) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_occ) return;
  float m = cand[nc - 1];
  for (int j = 0; j < nc; ++j)
    if (y[b * nc + j] >= ln_need) {
      m = cand[j];
      break;
    }
  bin_margin[occ[b]] = m;
}

// The clump's margin: its home bin's, at least floor_scale times its speed
// bound (the distance it covers in the interval at its current speed).
__global__ void k_clump_margin(DevState d, const uint32_t* __restrict__ chome,
                               const float* __restrict__ bin_margin, float floor_scale,
                               float* __restrict__ cmargin) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  float m = bin_margin[chome[c]];
  if (floor_scale > 0.f) m = fmaxf(m, floor_scale * clump_speed_bound(d, c, d.cinfo[c].x));
  cmargin[c] = m;
}

// Displacement bound of every clump since the trace reference, maxed per home bin.
__global__ void k_trace_disp(DevState d, TraceRef tr, const uint32_t* __restrict__ chome,
                             int* __restrict__ dmax) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const int tpl = d.cinfo[c].x;
  float dx, dy, dz;
  float4 q;
  if (d.prec == 1) {
    const int4 v = d.cvox[c], v0 = tr.vox[c];
    const float4 o = d.coff[c], o0 = tr.off[c];
    const float kV = (float)kVoxel;
    dx = (float)(v.x - v0.x) * kV + (o.x - o0.x);
    dy = (float)(v.y - v0.y) * kV + (o.y - o0.y);
    dz = (float)(v.z - v0.z) * kV + (o.z - o0.z);
  } else {
    const double4_32a p = d.cpos[c], p0 = tr.pos[c];
    dx = (float)(p.x - p0.x); dy = (float)(p.y - p0.y); dz = (float)(p.z - p0.z);
  }
  const double4_32a qd = d.cq[c];
  q = make_float4(d2f(qd.x), d2f(qd.y), d2f(qd.z), d2f(qd.w));
  const float4 r0 = tr.q[c];
  // vec(conj(q0) q)
  const float e1 = r0.x * q.y - r0.y * q.x - r0.z * q.w + r0.w * q.z;
  const float e2 = r0.x * q.z + r0.y * q.w - r0.z * q.x - r0.w * q.y;
  const float e3 = r0.x * q.w - r0.y * q.z + r0.z * q.y - r0.w * q.x;
  const float disp = sqrtf(dx * dx + dy * dy + dz * dz) +
                     2.f * d.tpbound[tpl] * sqrtf(e1 * e1 + e2 * e2 + e3 * e3);
  atomicMax(&dmax[chome[c]], __float_as_int(disp));
}

__global__ void k_trace_bins(const uint32_t* __restrict__ occ, long long n_occ, int nc,
                             const float* __restrict__ cand, int* __restrict__ dmax,
                             int* __restrict__ T, int step) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_occ) return;
  const uint32_t key = occ[b];
  const float dm = __int_as_float(dmax[key]);
  for (int j = 0; j < nc; ++j)
    if (T[b * nc + j] == 0 && dm > cand[j]) T[b * nc + j] = step;
  dmax[key] = 0;
}

// Row i of this window (occupied bin i / nc, candidate i % nc) goes to row
// base + i of the output, so the candidates of one bin stay adjacent and in
// order.
__global__ void k_trace_emit(long long n_rows, const float* __restrict__ xw,
                             const int* __restrict__ T, int window, float* __restrict__ x,
                             float* __restrict__ t, long long base, long long cap) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  const long long k = base + i;
  if (k >= cap) return;
  for (int f = 0; f < kMlpIn; ++f) x[k * kMlpIn + f] = xw[i * kMlpIn + f];
  const int tt = T[i] > 0 ? T[i] : window;
  t[k] = logf((float)tt);
}

__global__ void k_trace_ref(DevState d, TraceRef tr) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.ncl) return;
  const double4_32a q = d.cq[c];
  tr.q[c] = make_float4(d2f(q.x), d2f(q.y), d2f(q.z), d2f(q.w));
  if (d.prec == 1) {
    tr.vox[c] = d.cvox[c];
    tr.off[c] = d.coff[c];
  } else {
    tr.pos[c] = d.cpos[c];
  }
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_clump_home(const DevState& d, const BinStats& bs, cudaStream_t st) {
  if (d.ncl == 0) return;
  k_clump_home<<<nblk(d.ncl, 256), 256, 0, st>>>(d, bs);
  count_launch();
}
void launch_bin_compact(const uint32_t* cnt, long long nbins, uint32_t* occ, uint32_t* n_occ,
                        cudaStream_t st) {
  if (nbins == 0) return;
  k_bin_compact<<<nblk(nbins, 256), 256, 0, st>>>(cnt, nbins, occ, n_occ);
  count_launch();
}
void launch_bin_features(const BinStats& bs, const uint32_t* occ, long long n_occ, int nc,
                         const float* cand, const FeatureScales& fs, float* x, cudaStream_t st) {
  if (n_occ == 0) return;
  k_bin_features<<<nblk(n_occ * nc, 256), 256, 0, st>>>(bs, occ, n_occ, nc, cand, fs, x);
  count_launch();
}
void launch_choose_margin(const uint32_t* occ, long long n_occ, int nc, const float* cand,
                          const float* y, float ln_need, float* bin_margin, cudaStream_t st) {
  if (n_occ == 0) return;
  k_choose_margin<<<nblk(n_occ, 256), 256, 0, st>>>(occ, n_occ, nc, cand, y, ln_need, bin_margin);
  count_launch();
}
void launch_clump_margin(const DevState& d, const uint32_t* chome, const float* bin_margin,
                         float floor_scale, float* cmargin, cudaStream_t st) {
  if (d.ncl == 0) return;
  k_clump_margin<<<nblk(d.ncl, 256), 256, 0, st>>>(d, chome, bin_margin, floor_scale, cmargin);
  count_launch();
}
void launch_trace_ref(const DevState& d, const TraceRef& tr, cudaStream_t st) {
  if (d.ncl == 0) return;
  k_trace_ref<<<nblk(d.ncl, 256), 256, 0, st>>>(d, tr);
  count_launch();
}
void launch_trace_step(const DevState& d, const TraceRef& tr, const uint32_t* chome, int* dmax,
                       const uint32_t* occ, long long n_occ, int nc, const float* cand, int* T,
                       int step, cudaStream_t st) {
  if (d.ncl == 0) return;
  k_trace_disp<<<nblk(d.ncl, 256), 256, 0, st>>>(d, tr, chome, dmax);
  k_trace_bins<<<nblk(n_occ, 256), 256, 0, st>>>(occ, n_occ, nc, cand, dmax, T, step);
  count_launch(2);
}
void launch_trace_emit(long long n_rows, const float* xw, const int* T, int window, float* x,
                       float* t, long long base, long long cap, cudaStream_t st) {
  if (n_rows == 0 || base >= cap) return;
  k_trace_emit<<<nblk(n_rows, 256), 256, 0, st>>>(n_rows, xw, T, window, x, t, base, cap);
  count_launch();
}

}  // namespace dem
