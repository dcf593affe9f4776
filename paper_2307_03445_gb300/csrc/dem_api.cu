// dem_api.cu -- host runtime and the C ABI declared in include/dem.h.
//
// One context owns every device buffer of one simulation (one or more
// scenes) on one device and one stream.  A step is a fixed sequence of
// launches on that stream: [rebuild] -> sphere-sphere forces -> sphere-wall
// forces -> clump update (integration + sphere poses + certificate).  The
// rebuild synchronises twice (to size the bin registrations and the pair
// list); steps without a rebuild never synchronise.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dem.h"
#include "dem_dev.cuh"
#include "dem_prims.cuh"
#include "dem_learn.cuh"
#include "dem_mlp.cuh"

using namespace dem;

namespace {

thread_local std::string g_create_error;

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct SceneH {
  double lo[3], hi[3], bin;
};

// Scratch of one detection (the main one on the context stream; a second
// set for the outer list detected on the second stream, see
// dem_set_outer_list).
struct DetScratch {
  Buf det, wall_mask, wall_cnt, pair_cnt, bin_size, bin_start, scan_scr, trho, totals;
  Buf rec, upairs, fbin_size, fbin_start, fcnt, frec, fcand;
  Buf fkeep, wkeep;  // the filter's decisions (lists filtered from the outer list)
  unsigned long long ucap = 0;  // capacity of the unordered pair buffer
  unsigned long long fcap = 0;  // capacity of the facet candidate buffer
};

// A detection in two parts.  detect_prepare reads the clump state (the
// lattice points, the bin counts, the analytic wall candidates) on stream
// st; detect_finish does the rest (scans, bin scatter, facets, narrow phase,
// the list's rows) on stream st2, which may be another stream once it waits
// for the first part, since nothing there reads the state again except the
// facet passes (a detection with facets finishes on the same stream at once).
struct DetJob {
  DetectOut o{};
  int li = 0, si = 0, K = 1;
  double m = 0.0, t = 0.0, travel = 0.0;
};


}  // namespace

struct dem_ctx {
  dem_params P{};
  std::vector<double> E, nu, mu, cor;
  std::vector<dem_wall> user_walls;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  // templates
  int n_tpl = 0;
  std::vector<int> tpl_off, tpl_mat;
  std::vector<double> tpl_pos, tpl_rad, tpl_mass, tpl_inert;
  double r_max = 0.0;
  double r_mean = 1e-3, r_sum = 0.0;
  // scenes and walls
  std::vector<SceneH> scenes;
  std::vector<WallDev> walls;
  std::vector<int> wall_user, wall_scene;
  std::vector<SceneGrid> grids;
  uint32_t nbins = 0;
  std::vector<SceneGrid> lgrids;  // the learned rule's feature grids (base bin edge)
  uint32_t n_lbins = 0;
  // clumps (host bookkeeping)
  std::vector<int> h_ctpl, h_cscene;
  long long ncl = 0, ns = 0;
  // all device buffers
  std::vector<Buf*> owned;
  Buf b_tpl_off, b_tp64, b_tp32, b_trm, b_tmat, b_tmass, b_tinert, b_tpbound, b_tmassf, b_tinertf;
  Buf b_cinfo, b_csph, b_cpos, b_cvox, b_coff, b_cq, b_cvw, b_mv64, b_mw64, b_mv32, b_mw32;
  Buf b_acc64, b_acc32, b_ref_pos, b_ref_vox, b_ref_off, b_ref_q;
  Buf b_sinfo, b_sa64, b_sb64, b_srec32;
  Buf b_grids, b_lgrids, b_walls, b_wall_idx, b_wall_scene, b_wfix, b_wpos, b_wforce, b_wtorque, b_pm64, b_pm32;
  Buf b_flags, b_counters, b_totals, b_dstep;
  // detection scratch
  DetScratch ds[2];  // 0: detections on the context stream; 1: the outer list on st2
  Buf b_tmp, b_facet_idx;
  int n_facets = 0;
  // two-level list: an outer list at outer_factor x the margin serves
  // outer_n rebuilds; b_q0 holds its lattice points and enlarged radii
  double outer_factor = 0.0;
  int outer_n = 0, outer_used = 0;
  bool outer_valid = false;
  long long outer_ns = 0;
  double outer_m = 0.0;
  int outer_K = 0;
  long long outer_until = 0;  // its wall candidates cover the steps before this one
  Buf b_q0;
  // the next outer list detected on a second stream while the steps run
  // (async_state 0: none; 1: its state-reading part is queued on st, the
  // rest still to be queued on st2; 2: queued in full, ev_ready marks its end)
  bool outer_async = false;
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_snap = nullptr, ev_ready = nullptr;
  int async_state = 0;
  DetJob async_job;
  double async_m = 0.0;
  int async_K = 0;
  long long async_ns = 0, async_until = 0;
  Buf b_q1;
  double bin_factor = 1.0;      // bin edge multiplier chosen by dem_autotune_bins
  dem_tiles tiles = {8, 128, 8}; // launch shapes (dem_set_tiles / dem_autotune_tiles)
  long long n_entries = 0;       // bin registrations of the last rebuild (records in
                                 // b_rec, bins delimited by b_bin_start)
  long long n_entry_bins = 0;    // bins of that rebuild
  // contact lists (current, next) and an audit list
  struct ListBufs {
    Buf pa, pb, pown, ppm, u, row, ws, ww, uw, wrow, dnb;
    ContactList L{};
  } lists[5];  // 0, 1: current and next; 2: audit; 3: outer list; 4: the next outer list
  int cur = 0;
  long long list_ns = 0;  // spheres when the current list was built
  // state
  bool finalized = false, need_rebuild = true, have_list = false, acc_dirty = true;
  long long step = 0;
  int since = 0;
  double margin = 0.0;
  int timing = 0;
  dem_stats stats{};
  DevState D{};
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // learned rule, halt mode: the halt step read back after every chunk of
  // steps (pinned host slots, one per chunk in flight, and their events)
  long long* h_halt = nullptr;
  cudaEvent_t ev_halt[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> evpool;  // 4 per timed step, read at the end of dem_step
  // learned rebuild rule (extension) and rollback snapshots
  dem_mlp* mlp = nullptr;
  int l_interval = 0;
  double l_safety = 1.0;
  int l_mode = 0;
  double l_floor = 0.0;  // speed floor factor of the learned margins (0: off)
  // deterministic reduction: slot buffers and per-clump slot lists of the current list
  int det = 0;
  bool det_ready = false;
  Buf b_det_cnt, b_det_fill, b_det_off, b_det_ids, b_det_pair, b_det_wall;
  std::vector<double> l_cand;
  long long n_occ = 0;
  Buf b_alast, b_chome, b_cmargin, b_bcnt, b_bvmax, b_bvsum, b_bamax, b_occ, b_nocc, b_binm, b_cand;
  Buf b_feat, b_pred, b_dmax, b_T, b_tr_vox, b_tr_off, b_tr_pos, b_tr_q, b_tx, b_tt;
  Buf s_state, s_pb, s_u, s_ww, s_uw;
  long long snap_step = 0;
  // CUDA graphs of the steps between rebuilds (plain rule)
  int use_graphs = 0;
  long long layout = 0;        // bumped whenever a device buffer is reallocated
  long long graph_layout = -1;
  struct GraphEntry {
    int cur, m, cert;
    double margin;
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<GraphEntry> graphs;
};

namespace {

int fail(dem_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Device memory, stream-ordered on `st` (the context stream unless given).
void* dalloc(dem_ctx* c, size_t bytes, cudaStream_t st = nullptr) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->P.alloc) {
    p = c->P.alloc(bytes, c->P.alloc_user);
    if (p && ((uintptr_t)p & 255u)) {  // the kernels' 16- and 32-byte records need it
      if (c->P.free) c->P.free(p, c->P.alloc_user);
      p = nullptr;
    }
  } else if (cudaMallocAsync(&p, bytes, st ? st : c->st) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}
void dfree(dem_ctx* c, void* p, cudaStream_t st = nullptr) {
  if (!p) return;
  if (c->P.free) c->P.free(p, c->P.alloc_user);
  else cudaFreeAsync(p, st ? st : c->st);
}

// Grows b to at least `bytes`, preserving the first `keep` bytes; the new
// block is allocated and the old one freed in the order of stream `st`.
bool grow(dem_ctx* c, Buf& b, size_t bytes, size_t keep = 0, cudaStream_t st = nullptr) {
  if (b.bytes >= bytes && b.p) return true;
  if (!st) st = c->st;
  size_t nb = std::max(bytes, b.bytes + b.bytes / 4);
  nb = (nb + 255) & ~(size_t)255;
  void* p = dalloc(c, nb, st);
  if (!p) return false;
  c->layout++;
  if (keep && b.p) cudaMemcpyAsync(p, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, st);
  dfree(c, b.p, st);
  b.p = p;
  b.bytes = nb;
  return true;
}

template <typename T>
T* ptr(const Buf& b) {
  return reinterpret_cast<T*>(b.p);
}

int cuda_check(dem_ctx* c, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, DEM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return DEM_OK;
}

void split_ff(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}

// Rotation by a unit quaternion (host, double).
void qrot(const double* q, const double* p, double* o, bool transpose) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  double r[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                 2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                 2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 3; ++i) {
    o[i] = 0;
    for (int k = 0; k < 3; ++k) o[i] += (transpose ? r[3 * k + i] : r[3 * i + k]) * p[k];
  }
}

// Deterministic-reduction pointers of the device view (NULL unless the mode
// is on and the slot lists of the current list exist).
void set_det_pointers(dem_ctx* c) {
  DevState& d = c->D;
  const bool det = c->det && c->det_ready;
  d.det_off = det ? ptr<uint32_t>(c->b_det_off) : nullptr;
  d.det_ids = det ? ptr<uint32_t>(c->b_det_ids) : nullptr;
  d.det_pair32 = det ? ptr<float4>(c->b_det_pair) : nullptr;
  d.det_wall32 = det ? ptr<float4>(c->b_det_wall) : nullptr;
  d.det_pair64 = det ? ptr<double4_32a>(c->b_det_pair) : nullptr;
  d.det_wall64 = det ? ptr<double4_32a>(c->b_det_wall) : nullptr;
}

void refresh_devstate(dem_ctx* c) {
  DevState& d = c->D;
  d.pairs_bpsm = c->tiles.pairs_blocks_per_sm;
  d.upd_block = c->tiles.update_block;
  d.prec = c->P.precision;
  d.ncl = c->ncl;
  d.ns = c->ns;
  d.nmat = c->P.n_materials;
  d.nwalls = (int)c->walls.size();
  d.h = c->P.dt;
  for (int k = 0; k < 3; ++k) {
    d.g[k] = c->P.g[k];
    d.hg[k] = c->P.dt * c->P.g[k];
    d.hgf[k] = (float)d.hg[k];
  }
  d.tpl_off = ptr<int>(c->b_tpl_off);
  d.tp64 = ptr<double4_32a>(c->b_tp64);
  d.tp32 = ptr<float4>(c->b_tp32);
  d.tmat = ptr<int>(c->b_tmat);
  d.trm = ptr<float2>(c->b_trm);
  d.tmass = ptr<double>(c->b_tmass);
  d.tinert = ptr<double>(c->b_tinert);
  d.tmassf = ptr<float>(c->b_tmassf);
  d.tinertf = ptr<float>(c->b_tinertf);
  d.hf = (float)c->P.dt;
  d.tpbound = ptr<float>(c->b_tpbound);
  d.cinfo = ptr<int2>(c->b_cinfo);
  d.csph = ptr<int>(c->b_csph);
  d.cpos = ptr<double4_32a>(c->b_cpos);
  d.cvox = ptr<int4>(c->b_cvox);
  d.coff = ptr<float4>(c->b_coff);
  d.cq = ptr<double4_32a>(c->b_cq);
  d.cvw = ptr<VelRec>(c->b_cvw);
  d.mv64 = ptr<double4_32a>(c->b_mv64);
  d.mw64 = ptr<double4_32a>(c->b_mw64);
  d.mv32 = ptr<float4>(c->b_mv32);
  d.mw32 = ptr<float4>(c->b_mw32);
  d.acc64 = ptr<double>(c->b_acc64);
  d.acc32 = ptr<float>(c->b_acc32);
  d.ref_pos = ptr<double4_32a>(c->b_ref_pos);
  d.ref_vox = ptr<int4>(c->b_ref_vox);
  d.ref_off = ptr<float4>(c->b_ref_off);
  d.ref_q = ptr<float4>(c->b_ref_q);
  d.cmargin = nullptr;
  d.alast = ptr<float>(c->b_alast);
  d.sinfo = ptr<int2>(c->b_sinfo);
  d.sa64 = ptr<SphA64>(c->b_sa64);
  d.sb64 = ptr<double4_32a>(c->b_sb64);
  d.srec32 = ptr<uint4>(c->b_srec32);
  d.grids = ptr<SceneGrid>(c->b_grids);
  d.walls = ptr<WallDev>(c->b_walls);
  d.wall_idx = ptr<int>(c->b_wall_idx);
  d.wall_scene = ptr<int>(c->b_wall_scene);
  d.facet_idx = ptr<int>(c->b_facet_idx);
  d.nfacets = c->n_facets;
  d.wfix = ptr<long long>(c->b_wfix);
  d.wpos = ptr<double>(c->b_wpos);
  d.wforce = ptr<double>(c->b_wforce);
  d.wtorque = ptr<double>(c->b_wtorque);
  d.pm64 = ptr<PairMat<double>>(c->b_pm64);
  d.pm32 = ptr<PairMat<float>>(c->b_pm32);
  d.flags = ptr<int>(c->b_flags);
  d.counters = ptr<unsigned long long>(c->b_counters);
  d.dstep = ptr<long long>(c->b_dstep);
  d.halt_at = nullptr;  // set by the learned rule's halting intervals only
  set_det_pointers(c);
}

ContactList& curL(dem_ctx* c);

// Slot buffers and per-clump slot lists of the current list (deterministic
// reduction); a no-op when the mode is off.
int build_det_lists(dem_ctx* c) {
  c->det_ready = false;
  if (!c->det) {
    set_det_pointers(c);
    return DEM_OK;
  }
  ContactList& L = curL(c);
  const long long ncl = c->ncl, n = L.n, nw = L.nw;
  if (2 * n + nw >= (1ll << 32) - 1) return fail(c, DEM_ERR_CAPACITY, "deterministic mode: list too long");
  const size_t slot = c->P.precision == DEM_FP64 ? 32 : 16;
  if (!grow(c, c->b_det_cnt, 4 * (size_t)(ncl + 1)) || !grow(c, c->b_det_fill, 4 * (size_t)(ncl + 1)) ||
      !grow(c, c->b_det_off, 4 * (size_t)(ncl + 1)) || !grow(c, c->b_det_ids, 4 * (size_t)(2 * n + nw + 1)) ||
      !grow(c, c->b_det_pair, 3 * slot * (size_t)(L.cap + 1)) ||
      !grow(c, c->b_det_wall, 2 * slot * (size_t)(L.capw + 1)))
    return fail(c, DEM_ERR_OOM, "deterministic-mode buffers");
  cudaMemsetAsync(c->b_det_cnt.p, 0, 4 * (size_t)(ncl + 1), c->st);
  cudaMemsetAsync(c->b_det_fill.p, 0, 4 * (size_t)(ncl + 1), c->st);
  launch_det_lists(c->D, L, n, nw, ptr<uint32_t>(c->b_det_cnt), ptr<uint32_t>(c->b_det_fill),
                   ptr<uint32_t>(c->b_det_off), ptr<uint32_t>(c->b_det_ids), c->ds[0].scan_scr.p,
                   ptr<unsigned long long>(c->ds[0].totals) + 6, c->st);
  c->det_ready = true;
  set_det_pointers(c);
  return cuda_check(c, "deterministic lists");
}

ContactList& curL(dem_ctx* c) { return c->lists[c->cur].L; }

// Pair material table (section 2.1: stiffness and damping of a contact from
// the E, nu, mu, CoR of its two spheres).
int build_pair_materials(dem_ctx* c) {
  const int M = c->P.n_materials;
  std::vector<PairMat<double>> pm64((size_t)M * M);
  std::vector<PairMat<float>> pm32((size_t)M * M);
  const double kPi = 3.14159265358979323846;
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      const double Ea = c->E[a], Eb = c->E[b], na = c->nu[a], nb = c->nu[b];
      const double Es = 1.0 / ((1.0 - na * na) / Ea + (1.0 - nb * nb) / Eb);
      const double Gs = 1.0 / (2.0 * (2.0 - na) * (1.0 + na) / Ea + 2.0 * (2.0 - nb) * (1.0 + nb) / Eb);
      double mu, e;
      const double ma = c->mu[a], mb = c->mu[b], ca = c->cor[a], cb = c->cor[b];
      switch (c->P.mix_rule) {
        case DEM_MIX_MIN: mu = std::min(ma, mb); e = std::min(ca, cb); break;
        case DEM_MIX_MAX: mu = std::max(ma, mb); e = std::max(ca, cb); break;
        default: mu = 0.5 * (ma + mb); e = 0.5 * (ca + cb); break;
      }
      double beta;
      if (e >= 1.0) beta = 0.0;
      else if (e <= 0.0) beta = -1.0;
      else beta = std::log(e) / std::sqrt(std::log(e) * std::log(e) + kPi * kPi);
      PairMat<double> p{};
      p.kn = 4.0 / 3.0 * Es;
      p.kt = 8.0 * Gs;
      p.mu = mu;
      p.cn = -2.0 * std::sqrt(5.0 / 6.0) * beta * std::sqrt(2.0 * Es);
      p.ct = -2.0 * std::sqrt(5.0 / 6.0) * beta * std::sqrt(8.0 * Gs);
      pm64[(size_t)a * M + b] = p;
      PairMat<float> q{};
      q.kn = (float)p.kn; q.kt = (float)p.kt; q.mu = (float)p.mu; q.cn = (float)p.cn; q.ct = (float)p.ct;
      pm32[(size_t)a * M + b] = q;
    }
  if (!grow(c, c->b_pm64, sizeof(PairMat<double>) * pm64.size()) ||
      !grow(c, c->b_pm32, sizeof(PairMat<float>) * pm32.size()))
    return fail(c, DEM_ERR_OOM, "pair material table");
  cudaMemcpyAsync(c->b_pm64.p, pm64.data(), sizeof(PairMat<double>) * pm64.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_pm32.p, pm32.data(), sizeof(PairMat<float>) * pm32.size(), cudaMemcpyHostToDevice, c->st);
  cudaStreamSynchronize(c->st);
  return DEM_OK;
}

double current_margin(const dem_ctx* c) {
  if (c->P.margin > 0.0) return c->P.margin;
  return c->P.v_bound * c->P.dt * (double)std::max(1, c->P.rebuild_interval);
}

// Detection grids of all scenes (bin edge = the scene's base edge times
// bin_factor); the wall ranges of existing grids are kept.
// Per-scene grids with bin edge `factor` times the scene's base edge (its
// bin_size, else twice the largest enlarged radius).
int make_grids(dem_ctx* c, double factor, std::vector<SceneGrid>& grids, uint32_t& nbins) {
  grids.clear();
  uint64_t base = 0;
  for (size_t s = 0; s < c->scenes.size(); ++s) {
    const SceneH& sh = c->scenes[s];
    SceneGrid g{};
    const double bin = (sh.bin > 0.0 ? sh.bin : 2.0 * (c->r_max + c->margin)) * factor;
    long long L = (long long)std::ceil(bin * kDetScale);
    if (L < 1) L = 1;
    for (int k = 0; k < 3; ++k) {
      g.lo[k] = sh.lo[k];
      g.lof[k] = (float)sh.lo[k];
      long long ext = std::llrint((sh.hi[k] - sh.lo[k]) * kDetScale);
      long long dd = (ext + L - 1) / L;
      if (dd < 1) dd = 1;
      // bin coordinates are packed in 21 bits per axis
      if (dd >= (1ll << 21)) return fail(c, DEM_ERR_INVALID_ARG, "detection grid too fine (2^21 bins per axis)");
      g.dims[k] = (int)dd;
    }
    g.L = L;
    g.invL = (float)(1.0 / (double)L);
    g.key_base = (uint32_t)base;
    base += (uint64_t)g.dims[0] * g.dims[1] * g.dims[2];
    if (base >= (1ull << 32) - 1) return fail(c, DEM_ERR_INVALID_ARG, "too many bins (> 2^32)");
    grids.push_back(g);
  }
  nbins = (uint32_t)base;
  return DEM_OK;
}

// The detection grids (bin edge scaled by the tuned bin factor) and the
// learned rule's feature grids (the base edge itself, so that the features
// and the trained model do not depend on the detection tuning).
int build_grids(dem_ctx* c) {
  std::vector<SceneGrid> grids, lgrids;
  uint32_t nb = 0, nlb = 0;
  int rc = make_grids(c, c->bin_factor, grids, nb);
  if (rc == DEM_OK) rc = make_grids(c, 1.0, lgrids, nlb);
  if (rc) return rc;
  for (size_t s = 0; s < grids.size() && s < c->grids.size(); ++s) {
    grids[s].wall_start = c->grids[s].wall_start;
    grids[s].wall_count = c->grids[s].wall_count;
  }
  c->grids = grids;
  c->nbins = nb;
  c->lgrids = lgrids;
  c->n_lbins = nlb;
  return DEM_OK;
}

// Grids, walls and zeroed accumulators; called before the first step.
int finalize(dem_ctx* c) {
  if (c->finalized) return DEM_OK;
  if (c->n_tpl == 0) return fail(c, DEM_ERR_STATE, "no clump templates loaded");
  c->margin = current_margin(c);
  // the detection lattice holds r + m in 31 bits (2^-24 m units)
  if (!(c->r_max + c->margin < 32.0)) return fail(c, DEM_ERR_INVALID_ARG, "sphere radius plus margin must be below 32 m");
  c->grids.clear();
  int rc = build_grids(c);
  if (rc) return rc;
  // internal walls: one copy per scene they apply to
  c->walls.clear();
  c->wall_user.clear();
  c->wall_scene.clear();
  std::vector<int> idx, fidx;  // analytic walls per scene; mesh facets (found through the bins)
  for (size_t s = 0; s < c->scenes.size(); ++s) {
    c->grids[s].wall_start = (int)idx.size();
    int cnt = 0;
    for (size_t w = 0; w < c->user_walls.size(); ++w) {
      const dem_wall& uw = c->user_walls[w];
      if (uw.scene != -1 && uw.scene != (int)s) continue;
      WallDev d{};
      d.type = uw.type;
      d.material = uw.material;
      for (int k = 0; k < 3; ++k) {
        d.p[k] = uw.p[k];
        d.n[k] = uw.n[k];
        d.vel[k] = uw.vel[k];
        split_ff(uw.n[k], d.nh[k], d.nl[k]);
      }
      d.radius = uw.radius;
      d.half_angle = uw.half_angle;
      d.height = uw.height;
      d.rb = uw.height * std::tan(uw.half_angle);
      split_ff(uw.radius, d.rh, d.rl);
      split_ff(std::cos(uw.half_angle), d.ch, d.cl);
      split_ff(std::sin(uw.half_angle), d.sh, d.sl);
      split_ff(uw.height, d.hh, d.hl);
      split_ff(d.rb, d.rbh, d.rbl);
      d.speed_d = std::sqrt((uw.vel[0] * uw.vel[0] + uw.vel[1] * uw.vel[1]) + uw.vel[2] * uw.vel[2]);
      d.speed = (float)d.speed_d;
      for (int k = 0; k < 3; ++k) {
        d.pf[k] = (float)uw.p[k];
        d.vf[k] = (float)uw.vel[k];
      }
      d.radf = (float)uw.radius;
      d.heightf = (float)uw.height;
      d.rbf = (float)d.rb;
      if (uw.type == DEM_WALL_TRIANGLE) {
        for (int k = 0; k < 3; ++k) {
          d.e1[k] = uw.b[k] - uw.p[k];
          d.e2[k] = uw.c[k] - uw.p[k];
          split_ff(d.e1[k], d.e1h[k], d.e1l[k]);
          split_ff(d.e2[k], d.e2h[k], d.e2l[k]);
        }
      }
      if (uw.type == DEM_WALL_TRIANGLE) {
        fidx.push_back((int)c->walls.size());
      } else {
        idx.push_back((int)c->walls.size());
        ++cnt;
      }
      c->wall_user.push_back((int)w);
      c->wall_scene.push_back((int)s);
      c->walls.push_back(d);
    }
    // analytic walls are tested by every sphere of the scene (a bit mask per
    // sphere); facets are registered in the bins and have no such limit
    if (cnt > 32) return fail(c, DEM_ERR_INVALID_ARG, "more than 32 analytic walls in one scene");
    c->grids[s].wall_count = cnt;
  }
  c->n_facets = (int)fidx.size();
  const size_t nw = std::max<size_t>(1, c->walls.size());
  if (!grow(c, c->b_grids, sizeof(SceneGrid) * c->grids.size()) ||
      !grow(c, c->b_lgrids, sizeof(SceneGrid) * c->lgrids.size()) ||
      !grow(c, c->b_walls, sizeof(WallDev) * nw) || !grow(c, c->b_wall_idx, sizeof(int) * std::max<size_t>(1, idx.size())) ||
      !grow(c, c->b_wall_scene, sizeof(int) * nw) || !grow(c, c->b_wfix, 3 * sizeof(long long) * nw) ||
      !grow(c, c->b_wpos, 3 * sizeof(double) * nw) || !grow(c, c->b_wforce, 3 * sizeof(double) * nw) ||
      !grow(c, c->b_wtorque, 3 * sizeof(double) * nw) ||
      !grow(c, c->b_facet_idx, sizeof(int) * std::max<size_t>(1, fidx.size())) ||
      !grow(c, c->b_flags, 64) || !grow(c, c->b_counters, 64) || !grow(c, c->ds[0].totals, 128) ||
      !grow(c, c->b_dstep, 64))
    return fail(c, DEM_ERR_OOM, "scene tables");
  cudaMemcpyAsync(c->b_grids.p, c->grids.data(), sizeof(SceneGrid) * c->grids.size(), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_lgrids.p, c->lgrids.data(), sizeof(SceneGrid) * c->lgrids.size(),
                  cudaMemcpyHostToDevice, c->st);
  if (!c->walls.empty()) {
    cudaMemcpyAsync(c->b_walls.p, c->walls.data(), sizeof(WallDev) * c->walls.size(), cudaMemcpyHostToDevice, c->st);
    if (!idx.empty())
      cudaMemcpyAsync(c->b_wall_idx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, c->st);
    if (!fidx.empty())
      cudaMemcpyAsync(c->b_facet_idx.p, fidx.data(), sizeof(int) * fidx.size(), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->b_wall_scene.p, c->wall_scene.data(), sizeof(int) * c->wall_scene.size(), cudaMemcpyHostToDevice, c->st);
  }
  cudaMemsetAsync(c->b_wforce.p, 0, c->b_wforce.bytes, c->st);
  cudaMemsetAsync(c->b_wtorque.p, 0, c->b_wtorque.bytes, c->st);
  cudaMemsetAsync(c->b_flags.p, 0, 64, c->st);
  cudaMemsetAsync(c->b_counters.p, 0, 64, c->st);
  c->stats.margin = c->margin;
  c->finalized = true;
  refresh_devstate(c);
  // sphere poses and mirrors of the initial state, walls at the current time
  launch_update(c->D, false, c->step, c->margin, false, c->st);
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "finalize");
}

// Lists[li] sized for NP pairs and NW wall contacts (25 % headroom when it
// grows) and its device view set; hist = false leaves out the tangential
// history arrays (the outer list carries none).
int size_list(dem_ctx* c, int li, unsigned long long NP, unsigned long long NW, bool hist,
              cudaStream_t st = nullptr) {
  auto& LB = c->lists[li];
  ContactList& L = LB.L;
  if ((long long)NP > L.cap || !LB.pa.p) {
    const long long cap = std::max<long long>((long long)(NP + NP / 4), 1024);
    dfree(c, LB.pa.p, st); dfree(c, LB.pb.p, st); dfree(c, LB.u.p, st); dfree(c, LB.pown.p, st);
    dfree(c, LB.ppm.p, st);
    LB.pa = Buf(); LB.pb = Buf(); LB.u = Buf(); LB.pown = Buf(); LB.ppm = Buf();
    const bool own = hist && c->P.precision != DEM_FP64;
    if (!grow(c, LB.pa, 4 * cap, 0, st) || !grow(c, LB.pb, 4 * cap, 0, st) ||
        (hist && !grow(c, LB.u, 24 * cap, 0, st)) ||
        (own && (!grow(c, LB.pown, 16 * cap, 0, st) || !grow(c, LB.ppm, 4 * cap, 0, st))))
      return fail(c, DEM_ERR_OOM, "pair list");
    L.cap = cap;
  }
  if ((long long)NW > L.capw || !LB.ws.p) {
    const long long cap = std::max<long long>((long long)(NW + NW / 4), 1024);
    dfree(c, LB.ws.p, st); dfree(c, LB.ww.p, st); dfree(c, LB.uw.p, st);
    LB.ws = Buf(); LB.ww = Buf(); LB.uw = Buf();
    if (!grow(c, LB.ws, 4 * cap, 0, st) || !grow(c, LB.ww, 4 * cap, 0, st) || (hist && !grow(c, LB.uw, 24 * cap, 0, st)))
      return fail(c, DEM_ERR_OOM, "wall list");
    L.capw = cap;
  }
  L.pa = ptr<int>(LB.pa);
  L.pb = ptr<uint32_t>(LB.pb);
  L.pown = ptr<int4>(LB.pown);
  L.ppm = ptr<int>(LB.ppm);
  L.u = ptr<double>(LB.u);
  L.row = ptr<uint32_t>(LB.row);
  L.ws = ptr<int>(LB.ws);
  L.ww = ptr<uint32_t>(LB.ww);
  L.uw = ptr<double>(LB.uw);
  L.wrow = ptr<uint32_t>(LB.wrow);
  if (!grow(c, LB.dnb, 16, 0, st)) return fail(c, DEM_ERR_OOM, "list lengths");
  L.dn = ptr<long long>(LB.dnb);
  L.n = (long long)NP;
  L.nw = (long long)NW;
  return DEM_OK;
}

int detect_prepare(dem_ctx* c, int li, double m, int K, double wall_extra, int si, cudaStream_t st,
                   DetJob& J) {
  DetScratch& S = c->ds[si];
  const long long ns = c->ns;
  const double t = (double)c->step * c->P.dt;
  const double travel = c->P.dt * (double)std::max(1, K);
  auto& LB = c->lists[li];
  const size_t nb = (size_t)c->nbins;
  if (!grow(c, S.det, sizeof(int4) * (ns + 1), 0, st) || !grow(c, S.wall_mask, 4 * (ns + 1), 0, st) ||
      !grow(c, S.wall_cnt, 4 * (ns + 1), 0, st) || !grow(c, S.pair_cnt, 4 * (ns + 1), 0, st) ||
      !grow(c, S.bin_size, 4 * (nb + 1), 0, st) || !grow(c, S.bin_start, 4 * (nb + 1), 0, st) ||
      !grow(c, LB.row, 4 * (ns + 1), 0, st) || !grow(c, LB.wrow, 4 * (ns + 1), 0, st) ||
      !grow(c, S.scan_scr, scan_scratch_bytes(std::max<size_t>(ns, nb) + 1) + 256, 0, st) ||
      !grow(c, S.totals, 128, 0, st))
    return fail(c, DEM_ERR_OOM, "detection buffers");
  DetectOut& o = J.o;
  o = DetectOut{};
  J.li = li;
  J.si = si;
  J.K = K;
  J.m = m;
  J.t = t;
  J.travel = travel;
  o.det = ptr<int4>(S.det);
  o.wall_mask = ptr<uint32_t>(S.wall_mask);
  o.wall_cnt = ptr<uint32_t>(S.wall_cnt);
  o.wall_off = ptr<uint32_t>(LB.wrow);
  o.pair_cnt = ptr<uint32_t>(S.pair_cnt);
  o.pair_off = ptr<uint32_t>(LB.row);
  o.bin_size = ptr<uint32_t>(S.bin_size);
  o.bin_start = ptr<uint32_t>(S.bin_start);
  o.nbins = c->nbins;
  o.wall_extra = wall_extra;
  if (!c->D.cmargin) {  // one margin for all clumps: radii from a per template sphere table
    o.n_tsph = (int)c->tpl_rad.size();
    if (!grow(c, S.trho, 4 * (size_t)(o.n_tsph + 1), 0, st)) return fail(c, DEM_ERR_OOM, "detection buffers");
    o.trho = ptr<int>(S.trho);
  }
  unsigned long long* tot = ptr<unsigned long long>(S.totals);
  // b_totals: 0 entries, 1 analytic wall contacts, 3 pairs, 4 audit, 5 d_np,
  // 6 slot lists, 7 next bin, 8 facet registrations, 9 facet candidates,
  // 10 wall contacts with the facets
  const bool facets = c->n_facets > 0;
  if (facets && (!grow(c, S.fbin_size, 4 * (nb + 1), 0, st) || !grow(c, S.fbin_start, 4 * (nb + 1), 0, st) ||
                 !grow(c, S.fcnt, 4 * (ns + 1), 0, st)))
    return fail(c, DEM_ERR_OOM, "facet bin buffers");
  o.fbin_size = ptr<uint32_t>(S.fbin_size);
  o.fbin_start = ptr<uint32_t>(S.fbin_start);
  o.fcnt = ptr<uint32_t>(S.fcnt);
  o.d_nf = tot + 9;
  // bin sort by counting: sizes (detection pass), starts (scan; the extra
  // zero entry makes start[nbins] the total), then the scatter below; the
  // mesh facets' registrations the same way
  cudaMemsetAsync(o.bin_size, 0, 4 * (nb + 1), st);
  launch_detect(c->D, o, m, nullptr, t, travel, st);
  return cuda_check(c, "detect_prepare");
}

int detect_finish(dem_ctx* c, DetJob& J, const ContactList* old, long long old_ns, cudaStream_t st) {
  DetScratch& S = c->ds[J.si];
  DetectOut& o = J.o;
  const int li = J.li;
  const double m = J.m, t = J.t, travel = J.travel;
  const long long ns = c->ns;
  auto& LB = c->lists[li];
  const size_t nb = (size_t)c->nbins;
  unsigned long long* tot = ptr<unsigned long long>(S.totals);
  const bool facets = c->n_facets > 0;
  exclusive_scan_u32(o.bin_size, o.bin_start, (long long)nb + 1, S.scan_scr.p, tot + 0, st);
  exclusive_scan_u32(o.wall_cnt, o.wall_off, ns, S.scan_scr.p, tot + 1, st);
  unsigned long long h_tot[12] = {};
  if (facets) {
    cudaMemsetAsync(o.fbin_size, 0, 4 * (nb + 1), st);
    launch_facet_count(c->D, o, t, travel, st);
    exclusive_scan_u32(o.fbin_size, o.fbin_start, (long long)nb + 1, S.scan_scr.p, tot + 8, st);
    cudaMemcpyAsync(h_tot + 8, tot + 8, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  }
  cudaMemcpyAsync(h_tot, tot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "detect");
  const unsigned long long B = h_tot[0], NWA = h_tot[1], NFR = h_tot[8];
  if (B >= (1ull << 32) || NWA >= (1ull << 31) || NFR >= (1ull << 31))
    return fail(c, DEM_ERR_CAPACITY, "bin registrations exceed 2^32");
  if (J.si == 0) {
    c->n_entries = (long long)B;
    c->n_entry_bins = (long long)nb;
  }
  if (!grow(c, S.rec, sizeof(EntryRec) * (B + 1), 0, st)) return fail(c, DEM_ERR_OOM, "bin buffers");
  o.rec = ptr<EntryRec>(S.rec);
  launch_bin_scatter(c->D, o, st);
  if (facets) {
    if (!grow(c, S.frec, sizeof(uint4) * (NFR + 1), 0, st)) return fail(c, DEM_ERR_OOM, "facet bin buffers");
    o.frec = ptr<uint4>(S.frec);
    o.nfreg = (long long)NFR;
    launch_facet_scatter(c->D, o, t, travel, st);
  }
  o.d_np = tot + 5;
  o.next_bin = tot + 7;
  o.chunk = c->tiles.narrow_chunk;
  // the find passes append the kept pairs (and facet candidates) to
  // unordered buffers sized from the last rebuild; if they did not fit they
  // grow and the passes run again
  unsigned long long NP = 0, NF = 0;
  for (int attempt = 0;; ++attempt) {
    if (S.ucap == 0) S.ucap = (unsigned long long)std::max<long long>(2 * ns, 1 << 16);
    if (!grow(c, S.upairs, 8 * (size_t)S.ucap, 0, st)) return fail(c, DEM_ERR_OOM, "pair buffer");
    o.upairs = ptr<uint2>(S.upairs);
    o.ucap = S.ucap;
    cudaMemsetAsync(o.pair_cnt, 0, 4 * (size_t)ns, st);
    cudaMemsetAsync(o.d_np, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(o.next_bin, 0, sizeof(unsigned long long), st);
    launch_narrow(c->D, o, st);
    exclusive_scan_u32(o.pair_cnt, o.pair_off, ns, S.scan_scr.p, tot + 3, st);
    cudaMemcpyAsync(h_tot + 3, tot + 3, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (facets) {
      if (S.fcap == 0) S.fcap = 1 << 16;
      if (!grow(c, S.fcand, 8 * (size_t)S.fcap, 0, st)) return fail(c, DEM_ERR_OOM, "facet candidates");
      o.fcand = ptr<uint2>(S.fcand);
      o.fcap = S.fcap;
      cudaMemsetAsync(o.fcnt, 0, 4 * (size_t)ns, st);
      cudaMemsetAsync(o.d_nf, 0, sizeof(unsigned long long), st);
      launch_facet_narrow(c->D, o, m, nullptr, t, travel, st);
      cudaMemcpyAsync(h_tot + 9, tot + 9, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check(c, "narrow phase");
    NP = h_tot[3];
    NF = h_tot[9];
    if (NP <= S.ucap && NF <= S.fcap) break;
    if (attempt > 0) return fail(c, DEM_ERR_STATE, "internal: pair buffer regrown twice");
    if (NP > S.ucap) S.ucap = NP + NP / 4 + 1024;
    if (NF > S.fcap) S.fcap = NF + NF / 4 + 1024;
  }
  const unsigned long long NW = NWA + NF;
  if (NW >= (1ull << 31)) return fail(c, DEM_ERR_CAPACITY, "wall list exceeds 2^31 entries");
  if (NF > 0) {  // rows hold analytic walls and facets: counts and offsets again
    launch_add_facet_counts(c->D, o, st);
    exclusive_scan_u32(o.wall_cnt, o.wall_off, ns, S.scan_scr.p, tot + 10, st);
  }
  o.np = (long long)NP;
  if (NP >= (1ull << 31)) return fail(c, DEM_ERR_CAPACITY, "pair list exceeds 2^31 entries");
  if (li < 3 && c->P.max_contacts > 0 && (long long)NP > c->P.max_contacts)
    return fail(c, DEM_ERR_CAPACITY, "pair list exceeds max_contacts");
  int rc = size_list(c, li, NP, NW, li < 3, st);
  if (rc) return rc;
  ContactList& L = LB.L;
  const uint32_t np32 = (uint32_t)NP, nw32 = (uint32_t)NW;
  const long long lens[2] = {(long long)NP, (long long)NW};
  cudaMemcpyAsync(L.dn, lens, sizeof(lens), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.row + ns, &np32, 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.wrow + ns, &nw32, 4, cudaMemcpyHostToDevice, st);
  launch_list_rows(c->D, o, L, old, old_ns, st);
  launch_wall_emit(c->D, o, L.ws, L.ww, st);
  launch_facet_finish(c->D, o, (long long)NF, L.ws, L.ww, st);
  cudaStreamSynchronize(st);  // the two host scalars above must outlive their copies
  return cuda_check(c, "detect_into");
}

// Detection into lists[li] with margin m (per clump from D.cmargin when set),
// for a list that must last K steps (wall travel) -- also used by the audit.
// With an old list (old != NULL) the tangential history of the pairs both
// lists hold is carried over as the rows are built.  wall_extra widens the
// wall candidates' threshold; si picks the scratch set, st the stream.
int detect_into(dem_ctx* c, int li, double m, int K, const ContactList* old = nullptr,
                long long old_ns = 0, double wall_extra = 0.0, int si = 0, cudaStream_t st = nullptr) {
  if (!st) st = c->st;
  DetJob J;
  int rc = detect_prepare(c, li, m, K, wall_extra, si, st, J);
  if (rc) return rc;
  return detect_finish(c, J, old, old_ns, st);
}

// The list at margin m for K steps into lists[li], filtered from the outer
// list (lists[3]); with an old list its tangential history is carried over.
// *bad is set, and lists[li] left unused, when a sphere has left the
// allowance around its outer-list lattice point.
int filter_into(dem_ctx* c, int li, double m, int K, const ContactList* old, long long old_ns,
                bool* bad) {
  const long long ns = c->ns;
  const double t = (double)c->step * c->P.dt;
  const double travel = c->P.dt * (double)std::max(1, K);
  auto& LB = c->lists[li];
  const ContactList& O = c->lists[3].L;
  if (!grow(c, c->ds[0].det, sizeof(int4) * (ns + 1)) || !grow(c, c->ds[0].wall_cnt, 4 * (ns + 1)) ||
      !grow(c, c->ds[0].pair_cnt, 4 * (ns + 1)) || !grow(c, LB.row, 4 * (ns + 1)) ||
      !grow(c, LB.wrow, 4 * (ns + 1)) || !grow(c, c->ds[0].scan_scr, scan_scratch_bytes(ns + 1) + 256) ||
      !grow(c, c->ds[0].fkeep, (size_t)O.n + 16) || !grow(c, c->ds[0].wkeep, 4 * (ns + 1)))
    return fail(c, DEM_ERR_OOM, "detection buffers");
  DetectOut o{};
  o.det = ptr<int4>(c->ds[0].det);
  o.fkeep = ptr<uint8_t>(c->ds[0].fkeep);
  o.wkeep = ptr<uint32_t>(c->ds[0].wkeep);
  o.wall_cnt = ptr<uint32_t>(c->ds[0].wall_cnt);
  o.wall_off = ptr<uint32_t>(LB.wrow);
  o.pair_cnt = ptr<uint32_t>(c->ds[0].pair_cnt);
  o.pair_off = ptr<uint32_t>(LB.row);
  o.n_tsph = (int)c->tpl_rad.size();
  if (!grow(c, c->ds[0].trho, 4 * (size_t)(o.n_tsph + 1))) return fail(c, DEM_ERR_OOM, "detection buffers");
  o.trho = ptr<int>(c->ds[0].trho);
  unsigned long long* tot = ptr<unsigned long long>(c->ds[0].totals);
  cudaMemsetAsync(tot + 11, 0, sizeof(unsigned long long), c->st);
  launch_lattice_check(c->D, o, m, ptr<int4>(c->b_q0), tot + 11, c->st);
  launch_filter_count(c->D, o, O, m, t, travel, c->st);
  exclusive_scan_u32(o.pair_cnt, o.pair_off, ns, c->ds[0].scan_scr.p, tot + 3, c->st);
  exclusive_scan_u32(o.wall_cnt, o.wall_off, ns, c->ds[0].scan_scr.p, tot + 1, c->st);
  unsigned long long h_tot[12] = {};
  cudaMemcpyAsync(h_tot, tot, 12 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "filter");
  *bad = h_tot[11] != 0;
  if (*bad) return DEM_OK;
  const unsigned long long NP = h_tot[3], NW = h_tot[1];
  if (c->P.max_contacts > 0 && (long long)NP > c->P.max_contacts)
    return fail(c, DEM_ERR_CAPACITY, "pair list exceeds max_contacts");
  int rc = size_list(c, li, NP, NW, true);
  if (rc) return rc;
  ContactList& L = LB.L;
  const uint32_t np32 = (uint32_t)NP, nw32 = (uint32_t)NW;
  const long long lens[2] = {(long long)NP, (long long)NW};
  cudaMemcpyAsync(L.dn, lens, sizeof(lens), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(L.row + ns, &np32, 4, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(L.wrow + ns, &nw32, 4, cudaMemcpyHostToDevice, c->st);
  launch_filter_emit(c->D, o, O, L, m, t, travel, c->st);
  if (old) launch_hist_pairs(*old, L, old_ns, c->st);
  cudaStreamSynchronize(c->st);  // the two host scalars above must outlive their copies
  return cuda_check(c, "filter_into");
}

// A new outer list: a detection at outer_factor x m whose wall candidates
// cover the walls' travel over outer_n intervals of K steps and 2^-21 m more
// than the margins' difference; its lattice points and radii are kept.
int build_outer(dem_ctx* c, double m, int K) {
  const double mo = c->outer_factor * m;
  int rc = detect_into(c, 3, mo, c->outer_n * std::max(1, K), nullptr, 0, 0x1p-21);
  if (rc) return rc;
  if (!grow(c, c->b_q0, sizeof(int4) * (c->ns + 1))) return fail(c, DEM_ERR_OOM, "outer list points");
  cudaMemcpyAsync(c->b_q0.p, c->ds[0].det.p, sizeof(int4) * c->ns, cudaMemcpyDeviceToDevice, c->st);
  c->outer_valid = true;
  c->outer_used = 0;
  c->outer_ns = c->ns;
  c->outer_m = m;
  c->outer_K = K;
  c->outer_until = c->step + (long long)c->outer_n * std::max(1, K);
  c->stats.outer_rebuilds++;
  return DEM_OK;
}

// The next outer list on the second stream (the paper's kinematics thread
// computing the contact list while the dynamics thread steps, section 2.2,
// on one GPU): its state-reading part is queued on the context stream now,
// in order with the steps, and ev_snap marks it; outer_async_finish queues
// the rest on st2 after the interval's steps have been queued, so that the
// host's waits for its sizes overlap them; outer_async_adopt makes it the
// outer list once the context stream has waited for ev_ready.  Its lattice
// points are those of the time it was started, so every rebuild's
// allowance check covers the steps since then.  st2 is idle whenever a call
// returns to the user (dem_step waits for it), so nothing the user changes
// between calls can be in use there.
int outer_async_start(dem_ctx* c, double m, int K) {
  if (!c->st2) {
    if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_snap, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess)
      return cuda_check(c, "second stream");
  }
  const long long layout = c->layout;
  // it is adopted at the next rebuild, at most K steps later, and serves
  // outer_n rebuilds from there: its wall candidates cover (outer_n + 1) K steps
  int rc = detect_prepare(c, 4, c->outer_factor * m, (c->outer_n + 1) * std::max(1, K), 0x1p-21, 1,
                          c->st, c->async_job);
  c->layout = layout;  // no captured graph refers to the second outer list's buffers
  if (rc) return rc;
  cudaEventRecord(c->ev_snap, c->st);
  c->async_state = 1;
  c->async_m = m;
  c->async_K = K;
  c->async_ns = c->ns;
  c->async_until = c->step + (long long)(c->outer_n + 1) * std::max(1, K);
  return cuda_check(c, "outer list start");
}

int outer_async_finish(dem_ctx* c) {
  if (c->async_state != 1) return DEM_OK;
  const long long layout = c->layout;
  cudaStreamWaitEvent(c->st2, c->ev_snap, 0);
  int rc = detect_finish(c, c->async_job, nullptr, 0, c->st2);
  if (rc == DEM_OK && !grow(c, c->b_q1, sizeof(int4) * (c->ns + 1), 0, c->st2))
    rc = fail(c, DEM_ERR_OOM, "outer list points");
  c->layout = layout;
  if (rc) return rc;
  cudaMemcpyAsync(c->b_q1.p, c->ds[1].det.p, sizeof(int4) * c->ns, cudaMemcpyDeviceToDevice, c->st2);
  cudaEventRecord(c->ev_ready, c->st2);
  c->async_state = 2;
  return cuda_check(c, "outer list finish");
}

void outer_async_adopt(dem_ctx* c) {
  cudaStreamWaitEvent(c->st, c->ev_ready, 0);
  std::swap(c->lists[3], c->lists[4]);
  std::swap(c->b_q0, c->b_q1);
  c->outer_valid = true;
  c->outer_used = 0;
  c->outer_ns = c->async_ns;
  c->outer_m = c->async_m;
  c->outer_K = c->async_K;
  c->outer_until = c->async_until;
  c->async_state = 0;
  c->stats.outer_rebuilds++;
}

// Drops an outer list in progress (its buffers are reused only after st2 is idle).
int outer_async_drop(dem_ctx* c) {
  int rc = DEM_OK;
  if (c->async_state == 1) rc = outer_async_finish(c);
  if (c->st2) cudaStreamSynchronize(c->st2);
  c->async_state = 0;
  return rc;
}

// The outer lists no longer hold (new clumps, a new wall motion).
int invalidate_outer(dem_ctx* c) {
  c->outer_valid = false;
  return outer_async_drop(c);
}

// Rebuilds the current list with margin m (per clump when D.cmargin is set)
// for a list meant to last K steps; history is carried from the old list.
// With the two-level list on (and one margin for all clumps) the list is
// filtered from the outer list, which is detected again when it has served
// its rebuilds or a sphere has left its allowance.
int rebuild(dem_ctx* c, double m, int K, bool allow_outer = true) {
  const int nxt = c->cur == 0 ? 1 : 0;
  if (c->timing) cudaEventRecord(c->ev[0], c->st);
  const ContactList* old = c->have_list ? &curL(c) : nullptr;
  int rc;
  if (allow_outer && c->outer_n > 0 && !c->D.cmargin && m > 0.0) {
    if (c->async_state == 1 && (rc = outer_async_finish(c))) return rc;
    // (a list whose wall candidates no longer cover this list's K steps, as
    // after steps of the learned rule in between, is not used)
    const long long until = c->step + std::max(1, K);
    if (c->async_state == 2 && (!c->outer_valid || c->outer_used >= c->outer_n) &&
        c->async_ns == c->ns && c->async_m == m && c->async_K == K && until <= c->async_until)
      outer_async_adopt(c);
    const bool stale = !c->outer_valid || c->outer_used >= c->outer_n || c->outer_ns != c->ns ||
                       c->outer_m != m || c->outer_K != K || until > c->outer_until;
    if (stale && (rc = outer_async_drop(c))) return rc;
    if (stale && (rc = build_outer(c, m, K))) return rc;
    bool bad = false;
    if ((rc = filter_into(c, nxt, m, K, old, c->list_ns, &bad))) return rc;
    if (bad) {  // a sphere moved past its allowance: a new outer list
      if ((rc = outer_async_drop(c)) || (rc = build_outer(c, m, K)) ||
          (rc = filter_into(c, nxt, m, K, old, c->list_ns, &bad)))
        return rc;
      if (bad) return fail(c, DEM_ERR_STATE, "internal: a fresh outer list fails its own check");
    }
    c->outer_used++;
    // the next outer list, started while this one serves its last interval;
    // the next rebuild finishes it (with the interval's steps already queued)
    if (c->outer_async && c->n_facets == 0 && c->async_state == 0 &&
        c->outer_used >= c->outer_n && (rc = outer_async_start(c, m, K)))
      return rc;
  } else {
    rc = detect_into(c, nxt, m, K, old, c->list_ns);
    if (rc) return rc;
  }
  ContactList& N = c->lists[nxt].L;
  if (old) launch_hist_walls(*old, N, c->list_ns, c->st);
  if (c->P.precision != DEM_FP64) launch_pair_owners(c->D, N, c->st);
  c->cur = nxt;
  c->list_ns = c->ns;
  c->have_list = true;
  c->need_rebuild = false;
  c->since = 0;
  launch_set_cert_ref(c->D, c->st);
  if ((rc = build_det_lists(c))) return rc;
  c->stats.rebuilds++;
  c->stats.bin_entries = c->n_entries;
  c->stats.n_pairs = N.n;
  c->stats.n_wall_contacts = N.nw;
  if (c->timing) {
    cudaEventRecord(c->ev[1], c->st);
    cudaEventSynchronize(c->ev[1]);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    c->stats.ms_detect += ms;
  }
  return cuda_check(c, "rebuild");
}
int rebuild(dem_ctx* c) { return rebuild(c, c->margin, c->P.rebuild_interval, false); }

// Sphere-sphere then sphere-wall contact forces; `mid` (optional) is recorded
// between the two kernels.
// Zeroes the per-clump force / torque accumulators if something other than
// the update kernel (which clears them as it reads them) left them dirty.
void clear_acc(dem_ctx* c) {
  if (!c->acc_dirty) return;
  if (c->P.precision == DEM_FP64) cudaMemsetAsync(c->b_acc64.p, 0, 64 * (size_t)c->ncl, c->st);
  else cudaMemsetAsync(c->b_acc32.p, 0, 32 * (size_t)c->ncl, c->st);
  c->acc_dirty = false;
}

int force_pass(dem_ctx* c, bool count_active, cudaEvent_t mid = nullptr) {
  clear_acc(c);
  if (!c->walls.empty()) {
    cudaMemsetAsync(c->b_wforce.p, 0, 24 * c->walls.size(), c->st);
    cudaMemsetAsync(c->b_wtorque.p, 0, 24 * c->walls.size(), c->st);
  }
  const double t = (double)c->step * c->P.dt;
  ContactList& L = curL(c);
  launch_force_pairs(c->D, L, count_active, c->st);
  if (mid) cudaEventRecord(mid, c->st);
  launch_force_walls(c->D, L, t, count_active, c->st);
  if (c->D.det_off) launch_det_gather(c->D, L, c->st);
  return DEM_OK;
}

// Reads and clears the device flags and counters; *guard_hit tells whether the
// displacement certificate failed since the last read.
int read_flags(dem_ctx* c, bool* guard_hit = nullptr) {
  int flags = 0;
  unsigned long long ctr[2] = {0, 0};
  cudaMemcpyAsync(&flags, c->b_flags.p, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(ctr, c->b_counters.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->st);
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "step");
  cudaMemsetAsync(c->b_flags.p, 0, sizeof(int), c->st);
  cudaMemsetAsync(c->b_counters.p, 0, 2 * sizeof(unsigned long long), c->st);
  if (ctr[0]) c->stats.active_last = (long long)ctr[0];
  c->stats.guard_violations += (long long)ctr[1];
  if (guard_hit) *guard_hit = (flags & kFlagGuard) != 0;
  if (flags & kFlagNonFinite) return fail(c, DEM_ERR_NONFINITE, "non-finite clump state");
  if (flags & kFlagBounds) return fail(c, DEM_ERR_STATE, "internal: narrow-phase row overflow");
  if (flags & kFlagTimeout) return fail(c, DEM_ERR_TIMEOUT, "a bounded device wait ran out");
  return cuda_check(c, "step");
}

// ---------------------------------------------------------------------------
// learned rebuild rule
// ---------------------------------------------------------------------------
FeatureScales feature_scales(const dem_ctx* c) {
  FeatureScales f;
  f.h = (float)c->P.dt;
  f.rmean = (float)c->r_mean;
  f.gmag = (float)std::sqrt(c->P.g[0] * c->P.g[0] + c->P.g[1] * c->P.g[1] + c->P.g[2] * c->P.g[2]);
  return f;
}

// Per-clump margins from the regressor (sets D.cmargin).
int predict_margins(dem_ctx* c) {
  const long long ncl = c->ncl, nb = c->n_lbins;  // bins of the feature grids
  const int nc = (int)c->l_cand.size();
  if (!grow(c, c->b_chome, 4 * (ncl + 1)) || !grow(c, c->b_cmargin, 4 * (ncl + 1)) ||
      !grow(c, c->b_bcnt, 4 * (nb + 1)) || !grow(c, c->b_bvmax, 4 * (nb + 1)) ||
      !grow(c, c->b_bvsum, 4 * (nb + 1)) || !grow(c, c->b_bamax, 4 * (nb + 1)) ||
      !grow(c, c->b_occ, 4 * (nb + 1)) || !grow(c, c->b_binm, 4 * (nb + 1)) ||
      !grow(c, c->b_nocc, 64) || !grow(c, c->b_cand, 4 * (size_t)nc))
    return fail(c, DEM_ERR_OOM, "learned-rule buffers");
  std::vector<float> cf(c->l_cand.begin(), c->l_cand.end());
  cudaMemcpyAsync(c->b_cand.p, cf.data(), 4 * (size_t)nc, cudaMemcpyHostToDevice, c->st);
  BinStats bs{ptr<uint32_t>(c->b_chome), ptr<uint32_t>(c->b_bcnt), ptr<int>(c->b_bvmax),
              ptr<float>(c->b_bvsum), ptr<int>(c->b_bamax)};
  cudaMemsetAsync(bs.cnt, 0, 4 * (size_t)nb, c->st);
  cudaMemsetAsync(bs.vmax, 0, 4 * (size_t)nb, c->st);
  cudaMemsetAsync(bs.vsum, 0, 4 * (size_t)nb, c->st);
  cudaMemsetAsync(bs.amax, 0, 4 * (size_t)nb, c->st);
  cudaMemsetAsync(c->b_nocc.p, 0, 4, c->st);
  c->D.cmargin = nullptr;
  DevState dl = c->D;
  dl.grids = ptr<SceneGrid>(c->b_lgrids);
  launch_clump_home(dl, bs, c->st);
  launch_bin_compact(bs.cnt, nb, ptr<uint32_t>(c->b_occ), ptr<uint32_t>(c->b_nocc), c->st);
  uint32_t nocc = 0;
  cudaMemcpyAsync(&nocc, c->b_nocc.p, 4, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  c->n_occ = nocc;
  const long long rows = (long long)nocc * nc;
  if (!grow(c, c->b_feat, 4 * (size_t)(rows + 1) * kMlpIn) || !grow(c, c->b_pred, 4 * (size_t)(rows + 1)))
    return fail(c, DEM_ERR_OOM, "feature buffers");
  launch_bin_features(bs, ptr<uint32_t>(c->b_occ), nocc, nc, ptr<float>(c->b_cand), feature_scales(c),
                      ptr<float>(c->b_feat), c->st);
  if (c->mlp) {
    mlp_forward_tc_dev(mlp_weights(c->mlp), ptr<float>(c->b_feat), rows, ptr<float>(c->b_pred),
                       ptr<int>(c->b_flags), c->st);
    const float ln_need = (float)std::log(std::max(1.0, c->l_interval * c->l_safety));
    launch_choose_margin(ptr<uint32_t>(c->b_occ), nocc, nc, ptr<float>(c->b_cand),
                         ptr<float>(c->b_pred), ln_need, ptr<float>(c->b_binm), c->st);
    const float floor_scale = (float)(c->l_floor * c->P.dt * c->l_interval);
    launch_clump_margin(c->D, bs.chome, ptr<float>(c->b_binm), floor_scale,
                        ptr<float>(c->b_cmargin), c->st);
    c->D.cmargin = ptr<float>(c->b_cmargin);
  }
  return cuda_check(c, "predict margins");
}

// State and list history at a rebuild, for a rollback.
int take_snapshot(dem_ctx* c) {
  const size_t n = (size_t)c->ncl;
  const bool f64 = c->P.precision == DEM_FP64;
  ContactList& L = curL(c);
  // position 32 | orientation 32 | velocity record 48 | certificate reference
  // 48 bytes per clump
  if (!grow(c, c->s_state, 160 * (n + 1)) || !grow(c, c->s_pb, 4 * (size_t)(L.n + 1)) ||
      !grow(c, c->s_u, 24 * (size_t)(L.n + 1)) || !grow(c, c->s_ww, 4 * (size_t)(L.nw + 1)) ||
      !grow(c, c->s_uw, 24 * (size_t)(L.nw + 1)))
    return fail(c, DEM_ERR_OOM, "snapshot");
  char* s = (char*)c->s_state.p;
  if (f64) {
    cudaMemcpyAsync(s, c->b_cpos.p, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  } else {
    cudaMemcpyAsync(s, c->b_cvox.p, 16 * n, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(s + 16 * n, c->b_coff.p, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  }
  cudaMemcpyAsync(s + 32 * n, c->b_cq.p, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(s + 64 * n, c->b_cvw.p, sizeof(VelRec) * n, cudaMemcpyDeviceToDevice, c->st);
  if (f64) {
    cudaMemcpyAsync(s + 112 * n, c->b_ref_pos.p, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  } else {
    cudaMemcpyAsync(s + 112 * n, c->b_ref_vox.p, 16 * n, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(s + 128 * n, c->b_ref_off.p, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  }
  cudaMemcpyAsync(s + 144 * n, c->b_ref_q.p, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->s_pb.p, L.pb, 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, c->st);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync((double*)c->s_u.p + k * L.n, L.u + k * L.cap, 8 * (size_t)L.n,
                    cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->s_ww.p, L.ww, 4 * (size_t)L.nw, cudaMemcpyDeviceToDevice, c->st);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync((double*)c->s_uw.p + k * L.nw, L.uw + k * L.capw, 8 * (size_t)L.nw,
                    cudaMemcpyDeviceToDevice, c->st);
  c->snap_step = c->step;
  return cuda_check(c, "snapshot");
}

int restore_snapshot(dem_ctx* c) {
  const size_t n = (size_t)c->ncl;
  const bool f64 = c->P.precision == DEM_FP64;
  ContactList& L = curL(c);
  const char* s = (const char*)c->s_state.p;
  if (f64) {
    cudaMemcpyAsync(c->b_cpos.p, s, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  } else {
    cudaMemcpyAsync(c->b_cvox.p, s, 16 * n, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->b_coff.p, s + 16 * n, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  }
  cudaMemcpyAsync(c->b_cq.p, s + 32 * n, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(c->b_cvw.p, s + 64 * n, sizeof(VelRec) * n, cudaMemcpyDeviceToDevice, c->st);
  if (f64) {
    cudaMemcpyAsync(c->b_ref_pos.p, s + 112 * n, 32 * n, cudaMemcpyDeviceToDevice, c->st);
  } else {
    cudaMemcpyAsync(c->b_ref_vox.p, s + 112 * n, 16 * n, cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->b_ref_off.p, s + 128 * n, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  }
  cudaMemcpyAsync(c->b_ref_q.p, s + 144 * n, 16 * n, cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(L.pb, c->s_pb.p, 4 * (size_t)L.n, cudaMemcpyDeviceToDevice, c->st);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync(L.u + k * L.cap, (double*)c->s_u.p + k * L.n, 8 * (size_t)L.n,
                    cudaMemcpyDeviceToDevice, c->st);
  cudaMemcpyAsync(L.ww, c->s_ww.p, 4 * (size_t)L.nw, cudaMemcpyDeviceToDevice, c->st);
  for (int k = 0; k < 3; ++k)
    cudaMemcpyAsync(L.uw + k * L.capw, (double*)c->s_uw.p + k * L.nw, 8 * (size_t)L.nw,
                    cudaMemcpyDeviceToDevice, c->st);
  c->step = c->snap_step;
  // accumulators are zero after every update; poses, mirrors and walls follow
  // the state; the motion bounds hold for the restored certificate reference
  c->D.cmargin = nullptr;
  launch_update(c->D, false, c->step, c->margin, true, c->st);
  return cuda_check(c, "restore");
}


void drop_graphs(dem_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

// Captures (once per list buffer, step count and margin) and launches a graph
// of m force + update steps with the current list.
int launch_graph_steps(dem_ctx* c, int m, double margin, bool cert) {
  // accumulators left dirty are cleared on the stream, before and outside the
  // graph (so the captured force passes hold no clear)
  clear_acc(c);
  if (c->graph_layout != c->layout) {
    drop_graphs(c);
    c->graph_layout = c->layout;
  }
  dem_ctx::GraphEntry* ge = nullptr;
  for (auto& g : c->graphs)
    if (g.cur == c->cur && g.m == m && g.cert == (int)cert && g.margin == margin) ge = &g;
  if (!ge) {
    const long long k0 = g_kernel_launches;
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return cuda_check(c, "begin capture");
    for (int j = 0; j < m; ++j) {
      force_pass(c, false);
      launch_update(c->D, true, c->step + j + 1, margin, cert, c->st);
    }
    if (cudaStreamEndCapture(c->st, &graph) != cudaSuccess) return cuda_check(c, "end capture");
    cudaGraphExec_t exec;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_check(c, "instantiate");
    }
    cudaGraphDestroy(graph);
    const long long kernels = g_kernel_launches - k0;
    g_kernel_launches = k0;
    c->graphs.push_back({c->cur, m, (int)cert, margin, exec, kernels});
    ge = &c->graphs.back();
  }
  if (cudaGraphLaunch(ge->exec, c->st) != cudaSuccess) return cuda_check(c, "graph launch");
  g_kernel_launches += ge->kernels;
  return DEM_OK;
}

int audit_now(dem_ctx* c, long long* missed);

// Runs steps on the context stream.  The plain rule rebuilds every K steps;
// the guarded path runs blocks that start with a rebuild and a snapshot and,
// when the displacement certificate failed inside a block, rolls back and
// replays it with the plain rule, or with a rebuild every step if that fails
// too.  Per-phase events are recorded for the first 8192 steps of a call.
struct StepRunner {
  dem_ctx* c;
  int n_calls;
  int n_timed = 0;
  int it = 0;
  StepRunner(dem_ctx* cc, int n) : c(cc), n_calls(n) {}
  int init() {
    n_timed = c->timing ? 8192 : 0;
    while ((int)c->evpool.size() < 4 * n_timed) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(c, "event pool");
      c->evpool.push_back(e);
    }
    return DEM_OK;
  }
  // one force evaluation + update with the current list
  void step(double margin, bool cert, bool last) {
    const bool tm = it < n_timed;
    cudaEvent_t* ev = tm ? &c->evpool[4 * (size_t)it] : nullptr;
    if (tm) cudaEventRecord(ev[0], c->st);
    force_pass(c, last, tm ? ev[1] : nullptr);
    if (tm) cudaEventRecord(ev[2], c->st);
    launch_update(c->D, true, c->step + 1, margin, cert, c->st);
    if (tm) cudaEventRecord(ev[3], c->st);
    ++it;
    c->step++;
    c->since++;
    c->stats.steps++;
    c->stats.pair_steps += curL(c).n + curL(c).nw;
  }
  int run_plain(int n, double margin, int K, bool last_counts) {
    const bool cert = c->P.guard != DEM_GUARD_OFF && margin > 0.0;
    c->D.cmargin = nullptr;
    for (int i = 0; i < n;) {
      if (c->need_rebuild || !c->have_list || c->since >= K) {
        int rc = rebuild(c, margin, K);
        if (rc) return rc;
      }
      // steps left on this list; the call's last step runs on its own so that
      // it can count the active contacts
      int m = std::min(K - c->since, n - i);
      if (last_counts && i + m == n) --m;
      if (c->use_graphs && !c->timing && m >= 2) {
        int rc = launch_graph_steps(c, m, margin, cert);
        if (rc) return rc;
        for (int j = 0; j < m; ++j) {
          c->step++;
          c->since++;
          c->stats.steps++;
          c->stats.pair_steps += curL(c).n + curL(c).nw;
        }
        i += m;
        continue;
      }
      step(margin, cert, last_counts && i == n - 1);
      ++i;
    }
    return DEM_OK;
  }
  // Learned rule, halt mode: one interval of up to K steps with per-clump
  // margins; the device skips every step after the first state that fails
  // the certificate.  Returns the steps completed (>= 1) in *done.
  int run_halting(int nb, int* done) {
    long long* halt = ptr<long long>(c->b_dstep) + 1;
    static const long long big = LLONG_MAX;
    cudaMemcpyAsync(halt, &big, sizeof(big), cudaMemcpyHostToDevice, c->st);
    const float* cm = c->D.cmargin;
    const long long step0 = c->step, n_list = curL(c).n + curL(c).nw;
    c->D.halt_at = halt;
    if (!c->h_halt) {
      if (cudaHostAlloc(reinterpret_cast<void**>(&c->h_halt), 2 * sizeof(long long),
                        cudaHostAllocDefault) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_halt[0], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_halt[1], cudaEventDisableTiming) != cudaSuccess)
        return cuda_check(c, "halt read-back");
    }
    // the interval is launched in chunks; after each chunk the halt step is
    // copied to the host, and the copy of the chunk before is waited for
    // while this one runs: once a halt is seen, no further chunk is launched
    // (the steps launched after the halt return at once on the device)
    constexpr int kChunk = 8;
    int launched = 0, k = 0;
    while (launched < nb) {
      const int m = std::min(kChunk, nb - launched);
      for (int j = 0; j < m; ++j) {
        c->D.cmargin = cm;
        step(c->margin, true, launched + j == nb - 1);
      }
      launched += m;
      cudaMemcpyAsync(c->h_halt + (k & 1), halt, sizeof(long long), cudaMemcpyDeviceToHost, c->st);
      cudaEventRecord(c->ev_halt[k & 1], c->st);
      if (k > 0) {
        cudaEventSynchronize(c->ev_halt[(k - 1) & 1]);
        if (c->h_halt[(k - 1) & 1] != LLONG_MAX) break;
      }
      ++k;
    }
    c->D.halt_at = nullptr;
    long long dstep = 0;
    cudaMemcpyAsync(&dstep, c->b_dstep.p, sizeof(dstep), cudaMemcpyDeviceToHost, c->st);
    bool hit = false;
    int rc = read_flags(c, &hit);  // synchronises: dstep and the halt value are in
    if (rc) return rc;
    const long long d = dstep - step0;
    if (d < 1 || d > launched) return fail(c, DEM_ERR_STATE, "internal: halted interval out of range");
    const long long undone = launched - d;
    if (undone > 0) {
      c->step -= undone;
      c->since -= (int)undone;
      c->stats.steps -= undone;
      c->stats.pair_steps -= undone * n_list;
      c->stats.early_rebuilds++;
    }
    *done = (int)d;
    return DEM_OK;
  }
  int run_guarded(int n) {
    while (n > 0) {
      const bool learned = c->mlp != nullptr;
      const int K = learned ? c->l_interval : std::max(1, c->P.rebuild_interval);
      const int nb = std::min(n, K);
      int rc;
      if (learned) {
        if (c->timing) cudaEventRecord(c->ev[2], c->st);
        if ((rc = predict_margins(c))) return rc;
        if (c->timing) {
          cudaEventRecord(c->ev[3], c->st);
          cudaEventSynchronize(c->ev[3]);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
          c->stats.ms_predict += ms;
        }
      } else {
        c->D.cmargin = nullptr;
      }
      const float* cm = c->D.cmargin;
      if ((rc = rebuild(c, c->margin, K))) return rc;
      if (learned && c->l_mode == DEM_LEARNED_HALT) {
        int done = 0;
        if ((rc = run_halting(nb, &done))) return rc;
        c->need_rebuild = true;  // the next interval starts with its own prediction and rebuild
        n -= done;
        continue;
      }
      if ((rc = take_snapshot(c))) return rc;
      bool hit = false;
      if ((rc = read_flags(c, &hit))) return rc;  // clears flags before the block
      for (int i = 0; i < nb; ++i) {
        c->D.cmargin = cm;
        step(c->margin, true, i == nb - 1);
      }
      if ((rc = read_flags(c, &hit))) return rc;
      if (!hit && learned) {
        // the learned interval is also judged by the exact check against a
        // fresh zero-margin detection
        long long missed = 0;
        if ((rc = audit_now(c, &missed))) return rc;
        hit = missed > 0;
      }
      if (hit) {
        // roll back and replay the block with the plain rule
        c->stats.rollbacks++;
        if ((rc = restore_snapshot(c))) return rc;
        c->need_rebuild = true;
        if ((rc = run_plain(nb, c->margin, std::max(1, c->P.rebuild_interval), true))) return rc;
        if ((rc = read_flags(c, &hit))) return rc;
        if (hit) {
          // the speed bound of the plain rule was exceeded too: rebuild every step
          c->stats.rollbacks++;
          if ((rc = restore_snapshot(c))) return rc;
          c->need_rebuild = true;
          if ((rc = run_plain(nb, 0.0, 1, true))) return rc;
        }
      }
      c->need_rebuild = true;  // the next block starts with its own rebuild
      n -= nb;
    }
    c->D.cmargin = nullptr;
    return DEM_OK;
  }
  void finish() {
    const int nt = std::min(it, n_timed);
    for (int k = 0; k < nt; ++k) {
      const cudaEvent_t* ev = &c->evpool[4 * (size_t)k];
      float a = 0.f, b = 0.f, u = 0.f;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[1], ev[2]);
      cudaEventElapsedTime(&u, ev[2], ev[3]);
      c->stats.ms_pairs += a;
      c->stats.ms_walls += b;
      c->stats.ms_update += u;
      c->stats.timed_steps++;
    }
  }
};

int upload_clumps(dem_ctx* c, long long first, int n, const int* tpl, const double* pos,
                  const double* quat, const double* vel, const double* angvel) {
  const bool f64 = c->P.precision == DEM_FP64;
  std::vector<double4_32a> vq(n), vp;
  std::vector<VelRec> vr(n);
  std::vector<int4> vx;
  std::vector<float4> vo;
  if (f64) vp.resize(n); else { vx.resize(n); vo.resize(n); }
  for (int i = 0; i < n; ++i) {
    const double* q = quat + 4 * i;
    vq[i] = make_double4_32a(q[0], q[1], q[2], q[3]);
    double wb[3];
    qrot(q, angvel + 3 * i, wb, true);
    vr[i] = VelRec{vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], wb[0], wb[1], wb[2]};
    if (f64) {
      vp[i] = make_double4_32a(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], 0.0);
    } else {
      const SceneH& s = c->scenes[c->h_cscene[first + i]];
      int vox[3];
      float off[3];
      for (int k = 0; k < 3; ++k) {
        const double rel = pos[3 * i + k] - s.lo[k];
        const double m = std::rint(rel / kVoxel);
        if (std::fabs(m) > 2.0e9) return fail(c, DEM_ERR_INVALID_ARG, "clump too far from its scene corner");
        vox[k] = (int)m;
        off[k] = (float)(rel - m * kVoxel);
      }
      vx[i] = make_int4(vox[0], vox[1], vox[2], 0);
      vo[i] = make_float4(off[0], off[1], off[2], 0.f);
    }
  }
  cudaMemcpyAsync(ptr<double4_32a>(c->b_cq) + first, vq.data(), 32 * (size_t)n, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(ptr<VelRec>(c->b_cvw) + first, vr.data(), sizeof(VelRec) * (size_t)n,
                  cudaMemcpyHostToDevice, c->st);
  if (f64) {
    cudaMemcpyAsync(ptr<double4_32a>(c->b_cpos) + first, vp.data(), 32 * (size_t)n, cudaMemcpyHostToDevice, c->st);
  } else {
    cudaMemcpyAsync(ptr<int4>(c->b_cvox) + first, vx.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(ptr<float4>(c->b_coff) + first, vo.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, c->st);
  }
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "upload clumps");
}

bool finite_all(const double* p, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int dem_create(const dem_params* params, dem_ctx** out) {
  if (out) *out = nullptr;
  if (!params || !out) { g_create_error = "null argument"; return DEM_ERR_INVALID_ARG; }
  const dem_params& p = *params;
  auto bad = [&](const char* m) { g_create_error = m; return DEM_ERR_INVALID_ARG; };
  if (!(p.dt > 0.0) || !std::isfinite(p.dt)) return bad("dt must be > 0");
  if (p.precision != DEM_FP64 && p.precision != DEM_FP32_VOXEL) return bad("unknown precision");
  if (p.n_materials < 1 || !p.E || !p.nu || !p.mu || !p.cor) return bad("material table missing");
  if (p.rebuild_interval < 1) return bad("rebuild_interval must be >= 1");
  if (p.margin < 0.0 || p.v_bound < 0.0 || p.bin_size < 0.0) return bad("negative margin / v_bound / bin_size");
  if (p.mix_rule < 0 || p.mix_rule > 2) return bad("unknown mix_rule");
  if (p.n_walls < 0 || (p.n_walls > 0 && !p.walls)) return bad("walls missing");
  if (p.guard < 0 || p.guard > 2) return bad("unknown guard mode");
  if (p.margin_policy != DEM_MARGIN_FIXED && p.margin_policy != DEM_MARGIN_LEARNED) return bad("unknown margin policy");
  if ((p.alloc == nullptr) != (p.free == nullptr)) return bad("alloc and free must be given together");
  for (int k = 0; k < 3; ++k)
    if (!(p.domain_hi[k] > p.domain_lo[k])) return bad("empty domain");
  for (int i = 0; i < p.n_materials; ++i)
    if (!(p.E[i] > 0) || !(p.nu[i] > -1 && p.nu[i] < 0.5) || !(p.mu[i] >= 0) || !(p.cor[i] >= 0 && p.cor[i] <= 1))
      return bad("material out of range");
  for (int w = 0; w < p.n_walls; ++w) {
    const dem_wall& wl = p.walls[w];
    if (wl.type < 0 || wl.type > 3) return bad("unknown wall type");
    if (wl.material < 0 || wl.material >= p.n_materials) return bad("wall material out of range");
    const double nn = wl.n[0] * wl.n[0] + wl.n[1] * wl.n[1] + wl.n[2] * wl.n[2];
    if (!(std::fabs(nn - 1.0) < 1e-9)) return bad("wall normal / axis must be a unit vector");
    if (wl.type == DEM_WALL_CYLINDER && !(wl.radius > 0)) return bad("cylinder radius must be > 0");
    if (wl.type == DEM_WALL_CONE && !(wl.height > 0 && wl.half_angle > 0 && wl.half_angle < 1.5707963)) return bad("bad cone");
    if (wl.type == DEM_WALL_TRIANGLE) {
      double e1[3], e2[3];
      for (int k = 0; k < 3; ++k) { e1[k] = wl.b[k] - wl.p[k]; e2[k] = wl.c[k] - wl.p[k]; }
      const double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
      const double l2 = std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
      const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                   cz = e1[0] * e2[1] - e1[1] * e2[0];
      const double area2 = std::sqrt(cx * cx + cy * cy + cz * cz);
      if (!(area2 > 1e-9 * l1 * l2)) return bad("degenerate triangle");
      // n must be the unit normal (b - p) x (c - p) / |...|
      if (!(std::fabs(cx * wl.n[0] + cy * wl.n[1] + cz * wl.n[2] - area2) <= 1e-9 * area2))
        return bad("triangle normal must be (b - p) x (c - p) normalised");
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    g_create_error = "no CUDA device";
    return DEM_ERR_CUDA;
  }
  if (p.device < 0 || p.device >= ndev) return bad("device ordinal out of range");
  if (cudaSetDevice(p.device) != cudaSuccess) { g_create_error = "cudaSetDevice failed"; return DEM_ERR_CUDA; }
  dem_ctx* c = new dem_ctx();
  c->P = p;
  c->E.assign(p.E, p.E + p.n_materials);
  c->nu.assign(p.nu, p.nu + p.n_materials);
  c->mu.assign(p.mu, p.mu + p.n_materials);
  c->cor.assign(p.cor, p.cor + p.n_materials);
  c->P.E = c->E.data(); c->P.nu = c->nu.data(); c->P.mu = c->mu.data(); c->P.cor = c->cor.data();
  c->user_walls.assign(p.walls, p.walls + p.n_walls);
  c->P.walls = c->user_walls.data();
  if (p.cuda_stream) {
    c->st = (cudaStream_t)p.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      g_create_error = "cudaStreamCreate failed";
      return DEM_ERR_CUDA;
    }
    c->own_stream = true;
  }
  for (auto& e : c->ev) cudaEventCreate(&e);
  SceneH s0{};
  for (int k = 0; k < 3; ++k) { s0.lo[k] = p.domain_lo[k]; s0.hi[k] = p.domain_hi[k]; }
  s0.bin = p.bin_size;
  c->scenes.push_back(s0);
  int rc = build_pair_materials(c);
  if (rc) {
    g_create_error = c->err;
    dem_destroy(c);
    return rc;
  }
  *out = c;
  return DEM_OK;
}

void dem_destroy(dem_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->P.device);
  if (c->st2) cudaStreamSynchronize(c->st2);
  Buf* all[] = {&c->b_tpl_off, &c->b_tp64, &c->b_tp32, &c->b_trm, &c->b_tmat, &c->b_tmass, &c->b_tinert, &c->b_tpbound,
                &c->b_cinfo, &c->b_csph, &c->b_cpos, &c->b_cvox, &c->b_coff, &c->b_cq, &c->b_cvw,
                &c->b_tmassf, &c->b_tinertf, &c->b_mv64, &c->b_mw64, &c->b_mv32, &c->b_mw32, &c->b_acc64, &c->b_acc32, &c->b_ref_pos,
                &c->b_ref_vox, &c->b_ref_off, &c->b_ref_q, &c->b_sinfo, &c->b_sa64, &c->b_sb64, &c->b_srec32,
                &c->b_grids, &c->b_lgrids, &c->b_walls, &c->b_wall_idx, &c->b_wall_scene, &c->b_wfix,
                &c->b_wpos, &c->b_wforce, &c->b_wtorque, &c->b_pm64, &c->b_pm32, &c->b_flags, &c->b_counters,
                &c->b_facet_idx, &c->b_q0,
                &c->b_tmp,
                &c->b_det_cnt, &c->b_det_fill, &c->b_det_off,
                &c->b_det_ids, &c->b_det_pair, &c->b_det_wall, &c->b_dstep, &c->b_alast, &c->b_chome, &c->b_cmargin,
                &c->b_bcnt, &c->b_bvmax, &c->b_bvsum, &c->b_bamax, &c->b_occ, &c->b_nocc,
                &c->b_binm, &c->b_cand, &c->b_feat, &c->b_pred, &c->b_dmax, &c->b_T, &c->b_tr_vox,
                &c->b_tr_off, &c->b_tr_pos, &c->b_tr_q, &c->b_tx, &c->b_tt,
                &c->s_state, &c->s_pb, &c->s_u, &c->s_ww, &c->s_uw};
  for (Buf* b : all) dfree(c, b->p);
  for (auto& S : c->ds) {
    Buf* sb[] = {&S.det, &S.wall_mask, &S.wall_cnt, &S.pair_cnt, &S.bin_size, &S.bin_start,
                 &S.scan_scr, &S.trho, &S.totals, &S.rec, &S.upairs, &S.fbin_size,
                 &S.fbin_start, &S.fcnt, &S.frec, &S.fcand, &S.fkeep, &S.wkeep};
    for (Buf* b : sb) dfree(c, b->p);
  }
  dfree(c, c->b_q1.p);
  for (auto& lb : c->lists) {
    Buf* lbs[] = {&lb.pa, &lb.pb, &lb.pown, &lb.ppm, &lb.u, &lb.row, &lb.ws, &lb.ww, &lb.uw, &lb.wrow, &lb.dnb};
    for (Buf* b : lbs) dfree(c, b->p);
  }
  cudaStreamSynchronize(c->st);
  drop_graphs(c);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->ev_halt[0]) cudaEventDestroy(c->ev_halt[0]);
  if (c->ev_halt[1]) cudaEventDestroy(c->ev_halt[1]);
  if (c->h_halt) cudaFreeHost(c->h_halt);
  if (c->ev_snap) cudaEventDestroy(c->ev_snap);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->own_stream) cudaStreamDestroy(c->st);
  delete c;
}

const char* dem_last_error(const dem_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int dem_load_clump_templates(dem_ctx* c, int n_tpl, const int* off, const double* local_pos,
                             const double* radius, const int* material, const double* mass,
                             const double* inertia) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (c->n_tpl > 0) return fail(c, DEM_ERR_STATE, "templates already loaded");
  if (n_tpl < 1 || !off || !local_pos || !radius || !material || !mass || !inertia)
    return fail(c, DEM_ERR_INVALID_ARG, "template arrays missing");
  if (off[0] != 0) return fail(c, DEM_ERR_INVALID_ARG, "sphere_offsets[0] must be 0");
  for (int t = 0; t < n_tpl; ++t) {
    if (off[t + 1] <= off[t]) return fail(c, DEM_ERR_INVALID_ARG, "each template needs >= 1 sphere");
    if (!(mass[t] > 0) || !(inertia[3 * t] > 0) || !(inertia[3 * t + 1] > 0) || !(inertia[3 * t + 2] > 0))
      return fail(c, DEM_ERR_INVALID_ARG, "mass and inertia must be > 0");
  }
  const int S = off[n_tpl];
  if (!finite_all(local_pos, 3ll * S)) return fail(c, DEM_ERR_INVALID_ARG, "non-finite sphere position");
  for (int s = 0; s < S; ++s) {
    if (!(radius[s] > 0) || !std::isfinite(radius[s])) return fail(c, DEM_ERR_INVALID_ARG, "radius must be > 0");
    if (material[s] < 0 || material[s] >= c->P.n_materials) return fail(c, DEM_ERR_INVALID_ARG, "material out of range");
    // FP32_VOXEL keeps a sphere's centre relative to its clump's voxel corner
    // in 40-bit fixed point (2^-44 m): |p| + voxel must stay below 2^-5 m
    const double* p = local_pos + 3 * s;
    if (c->P.precision != DEM_FP64 &&
        !(std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) < 0.03125 - 2.0 * kVoxel))
      return fail(c, DEM_ERR_INVALID_ARG,
                  "FP32_VOXEL: a template sphere centre lies 31 mm or more from the clump's centre of mass");
  }
  c->n_tpl = n_tpl;
  c->tpl_off.assign(off, off + n_tpl + 1);
  c->tpl_pos.assign(local_pos, local_pos + 3 * S);
  c->tpl_rad.assign(radius, radius + S);
  c->tpl_mat.assign(material, material + S);
  c->tpl_mass.assign(mass, mass + n_tpl);
  c->tpl_inert.assign(inertia, inertia + 3 * n_tpl);
  c->r_max = *std::max_element(radius, radius + S);
  std::vector<double4_32a> tp64(S);
  std::vector<float4> tp32(S);
  std::vector<float2> trm(S);
  std::vector<float> pb(n_tpl, 0.f);
  for (int t = 0; t < n_tpl; ++t)
    for (int s = off[t]; s < off[t + 1]; ++s) {
      const double* p = local_pos + 3 * s;
      tp64[s] = make_double4_32a(p[0], p[1], p[2], radius[s]);
      tp32[s] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)radius[s]);
      float mat_bits;
      std::memcpy(&mat_bits, &material[s], sizeof mat_bits);
      trm[s] = make_float2((float)radius[s], mat_bits);
      pb[t] = std::max(pb[t], (float)std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) * 1.000001f);
    }
  if (!grow(c, c->b_tpl_off, 4 * (n_tpl + 1)) || !grow(c, c->b_tp64, 32 * S) || !grow(c, c->b_tp32, 16 * S) ||
      !grow(c, c->b_trm, 8 * S) || !grow(c, c->b_tmat, 4 * S) || !grow(c, c->b_tmass, 8 * n_tpl) || !grow(c, c->b_tinert, 24 * n_tpl) ||
      !grow(c, c->b_tpbound, 4 * n_tpl) || !grow(c, c->b_tmassf, 8 * n_tpl) ||
      !grow(c, c->b_tinertf, 24 * n_tpl))
    return fail(c, DEM_ERR_OOM, "template tables");
  cudaMemcpyAsync(c->b_tpl_off.p, off, 4 * (n_tpl + 1), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tp64.p, tp64.data(), 32 * (size_t)S, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tp32.p, tp32.data(), 16 * (size_t)S, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tmat.p, material, 4 * (size_t)S, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_trm.p, trm.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tmass.p, mass, 8 * (size_t)n_tpl, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tinert.p, inertia, 24 * (size_t)n_tpl, cudaMemcpyHostToDevice, c->st);
  // float tables of the FP32_VOXEL update: {m, 1/m} and {I0, I1, I2, 1/I0, 1/I1, 1/I2}
  std::vector<float> mf(2 * n_tpl), inf(6 * n_tpl);
  for (int t = 0; t < n_tpl; ++t) {
    mf[2 * t] = (float)mass[t];
    mf[2 * t + 1] = (float)(1.0 / mass[t]);
    for (int k = 0; k < 3; ++k) {
      inf[6 * t + k] = (float)inertia[3 * t + k];
      inf[6 * t + 3 + k] = (float)(1.0 / inertia[3 * t + k]);
    }
  }
  cudaMemcpyAsync(c->b_tmassf.p, mf.data(), 8 * (size_t)n_tpl, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tinertf.p, inf.data(), 24 * (size_t)n_tpl, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(c->b_tpbound.p, pb.data(), 4 * (size_t)n_tpl, cudaMemcpyHostToDevice, c->st);
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "load templates");
}

int dem_add_scene(dem_ctx* c, const double lo[3], const double hi[3], double bin_size, int* scene_id) {
  if (!c || !lo || !hi) return DEM_ERR_INVALID_ARG;
  if (c->finalized) return fail(c, DEM_ERR_STATE, "scenes must be added before the first step");
  for (int k = 0; k < 3; ++k)
    if (!(hi[k] > lo[k])) return fail(c, DEM_ERR_INVALID_ARG, "empty scene domain");
  if (!(bin_size >= 0)) return fail(c, DEM_ERR_INVALID_ARG, "negative bin size");
  SceneH s{};
  for (int k = 0; k < 3; ++k) { s.lo[k] = lo[k]; s.hi[k] = hi[k]; }
  s.bin = bin_size;
  c->scenes.push_back(s);
  if (scene_id) *scene_id = (int)c->scenes.size() - 1;
  return DEM_OK;
}

int dem_add_clumps(dem_ctx* c, int n, const int* tpl, const double* pos, const double* quat,
                   const double* vel, const double* angvel, int scene) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (c->n_tpl == 0) return fail(c, DEM_ERR_STATE, "load templates first");
  if (n < 0 || (n > 0 && (!tpl || !pos || !quat || !vel || !angvel)))
    return fail(c, DEM_ERR_INVALID_ARG, "clump arrays missing");
  if (scene < 0 || scene >= (int)c->scenes.size()) return fail(c, DEM_ERR_INVALID_ARG, "unknown scene");
  if (n == 0) return DEM_OK;
  for (int i = 0; i < n; ++i)
    if (tpl[i] < 0 || tpl[i] >= c->n_tpl) return fail(c, DEM_ERR_INVALID_ARG, "template id out of range");
  if (!finite_all(pos, 3ll * n) || !finite_all(quat, 4ll * n) || !finite_all(vel, 3ll * n) ||
      !finite_all(angvel, 3ll * n))
    return fail(c, DEM_ERR_NONFINITE, "non-finite clump state");
  long long add_s = 0;
  for (int i = 0; i < n; ++i) add_s += c->tpl_off[tpl[i] + 1] - c->tpl_off[tpl[i]];
  const long long ncl = c->ncl + n, ns = c->ns + add_s;
  // sphere ids share a 32-bit word with the history flag (bit 31)
  if (ns >= (1ll << 31) - 1) return fail(c, DEM_ERR_INVALID_ARG, "2^31 - 1 spheres or more");
  const size_t k0 = (size_t)c->ncl, s0 = (size_t)c->ns;
  bool ok = grow(c, c->b_cinfo, 8 * ncl, 8 * k0) && grow(c, c->b_csph, 4 * (ncl + 1), 4 * k0) &&
            grow(c, c->b_cq, 32 * ncl, 32 * k0) && grow(c, c->b_cvw, 48 * ncl, 48 * k0) &&
            grow(c, c->b_ref_q, 16 * ncl) &&
            grow(c, c->b_alast, 4 * ncl, 4 * k0) &&
            grow(c, c->b_sinfo, 8 * ns, 8 * s0);
  if (c->P.precision == DEM_FP64) {
    ok = ok && grow(c, c->b_cpos, 32 * ncl, 32 * k0) && grow(c, c->b_mv64, 32 * ncl) &&
         grow(c, c->b_mw64, 32 * ncl) && grow(c, c->b_acc64, 64 * ncl) && grow(c, c->b_ref_pos, 32 * ncl) &&
         grow(c, c->b_sa64, sizeof(SphA64) * ns) && grow(c, c->b_sb64, 32 * ns);
  } else {
    ok = ok && grow(c, c->b_cvox, 16 * ncl, 16 * k0) && grow(c, c->b_coff, 16 * ncl, 16 * k0) &&
         grow(c, c->b_mv32, 16 * ncl) && grow(c, c->b_mw32, 16 * ncl) && grow(c, c->b_acc32, 32 * ncl) &&
         grow(c, c->b_ref_vox, 16 * ncl) && grow(c, c->b_ref_off, 16 * ncl) &&
         grow(c, c->b_srec32, 16 * ns);
  }
  if (!ok) return fail(c, DEM_ERR_OOM, "clump buffers");
  std::vector<int2> ci(n), si(add_s);
  std::vector<int> cs(n + 1);
  long long s = c->ns;
  for (int i = 0; i < n; ++i) {
    ci[i] = make_int2(tpl[i], scene);
    cs[i] = (int)s;
    for (int j = c->tpl_off[tpl[i]]; j < c->tpl_off[tpl[i] + 1]; ++j, ++s)
      si[s - c->ns] = make_int2((int)(c->ncl + i), j);
  }
  cs[n] = (int)s;
  cudaMemcpyAsync(ptr<int2>(c->b_cinfo) + k0, ci.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(ptr<int>(c->b_csph) + k0, cs.data(), 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(ptr<int2>(c->b_sinfo) + s0, si.data(), 8 * (size_t)add_s, cudaMemcpyHostToDevice, c->st);
  for (int i = 0; i < n; ++i) {
    c->h_ctpl.push_back(tpl[i]);
    c->h_cscene.push_back(scene);
  }
  const long long first = c->ncl;
  c->ncl = ncl;
  c->ns = ns;
  int rc = upload_clumps(c, first, n, tpl, pos, quat, vel, angvel);
  if (rc) return rc;
  c->stats.n_clumps = ncl;
  c->stats.n_spheres = ns;
  {
    double rs = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = c->tpl_off[tpl[i]]; j < c->tpl_off[tpl[i] + 1]; ++j) rs += c->tpl_rad[j];
    c->r_sum += rs;
    c->r_mean = c->r_sum / (double)ns;
  }
  c->need_rebuild = true;
  if ((rc = invalidate_outer(c))) return rc;
  c->acc_dirty = true;
  if (c->finalized) {
    refresh_devstate(c);
    launch_update(c->D, false, c->step, c->margin, false, c->st);
    cudaStreamSynchronize(c->st);
  }
  return cuda_check(c, "add clumps");
}

int dem_step(dem_ctx* c, int n_steps) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (n_steps < 0) return fail(c, DEM_ERR_INVALID_ARG, "negative step count");
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  const long long launches0 = g_kernel_launches;
  StepRunner R(c, n_steps);
  if ((rc = R.init())) return rc;
  if (!c->mlp && c->P.guard != DEM_GUARD_ROLLBACK) {
    // plain rule: rebuild every rebuild_interval steps with the fixed margin
    rc = R.run_plain(n_steps, c->margin, std::max(1, c->P.rebuild_interval), true);
  } else {
    rc = R.run_guarded(n_steps);
  }
  if (rc) return rc;
  if (c->async_state == 1 && (rc = outer_async_finish(c))) return rc;
  if (c->st2) cudaStreamSynchronize(c->st2);
  c->stats.time = (double)c->step * c->P.dt;
  rc = read_flags(c);
  R.finish();
  c->stats.launches += g_kernel_launches - launches0;
  return rc;
}

int dem_get_state(dem_ctx* c, double* pos, double* quat, double* vel, double* angvel, int on_device) {
  if (!c) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  if (c->ncl == 0) return DEM_OK;
  if (on_device) {
    launch_get_state(c->D, pos, quat, vel, angvel, c->st);
    cudaStreamSynchronize(c->st);
    return cuda_check(c, "get_state");
  }
  const size_t n = (size_t)c->ncl;
  if (!grow(c, c->b_tmp, 8 * 13 * n)) return fail(c, DEM_ERR_OOM, "staging");
  double* t = ptr<double>(c->b_tmp);
  launch_get_state(c->D, t, t + 3 * n, t + 7 * n, t + 10 * n, c->st);
  if (pos) cudaMemcpyAsync(pos, t, 24 * n, cudaMemcpyDeviceToHost, c->st);
  if (quat) cudaMemcpyAsync(quat, t + 3 * n, 32 * n, cudaMemcpyDeviceToHost, c->st);
  if (vel) cudaMemcpyAsync(vel, t + 7 * n, 24 * n, cudaMemcpyDeviceToHost, c->st);
  if (angvel) cudaMemcpyAsync(angvel, t + 10 * n, 24 * n, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "get_state");
}

int dem_set_state(dem_ctx* c, const double* pos, const double* quat, const double* vel, const double* angvel) {
  if (!c || !pos || !quat || !vel || !angvel) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  const long long n = c->ncl;
  if (!c->finalized) {
    // before the first step the scene grids do not exist yet: convert on the host
    if (!finite_all(pos, 3 * n) || !finite_all(quat, 4 * n) || !finite_all(vel, 3 * n) ||
        !finite_all(angvel, 3 * n))
      return fail(c, DEM_ERR_NONFINITE, "non-finite clump state");
    int rc = upload_clumps(c, 0, (int)n, c->h_ctpl.data(), pos, quat, vel, angvel);
    if (rc) return rc;
    c->need_rebuild = true;
    c->acc_dirty = true;
    return DEM_OK;
  }
  if (n == 0) return DEM_OK;
  // stage the arrays as given (one copy each), validate and convert on the
  // device; a rejected state leaves the clump records untouched
  const size_t un = (size_t)n;
  if (!grow(c, c->b_tmp, 8 * 13 * un + 16)) return fail(c, DEM_ERR_OOM, "staging");
  double* t = ptr<double>(c->b_tmp);
  int* err = reinterpret_cast<int*>(t + 13 * un);
  cudaMemcpyAsync(t, pos, 24 * un, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(t + 3 * un, quat, 32 * un, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(t + 7 * un, vel, 24 * un, cudaMemcpyHostToDevice, c->st);
  cudaMemcpyAsync(t + 10 * un, angvel, 24 * un, cudaMemcpyHostToDevice, c->st);
  cudaMemsetAsync(err, 0, sizeof(int), c->st);
  refresh_devstate(c);
  launch_check_state(c->D, t, err, c->st);
  int bad = 0;
  cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  int rc = cuda_check(c, "set_state");
  if (rc) return rc;
  if (bad & 1) return fail(c, DEM_ERR_NONFINITE, "non-finite clump state");
  if (bad & 2) return fail(c, DEM_ERR_INVALID_ARG, "clump too far from its scene corner");
  launch_set_state(c->D, t, c->st);
  c->need_rebuild = true;
  c->acc_dirty = true;
  launch_update(c->D, false, c->step, c->margin, false, c->st);
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "set_state");
}

int dem_get_stats(dem_ctx* c, dem_stats* out) {
  if (!c || !out) return DEM_ERR_INVALID_ARG;
  *out = c->stats;
  out->n_clumps = c->ncl;
  out->n_spheres = c->ns;
  if (c->have_list) {
    out->n_pairs = curL(c).n;
    out->n_wall_contacts = curL(c).nw;
  }
  out->margin = c->finalized ? c->margin : current_margin(c);
  out->time = (double)c->step * c->P.dt;
  return DEM_OK;
}

int dem_reset_stats(dem_ctx* c) {
  if (!c) return DEM_ERR_INVALID_ARG;
  c->stats = dem_stats{};
  return DEM_OK;
}

int dem_set_timing(dem_ctx* c, int timing) {
  if (!c) return DEM_ERR_INVALID_ARG;
  c->timing = timing ? 1 : 0;
  if (c->timing) {
    // the per-step event pool is created here, not inside a timed dem_step
    // (creating thousands of events there leaves the device idle meanwhile)
    cudaSetDevice(c->P.device);
    StepRunner R(c, 0);
    return R.init();
  }
  return DEM_OK;
}

int dem_rebuild(dem_ctx* c) {
  if (!c) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  rc = rebuild(c);
  if (rc) return rc;
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "rebuild");
}

int dem_eval_forces(dem_ctx* c) {
  if (!c) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  if (c->need_rebuild || !c->have_list) {
    rc = rebuild(c);
    if (rc) return rc;
  }
  force_pass(c, true);
  c->acc_dirty = true;
  return read_flags(c);
}

int dem_get_forces(dem_ctx* c, double* F, double* T) {
  if (!c || !F || !T) return DEM_ERR_INVALID_ARG;
  const size_t n = (size_t)c->ncl;
  if (n == 0) return DEM_OK;
  if (!grow(c, c->b_tmp, 48 * n)) return fail(c, DEM_ERR_OOM, "staging");
  double* t = ptr<double>(c->b_tmp);
  launch_get_forces(c->D, t, t + 3 * n, c->st);
  cudaMemcpyAsync(F, t, 24 * n, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(T, t + 3 * n, 24 * n, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  return cuda_check(c, "get_forces");
}

int dem_get_wall_forces(dem_ctx* c, double* F) {
  if (!c || !F) return DEM_ERR_INVALID_ARG;
  const size_t nu = c->user_walls.size();
  std::fill(F, F + 3 * nu, 0.0);
  if (c->walls.empty()) return DEM_OK;
  std::vector<double> h(3 * c->walls.size());
  cudaMemcpyAsync(h.data(), c->b_wforce.p, 24 * c->walls.size(), cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  for (size_t w = 0; w < c->walls.size(); ++w)
    for (int k = 0; k < 3; ++k) F[3 * c->wall_user[w] + k] += h[3 * w + k];
  return cuda_check(c, "get_wall_forces");
}

int dem_get_wall_loads(dem_ctx* c, double* F, double* T) {
  if (!c || !F || !T) return DEM_ERR_INVALID_ARG;
  const size_t nu = c->user_walls.size();
  std::fill(F, F + 3 * nu, 0.0);
  std::fill(T, T + 3 * nu, 0.0);
  if (c->walls.empty()) return DEM_OK;
  const size_t nw = c->walls.size();
  std::vector<double> hf(3 * nw), ht(3 * nw);
  cudaMemcpyAsync(hf.data(), c->b_wforce.p, 24 * nw, cudaMemcpyDeviceToHost, c->st);
  cudaMemcpyAsync(ht.data(), c->b_wtorque.p, 24 * nw, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  // the copies of a wall in several scenes share its reference point
  for (size_t w = 0; w < nw; ++w)
    for (int k = 0; k < 3; ++k) {
      F[3 * c->wall_user[w] + k] += hf[3 * w + k];
      T[3 * c->wall_user[w] + k] += ht[3 * w + k];
    }
  return cuda_check(c, "get_wall_loads");
}

int dem_set_wall_motion(dem_ctx* c, int wall, const double* point, const double* vel) {
  if (!c || !point || !vel || wall < 0 || wall >= (int)c->user_walls.size())
    return DEM_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(point[k]) || !std::isfinite(vel[k]))
      return fail(c, DEM_ERR_NONFINITE, "non-finite wall motion");
  cudaSetDevice(c->P.device);
  // a wall moves as p(t) = p + vel t: re-base it so that p(now) = point
  const double t = (double)c->step * c->P.dt;
  dem_wall& uw = c->user_walls[wall];
  for (int k = 0; k < 3; ++k) {
    uw.vel[k] = vel[k];
    const double np = point[k] - vel[k] * t;
    // a facet moves rigidly: its other vertices follow the first
    uw.b[k] += np - uw.p[k];
    uw.c[k] += np - uw.p[k];
    uw.p[k] = np;
  }
  if (!c->finalized) return DEM_OK;  // the device tables are built from user_walls
  const double speed = std::sqrt((vel[0] * vel[0] + vel[1] * vel[1]) + vel[2] * vel[2]);
  for (size_t w = 0; w < c->walls.size(); ++w) {
    if (c->wall_user[w] != wall) continue;
    WallDev& d = c->walls[w];
    for (int k = 0; k < 3; ++k) {
      d.p[k] = uw.p[k];
      d.vel[k] = uw.vel[k];
      d.pf[k] = (float)uw.p[k];
      d.vf[k] = (float)uw.vel[k];
    }
    d.speed_d = speed;
    d.speed = (float)speed;
  }
  cudaMemcpyAsync(c->b_walls.p, c->walls.data(), sizeof(WallDev) * c->walls.size(),
                  cudaMemcpyHostToDevice, c->st);
  refresh_devstate(c);
  launch_walls_at(c->D, c->step, c->st);  // wall positions of the current step
  // the listed wall candidates assumed the old motion
  c->need_rebuild = true;
  int rc = invalidate_outer(c);
  drop_graphs(c);
  cudaStreamSynchronize(c->st);  // the host table must outlive its copy
  if (rc) return rc;
  return cuda_check(c, "set_wall_motion");
}

int dem_num_contacts(dem_ctx* c, long long* n_pairs, long long* n_wall) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (n_pairs) *n_pairs = c->have_list ? curL(c).n : 0;
  if (n_wall) *n_wall = c->have_list ? curL(c).nw : 0;
  return DEM_OK;
}

int dem_get_contacts(dem_ctx* c, int* a, int* b, double* u, int* wall_sphere, int* wall_id, double* wall_u) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (!c->have_list) return DEM_OK;
  ContactList& L = curL(c);
  std::vector<uint32_t> pb(L.n), ww(L.nw);
  std::vector<double> uu(3 * L.cap), uw(3 * L.capw);
  if (a && L.n) cudaMemcpyAsync(a, L.pa, 4 * L.n, cudaMemcpyDeviceToHost, c->st);
  if (L.n) cudaMemcpyAsync(pb.data(), L.pb, 4 * L.n, cudaMemcpyDeviceToHost, c->st);
  if (u && L.n) cudaMemcpyAsync(uu.data(), L.u, 24 * L.cap, cudaMemcpyDeviceToHost, c->st);
  if (wall_sphere && L.nw) cudaMemcpyAsync(wall_sphere, L.ws, 4 * L.nw, cudaMemcpyDeviceToHost, c->st);
  if (L.nw) cudaMemcpyAsync(ww.data(), L.ww, 4 * L.nw, cudaMemcpyDeviceToHost, c->st);
  if (wall_u && L.nw) cudaMemcpyAsync(uw.data(), L.uw, 24 * L.capw, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  // FP32_VOXEL keeps each pair history component as a float-float {high,
  // low} in its 8-byte slot; FP64 as a double
  const bool ffh = c->P.precision != DEM_FP64;
  for (long long i = 0; i < L.n; ++i) {
    if (b) b[i] = (int)(pb[i] & ~kHistFlag);
    if (u)
      for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        if (pb[i] & kHistFlag) {
          v = uu[k * L.cap + i];
          if (ffh) {
            float hl[2];
            std::memcpy(hl, &uu[k * L.cap + i], sizeof hl);
            v = (double)hl[0] + (double)hl[1];
          }
        }
        u[3 * i + k] = v;
      }
  }
  for (long long i = 0; i < L.nw; ++i) {
    if (wall_id) wall_id[i] = c->wall_user[ww[i] & ~kHistFlag];
    if (wall_u)
      for (int k = 0; k < 3; ++k) wall_u[3 * i + k] = (ww[i] & kHistFlag) ? uw[k * L.capw + i] : 0.0;
  }
  return cuda_check(c, "get_contacts");
}

int dem_get_bins(dem_ctx* c, long long cap, unsigned int* keys, int* ids, long long* n) {
  if (!c || !n) return DEM_ERR_INVALID_ARG;
  *n = c->n_entries;
  const long long m = std::min(cap, c->n_entries);
  if (m > 0 && keys && ids && c->ds[0].rec.p) {
    // the device holds the records grouped by bin in slot order: restore
    // the bin key of every entry and sort each bin by sphere id
    const long long B = c->n_entries, nb = c->n_entry_bins;
    if (!grow(c, c->b_tmp, 4 * (size_t)B)) return fail(c, DEM_ERR_OOM, "staging");
    launch_rec_ids(ptr<EntryRec>(c->ds[0].rec), B, ptr<uint32_t>(c->b_tmp), c->st);
    std::vector<uint32_t> start((size_t)nb + 1), v((size_t)B);
    cudaMemcpyAsync(start.data(), c->ds[0].bin_start.p, 4 * (size_t)(nb + 1), cudaMemcpyDeviceToHost, c->st);
    cudaMemcpyAsync(v.data(), c->b_tmp.p, 4 * (size_t)B, cudaMemcpyDeviceToHost, c->st);
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return cuda_check(c, "get_bins");
    for (long long k = 0; k < nb; ++k) {
      const uint32_t s0 = start[k], s1 = start[k + 1];
      std::sort(v.begin() + s0, v.begin() + s1);
      for (uint32_t i = s0; i < s1 && (long long)i < m; ++i) {
        keys[i] = (unsigned int)k;
        ids[i] = (int)v[i];
      }
    }
  }
  return cuda_check(c, "get_bins");
}


int dem_autotune_bins(dem_ctx* c, int n, const double* factors, int reps, double* best,
                      double* ms_out) {
  if (!c || n < 1 || !factors || reps < 1 || !best) return DEM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!(factors[i] > 0.0) || !std::isfinite(factors[i]))
      return fail(c, DEM_ERR_INVALID_ARG, "bin factors must be finite and > 0");
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  const dem_stats saved = c->stats;
  const double f0 = c->bin_factor;
  auto apply = [&](double f) -> int {
    c->bin_factor = f;
    int r = build_grids(c);
    if (r) return r;
    cudaMemcpyAsync(c->b_grids.p, c->grids.data(), sizeof(SceneGrid) * c->grids.size(),
                    cudaMemcpyHostToDevice, c->st);
    return rebuild(c);  // also sizes the buffers for this grid
  };
  double best_ms = 0.0;
  int best_i = -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int i = 0; i < n; ++i) {
    double ms = -1.0;
    if (apply(factors[i]) == DEM_OK) {
      cudaEventRecord(e0, c->st);
      for (int r = 0; r < reps && rc == DEM_OK; ++r) rc = rebuild(c);
      cudaEventRecord(e1, c->st);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rc) break;
      ms = (double)t / reps;
      if (best_i < 0 || ms < best_ms) {
        best_ms = ms;
        best_i = i;
      }
    }
    if (ms_out) ms_out[i] = ms;  // -1: this factor gives no valid grid
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double chosen = best_i >= 0 ? factors[best_i] : f0;
  c->err.clear();
  if ((rc = apply(chosen))) return rc;
  // the trial rebuilds change no state; only the counters are restored
  c->stats.rebuilds = saved.rebuilds;
  c->stats.ms_detect = saved.ms_detect;
  *best = chosen;
  return cuda_check(c, "autotune");
}

int dem_set_tiles(dem_ctx* c, const dem_tiles* t) {
  if (!c || !t) return DEM_ERR_INVALID_ARG;
  if (t->pairs_blocks_per_sm < 1 || t->pairs_blocks_per_sm > 32 ||
      (t->update_block != 64 && t->update_block != 128 && t->update_block != 256) ||
      t->narrow_chunk < 1 || t->narrow_chunk > 64)
    return fail(c, DEM_ERR_INVALID_ARG, "launch shapes out of range");
  c->tiles = *t;
  drop_graphs(c);  // captured graphs hold the old launch shapes
  refresh_devstate(c);
  return DEM_OK;
}

int dem_get_tiles(dem_ctx* c, dem_tiles* t) {
  if (!c || !t) return DEM_ERR_INVALID_ARG;
  *t = c->tiles;
  return DEM_OK;
}

int dem_autotune_tiles(dem_ctx* c, int steps, int reps, dem_tiles* best) {
  if (!c || steps < 1 || reps < 1 || !best) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  const dem_stats saved = c->stats;
  const float* cm = c->D.cmargin;
  c->D.cmargin = nullptr;
  StepRunner R(c, 0);
  if ((rc = R.init())) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto elapsed = [&]() -> double {
    cudaEventRecord(e1, c->st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    return (double)t;
  };
  // the narrow-phase chunk, timed on rebuilds (which change no state)
  const int chunks[] = {2, 4, 8, 16, 32};
  double best_ms = -1.0;
  dem_tiles cur = c->tiles;
  for (int ch : chunks) {
    c->tiles.narrow_chunk = ch;
    if ((rc = rebuild(c))) break;  // sizes the buffers
    cudaEventRecord(e0, c->st);
    for (int r = 0; r < reps && rc == DEM_OK; ++r) rc = rebuild(c);
    const double ms = elapsed() / reps;
    if (rc) break;
    if (best_ms < 0.0 || ms < best_ms) { best_ms = ms; cur.narrow_chunk = ch; }
  }
  c->tiles = cur;
  // the step kernels, timed on `steps` steps from a snapshot taken at a fresh
  // list; the snapshot is restored before every trial and at the end
  if (rc == DEM_OK && (rc = rebuild(c)) == DEM_OK && (rc = take_snapshot(c)) == DEM_OK) {
    auto time_steps = [&](const dem_tiles& t) -> double {
      c->tiles = t;
      refresh_devstate(c);
      if (restore_snapshot(c)) return -1.0;
      c->since = 0;
      R.step(c->margin, false, false);  // warm-up
      cudaEventRecord(e0, c->st);
      for (int i = 0; i < steps; ++i) R.step(c->margin, false, false);
      return elapsed() / steps;
    };
    const int bpsm[] = {2, 4, 8, 16};
    const int upd[] = {64, 128, 256};
    best_ms = -1.0;
    dem_tiles pick = cur;
    for (int b : bpsm) {
      dem_tiles t = pick;
      t.pairs_blocks_per_sm = b;
      const double ms = time_steps(t);
      if (ms >= 0.0 && (best_ms < 0.0 || ms < best_ms)) { best_ms = ms; pick = t; }
    }
    best_ms = -1.0;
    const dem_tiles base = pick;
    for (int u : upd) {
      dem_tiles t = base;
      t.update_block = u;
      const double ms = time_steps(t);
      if (ms >= 0.0 && (best_ms < 0.0 || ms < best_ms)) { best_ms = ms; pick = t; }
    }
    c->tiles = pick;
    refresh_devstate(c);
    rc = restore_snapshot(c);
    c->since = 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->D.cmargin = cm;
  drop_graphs(c);
  // trial steps and rebuilds leave no trace in the counters
  c->stats = saved;
  if (rc) return rc;
  *best = c->tiles;
  return cuda_check(c, "autotune tiles");
}

int dem_set_outer_list(dem_ctx* c, double factor, int n_inner, int async_detect) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (n_inner < 0 || (n_inner > 0 && !(factor > 1.0 && std::isfinite(factor))))
    return fail(c, DEM_ERR_INVALID_ARG, "outer list: factor must be > 1 and n_inner >= 0");
  if (async_detect && c->P.alloc)
    return fail(c, DEM_ERR_INVALID_ARG,
                "outer list on a second stream: needs the library's stream-ordered allocator");
  cudaSetDevice(c->P.device);
  int rc = outer_async_drop(c);
  if (rc) return rc;
  c->outer_factor = factor;
  c->outer_n = n_inner;
  c->outer_async = async_detect != 0;
  c->outer_valid = false;
  return DEM_OK;
}

int dem_set_deterministic(dem_ctx* c, int on) {
  if (!c) return DEM_ERR_INVALID_ARG;
  c->det = on ? 1 : 0;
  c->det_ready = false;
  c->need_rebuild = true;  // the slot lists are built with the next list
  drop_graphs(c);
  refresh_devstate(c);
  return DEM_OK;
}

int dem_set_graphs(dem_ctx* c, int enabled) {
  if (!c) return DEM_ERR_INVALID_ARG;
  c->use_graphs = enabled ? 1 : 0;
  return DEM_OK;
}

int dem_set_learned_policy(dem_ctx* c, dem_mlp* mlp, const dem_learned_params* lp) {
  if (!c) return DEM_ERR_INVALID_ARG;
  if (!mlp) {
    c->mlp = nullptr;
    return DEM_OK;
  }
  if (!lp || lp->interval < 1 || !(lp->safety > 0) || lp->n_candidates < 1 || !lp->candidates)
    return fail(c, DEM_ERR_INVALID_ARG, "learned policy parameters");
  for (int j = 0; j < lp->n_candidates; ++j) {
    if (!(lp->candidates[j] > 0) || !(c->r_max + lp->candidates[j] < 32.0))
      return fail(c, DEM_ERR_INVALID_ARG, "candidate margins must be > 0 and below 32 m minus the largest radius");
    if (j && !(lp->candidates[j] > lp->candidates[j - 1]))
      return fail(c, DEM_ERR_INVALID_ARG, "candidate margins must ascend");
  }
  if (c->P.guard == DEM_GUARD_OFF) return fail(c, DEM_ERR_STATE, "the learned rule needs the guard");
  c->mlp = mlp;
  if (lp->mode != DEM_LEARNED_HALT && lp->mode != DEM_LEARNED_ROLLBACK)
    return fail(c, DEM_ERR_INVALID_ARG, "learned policy mode");
  if (!(lp->speed_floor >= 0.0) || !std::isfinite(lp->speed_floor))
    return fail(c, DEM_ERR_INVALID_ARG, "learned policy speed floor must be finite and >= 0");
  c->l_interval = lp->interval;
  c->l_safety = lp->safety;
  c->l_mode = lp->mode;
  c->l_floor = lp->speed_floor;
  c->l_cand.assign(lp->candidates, lp->candidates + lp->n_candidates);
  c->need_rebuild = true;
  return DEM_OK;
}

int dem_trace(dem_ctx* c, int windows, int window, int n_candidates, const double* candidates,
              long long cap, float* x, float* t, long long* n_out) {
  if (!c || windows < 0 || window < 1 || n_candidates < 1 || !candidates || cap < 0 ||
      (cap > 0 && (!x || !t)) || !n_out)
    return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  dem_mlp* saved = c->mlp;
  std::vector<double> saved_cand = c->l_cand;
  c->mlp = nullptr;  // features only
  c->l_cand.assign(candidates, candidates + n_candidates);
  const int nc = n_candidates;
  const long long ncl = c->ncl;
  long long total = 0;
  const size_t capb = (size_t)std::max<long long>(cap, 1);
  if (!grow(c, c->b_tx, 4 * capb * kMlpIn) || !grow(c, c->b_tt, 4 * capb) ||
      !grow(c, c->b_tr_q, 16 * (ncl + 1)) || !grow(c, c->b_tr_vox, 16 * (ncl + 1)) ||
      !grow(c, c->b_tr_off, 16 * (ncl + 1)) || !grow(c, c->b_tr_pos, 32 * (ncl + 1)) ||
      !grow(c, c->b_dmax, 4 * ((size_t)c->n_lbins + 1))) {
    c->mlp = saved;
    c->l_cand = saved_cand;
    return fail(c, DEM_ERR_OOM, "trace buffers");
  }
  cudaMemsetAsync(c->b_dmax.p, 0, 4 * (size_t)c->n_lbins, c->st);
  TraceRef tr{ptr<int4>(c->b_tr_vox), ptr<float4>(c->b_tr_off), ptr<double4_32a>(c->b_tr_pos),
              ptr<float4>(c->b_tr_q)};
  StepRunner R(c, windows * window);
  if ((rc = R.init())) goto done;
  for (int w = 0; w < windows; ++w) {
    if ((rc = predict_margins(c))) goto done;
    {
      const long long rows = c->n_occ * nc;
      if (!grow(c, c->b_T, 4 * (size_t)(rows + 1))) { rc = fail(c, DEM_ERR_OOM, "trace labels"); goto done; }
      cudaMemsetAsync(c->b_T.p, 0, 4 * (size_t)rows, c->st);
      launch_trace_ref(c->D, tr, c->st);
      for (int s = 1; s <= window; ++s) {
        if ((rc = R.run_plain(1, c->margin, std::max(1, c->P.rebuild_interval), false))) goto done;
        launch_trace_step(c->D, tr, ptr<uint32_t>(c->b_chome), ptr<int>(c->b_dmax),
                          ptr<uint32_t>(c->b_occ), c->n_occ, nc, ptr<float>(c->b_cand),
                          ptr<int>(c->b_T), s, c->st);
      }
      launch_trace_emit(rows, ptr<float>(c->b_feat), ptr<int>(c->b_T), window, ptr<float>(c->b_tx),
                        ptr<float>(c->b_tt), total, cap, c->st);
      total += rows;
    }
  }
  if ((rc = read_flags(c))) goto done;
  {
    const long long n = std::min(total, cap);
    if (n > 0) {
      cudaMemcpyAsync(x, c->b_tx.p, 4 * (size_t)n * kMlpIn, cudaMemcpyDeviceToHost, c->st);
      cudaMemcpyAsync(t, c->b_tt.p, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->st);
      cudaStreamSynchronize(c->st);
    }
    *n_out = n;
  }
  R.finish();
done:
  c->mlp = saved;
  c->l_cand = saved_cand;
  c->stats.time = (double)c->step * c->P.dt;
  return rc ? rc : cuda_check(c, "trace");
}

int dem_audit(dem_ctx* c, long long* missed) {
  if (!c || !missed) return DEM_ERR_INVALID_ARG;
  cudaSetDevice(c->P.device);
  int rc = finalize(c);
  if (rc) return rc;
  refresh_devstate(c);
  if (!c->have_list) {
    rc = rebuild(c);
    if (rc) return rc;
  }
  return audit_now(c, missed);
}

}  // extern "C"

namespace {
// Touching contacts of the current state missing from the current list: a
// fresh detection with zero margin into the spare list, compared with it.
int audit_now(dem_ctx* c, long long* missed) {
  int rc;
  const float* saved_cm = c->D.cmargin;
  c->D.cmargin = nullptr;  // the exact check uses no margin
  rc = detect_into(c, 2, 0.0, 1);
  c->D.cmargin = saved_cm;
  if (rc) return rc;
  const ContactList& F = c->lists[2].L;
  unsigned long long* d_m = ptr<unsigned long long>(c->ds[0].totals) + 4;
  cudaMemsetAsync(d_m, 0, 8, c->st);
  DetectOut o{};
  launch_audit(c->D, o, curL(c), F.n, F.pa, F.pb, F.nw, F.ws, F.ww, (double)c->step * c->P.dt, d_m, c->st);
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, d_m, 8, cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  *missed = (long long)h;
  c->stats.missed_contacts += (long long)h;
  return cuda_check(c, "audit");
}
}  // namespace
