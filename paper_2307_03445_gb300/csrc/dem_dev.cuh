// dem_dev.cuh -- device view of a context and the kernel launchers.
#pragma once
#include "dem_internal.cuh"

namespace dem {

// Pointers into the context's device buffers, passed by value to kernels.
struct DevState {
  int prec;                 // 0 FP64, 1 FP32_VOXEL
  long long ncl, ns;
  int nmat, nwalls;
  double h, g[3];
  double hg[3];             // h * g
  float hgf[3];             // h * g as float
  float hf;                 // h as float
  // templates
  const int* tpl_off;
  const double4_32a* tp64;      // per template sphere: p (FP64), r
  const float4* tp32;       // per template sphere: p, r (float)
  const int* tmat;          // per template sphere: material
  const float2* trm;        // per template sphere: {radius (float), material (int bits)}
  const double* tmass;      // per template
  const double* tinert;     // per template, 3 principal moments
  const float* tmassf;      // per template {mass, 1 / mass} (float)
  const float* tinertf;     // per template {I0, I1, I2, 1/I0, 1/I1, 1/I2} (float)
  const float* tpbound;     // per template: max |p| over its spheres
  // clumps
  const int2* cinfo;        // {template, scene}
  const int* csph;          // first sphere of each clump (ncl + 1)
  double4_32a* cpos;            // FP64: centre of mass
  int4* cvox;               // FP32_VOXEL: voxel index (w unused)
  float4* coff;             // FP32_VOXEL: offset in the voxel (w unused)
  double4_32a* cq;              // orientation (both modes)
  VelRec* cvw;              // velocity and body-frame angular velocity (both modes)
  double4_32a* mv64;            // FP64 mirrors for contacts: {v, mass}
  double4_32a* mw64;            //                            {omega world, 0}
  float4* mv32;             // FP32 mirrors: {v, mass}
  float4* mw32;             //               {omega world, 0}
  double* acc64;            // 8 per clump: F, T (FP64)
  float* acc32;             // 8 per clump: F, T (FP32)
  // certificate reference (state at the last rebuild)
  double4_32a* ref_pos;         // FP64: CoM at the last rebuild
  int4* ref_vox;            // FP32_VOXEL: voxel / offset at the last rebuild
  float4* ref_off;
  float4* ref_q;            // orientation at the last rebuild (float)
  const float* cmargin;     // per clump margin for the certificate (or NULL)
  float* alast;             // per clump |F|/m of the last step (or NULL)
  // spheres
  const int2* sinfo;        // {owner, template sphere}
  SphA64* sa64;
  double4_32a* sb64;            // {rel = R p, bits(owner | mat << 32)}
  uint4* srec32;            // FP32_VOXEL pose record (pack_rel: centre from the voxel corner)
  // scenes, walls, materials
  const SceneGrid* grids;
  const WallDev* walls;
  const int* wall_idx;      // per scene wall lists (global wall ids)
  const int* wall_scene;    // scene of each (internal) wall
  const int* facet_idx;     // the mesh facets (wall ids), registered in the bins at a rebuild
  int nfacets;
  long long* wfix;          // FP32_VOXEL: wall reference point at the current time, fixed point
                            //   relative to its scene corner (3 per wall)
  double* wpos;             // wall reference point in world coordinates at the current time (3 per wall)
  double* wforce;           // 3 per wall (FP64 accumulation)
  double* wtorque;          // 3 per wall: moment of those forces about the wall's
                            //   reference point at the current time
  const PairMat<double>* pm64;
  const PairMat<float>* pm32;
  int* flags;
  unsigned long long* counters;  // [0] active contacts, [1] guard violations
  long long* dstep;         // device step counter: forces of step s see time s * h
  // deterministic reduction (det_off NULL: vector reductions straight into
  // the accumulators).  Each contact writes its force and moments to its own
  // slot; a per-clump pass adds the slots of the clump in a fixed order.
  float4* det_pair32;       // 3 per listed pair: F on b, moment on a, moment on b
  float4* det_wall32;       // 2 per wall contact: F on the clump, its moment
  double4_32a* det_pair64;  // FP64 mode, same layout
  double4_32a* det_wall64;
  const uint32_t* det_off;  // per clump: start of its slot ids (ncl + 1)
  const uint32_t* det_ids;  // slot ids: 2k pair k side a, 2k + 1 side b, 2n + j wall contact j
  long long* halt_at;       // learned rule, halt mode: the first step whose state failed
                            //   the displacement certificate (LLONG_MAX: none); every
                            //   per-step kernel of a later step returns at once.  NULL: off
  // launch shapes (read by the host launchers; chosen by dem_autotune_tiles)
  int pairs_bpsm;           // blocks of 256 threads per SM for the pair force kernels
  int upd_block;            // clumps per block of the FP32_VOXEL update kernel: 64, 128, 256
};

// Fixed-point centre (2^-44 m from the scene corner) of sphere s, owned by
// clump c (FP32_VOXEL): the clump's voxel corner plus the pose record.
__device__ __forceinline__ void sphere_fix(const DevState& d, long long s, int c, long long P[3]) {
  const int4 v = d.cvox[c];
  long long x, y, z;
  unpack_rel(d.srec32[s], x, y, z);
  P[0] = ((long long)v.x << (kFixBits - kVoxLog2)) + x;
  P[1] = ((long long)v.y << (kFixBits - kVoxLog2)) + y;
  P[2] = ((long long)v.z << (kFixBits - kVoxLog2)) + z;
}

// True when the kernels of the step that starts from state *d.dstep must not
// run (its state failed the certificate).  Uniform across a launch: halt_at is
// only lowered by the update kernel, to a step after the one it integrates.
__device__ __forceinline__ bool halted(const DevState& d) {
  return d.halt_at != nullptr && *d.dstep >= *d.halt_at;
}

// One bin registration, in its bin's slot, with everything the narrow phase tests:
// the lattice centre and enlarged radius, the owner clump, the sphere id and
// the owning-bin mask: bit k is set when the clamped bin of the box's lower
// corner equals this bin's coordinate on axis k.  A pair registered in a bin
// belongs to that bin iff the two masks together cover all three axes
// (floor division and clamping are monotone, so the bin of the per-axis max
// of two lower corners is the per-axis max of their lower-corner bins, and
// both of those are <= this bin's coordinates).
struct alignas(32) EntryRec {
  int qx, qy, qz, rho;
  int owner;
  uint32_t id;
  uint32_t mask;
  uint32_t pad;
};

struct DetectOut {
  EntryRec* rec;            // per entry, grouped by bin (any order inside a bin)
  int4* det;                // per sphere {qx, qy, qz, rho}
  uint32_t* wall_mask;      // per sphere
  uint32_t* wall_cnt;       // per sphere
  uint32_t* wall_off;       // per sphere (scan)
  uint32_t* bin_size;       // per bin (+1): registrations (counting pass)
  uint32_t* bin_start;      // per bin (+1): first entry; bin k is [start[k], start[k + 1])
  uint32_t nbins;
  uint2* upairs;            // narrow phase: kept pairs (a, b), unordered
  unsigned long long ucap;  //   capacity of upairs
  unsigned long long* d_np; //   pairs found (may exceed ucap)
  unsigned long long* next_bin;  // next unclaimed bin (zeroed by the caller)
  int chunk;                //   bins a warp claims at a time (a launch shape)
  long long np;             //   pairs found, on the host (write pass)
  uint32_t* pair_cnt;       // per sphere
  uint32_t* pair_off;       // per sphere (scan) -> row pointer (ns + 1 entries)
  int* trho;                // per template sphere: enlarged lattice radius, when all
                            //   clumps share one margin (else NULL: per sphere)
  int n_tsph;               // template spheres
  // mesh facets in the bins (when the scenes hold facets)
  uint32_t* fbin_size;      // per bin (+1): facet registrations (counting pass)
  uint32_t* fbin_start;     // per bin (+1): first facet registration (scan)
  uint4* frec;              // per facet registration {bin key, wall id, owning-bin mask, 0}
  long long nfreg;          //   facet registrations (host)
  uint2* fcand;             // (sphere, facet) candidates, unordered
  unsigned long long fcap;  //   capacity of fcand
  unsigned long long* d_nf; //   candidates found (may exceed fcap)
  uint32_t* fcnt;           // per sphere: facet candidates (then the slots taken)
  double wall_extra;        // added to the margin in the wall candidates' threshold
  // filtering a list from the outer list: the count pass records each outer
  // pair's decision and each sphere's wall decisions (bit j: its j-th outer
  // wall candidate, j < 32), which the emit pass then copies
  uint8_t* fkeep;           // per outer pair
  uint32_t* wkeep;          // per sphere
};

struct ContactList {
  int* pa;                  // sphere a (pairs)
  uint32_t* pb;             // sphere b | kHistFlag
  int4* pown;               // FP32_VOXEL lists the force kernel reads, written at the rebuild:
                            //   per pair {owner of a, owner of b, radius of a, of b (float bits)}
  int* ppm;                 //   and its row of the pair-material table (ma * nmat + mb)
  double* u;                // 3 * capacity (SoA: ux | uy | uz)
  uint32_t* row;            // ns + 1 row pointer by sphere a
  long long n, cap;
  int* ws;                  // wall contacts: sphere
  uint32_t* ww;             // wall id | kHistFlag
  double* uw;               // 3 * capacity (SoA)
  uint32_t* wrow;           // ns + 1
  long long nw, capw;
  long long* dn;            // device copy of {n, nw}: the per-step kernels read the
                            // lengths from here, so captured graphs stay valid
};

// detection
void launch_detect(const DevState& d, const DetectOut& o, double margin, const double* smargin,
                   double t, double travel_time, cudaStream_t st);
// Bin sort by counting: launch_detect adds every registration to o.bin_size
// (zeroed by the caller); after the exclusive scan of bin_size into
// o.bin_start (nbins + 1 entries), launch_bin_scatter writes the records
// o.rec grouped by bin and leaves bin_size at zero.
void launch_bin_scatter(const DevState& d, const DetectOut& o, cudaStream_t st);
// ids[i] = rec[i].id (inspection).
void launch_rec_ids(const EntryRec* rec, long long n, uint32_t* ids, cudaStream_t st);
// Narrow phase over the bins: the kept pairs go to o.upairs as (lower id,
// higher id) (count in *o.d_np, zeroed by the caller) and o.pair_cnt[a] +=
// partners b > a (pair_cnt zeroed by the caller).
void launch_narrow(const DevState& d, const DetectOut& o, cudaStream_t st);
// After the scan of pair_cnt into pair_off (= newl.row) with o.np set: rows
// newl.pa / newl.pb, each sorted by b (consumes pair_cnt); with an old list
// (oldl != NULL, its first old_ns spheres comparable) the tangential history
// of every pair both lists hold is carried into newl.u.
void launch_list_rows(const DevState& d, const DetectOut& o, const ContactList& newl,
                      const ContactList* oldl, long long old_ns, cudaStream_t st);
void launch_wall_emit(const DevState& d, const DetectOut& o, int* ws, uint32_t* ww,
                      cudaStream_t st);
// Mesh facets: count (into o.fbin_size, zeroed by the caller) and, after the
// scan into o.fbin_start, scatter the facets' bin registrations (o.frec);
// after the sphere bin scatter, the facet narrow phase (candidates into
// o.fcand, per-sphere counts into o.fcnt, both zeroed by the caller);
// launch_add_facet_counts adds o.fcnt into o.wall_cnt (rescanned by the
// caller into o.wall_off); after launch_wall_emit, launch_facet_finish puts
// the nf candidates into their rows and sorts those rows by wall id.
void launch_facet_count(const DevState& d, const DetectOut& o, double t, double travel_time,
                        cudaStream_t st);
void launch_facet_scatter(const DevState& d, const DetectOut& o, double t, double travel_time,
                          cudaStream_t st);
void launch_facet_narrow(const DevState& d, const DetectOut& o, double margin, const double* smargin,
                         double t, double travel_time, cudaStream_t st);
void launch_add_facet_counts(const DevState& d, const DetectOut& o, cudaStream_t st);
void launch_facet_finish(const DevState& d, const DetectOut& o, long long nf, int* ws, uint32_t* ww,
                         cudaStream_t st);
void launch_hist_walls(const ContactList& oldl, ContactList& newl, long long old_ns, cudaStream_t st);
void launch_hist_pairs(const ContactList& oldl, ContactList& newl, long long old_ns, cudaStream_t st);
// The per-pair records l.pown, l.ppm of a finished FP32_VOXEL list.
void launch_pair_owners(const DevState& d, const ContactList& l, cudaStream_t st);
// Inner list from an outer list (see dem_detect.cu): the lattice points at
// margin m into o.det, with the count of spheres past their allowance around
// q0 in *bad (zeroed by the caller); the per-sphere counts of kept pairs and
// wall candidates (o.pair_cnt, o.wall_cnt), and after their scans into
// o.pair_off / o.wall_off, the inner rows themselves.
void launch_lattice_check(const DevState& d, const DetectOut& o, double margin, const int4* q0,
                          unsigned long long* bad, cudaStream_t st);
void launch_filter_count(const DevState& d, const DetectOut& o, const ContactList& outer,
                         double margin, double t, double travel_time, cudaStream_t st);
void launch_filter_emit(const DevState& d, const DetectOut& o, const ContactList& outer,
                        const ContactList& inner, double margin, double t, double travel_time,
                        cudaStream_t st);
void launch_audit(const DevState& d, const DetectOut& o, const ContactList& cur, long long n_fresh,
                  const int* fa, const uint32_t* fb, long long nw_fresh, const int* fws,
                  const uint32_t* fww, double t, unsigned long long* d_missed, cudaStream_t st);

// per step
void launch_force_pairs(const DevState& d, ContactList& l, bool count_active, cudaStream_t st);
void launch_force_walls(const DevState& d, ContactList& l, double t, bool count_active,
                        cudaStream_t st);
void launch_update(const DevState& d, bool integrate, long long step, double margin,
                   bool check_cert, cudaStream_t st);
void launch_walls_at(const DevState& d, long long step, cudaStream_t st);
// Deterministic reduction: the clump slot lists of list l (cnt and fill are
// ncl zeroed scratch words; off gets ncl + 1 entries, ids 2 n + nw), and the
// per-clump sums of the slots into the accumulators.
void launch_det_lists(const DevState& d, const ContactList& l, long long n, long long nw,
                      uint32_t* cnt, uint32_t* fill, uint32_t* off, uint32_t* ids, void* scan_scratch,
                      unsigned long long* d_total, cudaStream_t st);
void launch_det_gather(const DevState& d, const ContactList& l, cudaStream_t st);
void launch_set_cert_ref(const DevState& d, cudaStream_t st);
void launch_get_state(const DevState& d, double* pos, double* quat, double* vel, double* angvel,
                      cudaStream_t st);
// Staged state: pos (3n) | quat (4n) | vel (3n) | angvel (3n) doubles.
void launch_check_state(const DevState& d, const double* staged, int* err, cudaStream_t st);
void launch_set_state(const DevState& d, const double* staged, cudaStream_t st);
void launch_get_forces(const DevState& d, double* F, double* T, cudaStream_t st);

}  // namespace dem
