/*
 * dem.h -- C ABI of the GB300 clump-of-spheres DEM library (libdem.so).
 *
 * The library runs the hot path of the discrete element method of
 * arXiv 2307.03445 on one GPU: contact detection with an enlarged geometry
 * (section 2.2), the Hertz-Mindlin contact law with persistent tangential
 * history (section 2.1, Eq. (1)-(4)), the reduction of sphere forces to their
 * clump and the explicit integration of the clumps (Eq. (5)).
 *
 * Conventions for every entry point:
 *   - the return value is DEM_OK (0) or a negative DEM_ERR_* code; nothing
 *     throws across this boundary; dem_last_error() describes the last failure;
 *   - input arrays are plain host pointers (unless a call says otherwise),
 *     are read during the call only and stay owned by the caller;
 *   - output arrays are caller-owned buffers of the stated size;
 *   - a context is bound to one CUDA device and one stream, and is used by one
 *     host thread at a time;
 *   - units are SI; quaternions are (w, x, y, z) and unit length; angular
 *     velocities are in the world frame.
 * Equation numbers refer to the paper's section 2.1 in reading order:
 * Eq. (1a)-(1e) contact forces, (2a)-(2c) contact kinematics, (3) tangential
 * micro-displacement update, (4) its cap, (5a)-(5b) equations of motion.
 */
#ifndef DEM_H
#define DEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define DEM_OK 0
#define DEM_ERR_INVALID_ARG (-1) /* bad pointer, size, enum or value          */
#define DEM_ERR_OOM (-2)         /* device allocation failed                  */
#define DEM_ERR_CAPACITY (-3)    /* a list outgrew max_contacts               */
#define DEM_ERR_NONFINITE (-4)   /* a NaN/Inf appeared in the state           */
#define DEM_ERR_TIMEOUT (-5)     /* a bounded device wait ran out             */
#define DEM_ERR_CUDA (-6)        /* any other CUDA runtime error              */
#define DEM_ERR_STATE (-7)       /* call out of order (e.g. no templates)     */
#define DEM_ERR_GUARD (-8)       /* a list failed its validity check and no   */
                                 /* recovery was configured                   */

/* ---- enumerations ------------------------------------------------------ */
enum { DEM_FP64 = 0, DEM_FP32_VOXEL = 1 };
enum { DEM_WALL_PLANE = 0, DEM_WALL_CYLINDER = 1, DEM_WALL_CONE = 2, DEM_WALL_TRIANGLE = 3 };
enum { DEM_MIX_MEAN = 0, DEM_MIX_MIN = 1, DEM_MIX_MAX = 2 };
enum { DEM_MARGIN_FIXED = 0, DEM_MARGIN_LEARNED = 1 };
enum { DEM_GUARD_OFF = 0, DEM_GUARD_COUNT = 1, DEM_GUARD_ROLLBACK = 2 };

/* An analytic boundary with a prescribed translation (section 4 uses meshes
 * for funnels, cones and wheels; the library offers analytic stand-ins).
 *   PLANE:    p = a point, n = unit normal pointing towards the grains.
 *   CYLINDER: p = a point on the axis, n = unit axis, radius; grains inside.
 *   CONE:     p = tip, n = unit axis from the tip towards the base,
 *             half_angle [rad], height (tip to base); grains outside the solid.
 *   TRIANGLE: one facet of a triangle mesh (the paper's funnel, cone and wheel
 *             boundaries, section 4): vertices p, b, c; n = the unit normal
 *             (b - p) x (c - p) / |...| on the grains' side (checked to 1e-9).
 *             Distance: the signed distance to the facet's plane where the
 *             centre projects inside the facet, else the distance to the
 *             nearest edge.  Every sphere-facet pair is its own contact (a
 *             mesh is a list of facets; its load is the sum of theirs).
 * The surface moves with velocity vel: its reference point at time t is
 * p + vel * t.  material indexes the material table.  scene = -1 applies the
 * wall to every scene, otherwise to one scene.  A scene holds at most 32
 * PLANE, CYLINDER and CONE walls (every sphere tests each of them at a
 * rebuild); TRIANGLE facets have no such limit: at a rebuild each facet is
 * registered in the detection bins its box (widened by its travel over the
 * list's lifetime) touches, and only the spheres registered in the same bins
 * are tested against it (section 2.2's binning, applied to the mesh). */
typedef struct {
    int type;
    int material;
    double p[3];
    double n[3];
    double radius;
    double half_angle;
    double height;
    double vel[3];
    int scene;
    double b[3], c[3];  /* TRIANGLE: second and third vertex (else unused) */
} dem_wall;

/* Creation parameters.  Arrays are copied by dem_create. */
typedef struct {
    double dt;                /* time step h [s] (> 0)                               */
    double g[3];              /* gravity [m/s^2]                                      */
    double domain_lo[3];      /* detection domain of scene 0 [m]; spheres outside it  */
    double domain_hi[3];      /*   are binned into the boundary bins (still detected)  */
    int precision;            /* DEM_FP64 or DEM_FP32_VOXEL                           */
    double bin_size;          /* bin edge [m]; 0 = twice the largest enlarged radius  */
    int margin_policy;        /* DEM_MARGIN_FIXED | DEM_MARGIN_LEARNED                */
    int rebuild_interval;     /* K: list rebuilt every K steps (>= 1)                 */
    double v_bound;           /* speed bound [m/s]; margin = v_bound * dt * K ...      */
    double margin;            /* ... unless margin > 0, which sets it directly [m]    */
    int mix_rule;             /* how mu and CoR of two spheres combine: DEM_MIX_*     */
    int n_materials;          /* >= 1                                                  */
    const double* E;          /* Young's modulus per material [Pa]                    */
    const double* nu;         /* Poisson ratio                                         */
    const double* mu;         /* friction coefficient                                  */
    const double* cor;        /* coefficient of restitution in [0, 1]                  */
    int n_walls;
    const dem_wall* walls;
    long long max_contacts;   /* cap on listed pairs; 0 = no cap (grows on demand)    */
    int guard;                /* DEM_GUARD_*: what a failed validity check does        */
    void* cuda_stream;        /* cudaStream_t to run on; NULL = the library's own     */
    int device;               /* CUDA device ordinal                                   */
    /* Optional device allocator (e.g. a framework's caching allocator); both
     * NULL = cudaMallocAsync / cudaFreeAsync on the context stream.  Its
     * blocks must be 256-byte aligned, as cudaMalloc's are (the kernels move
     * 16- and 32-byte records); a misaligned block fails the call with
     * DEM_ERR_OOM.  free is called where cudaFreeAsync would be: work queued
     * on the context stream may still use the block, so the allocator must
     * not hand it out again before that work is done (a caching allocator
     * whose blocks belong to the context stream, as PyTorch's do when
     * allocated on it, satisfies this). */
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* alloc_user;
} dem_params;

/* Counters and timings since creation (or the last dem_reset_stats). */
typedef struct {
    long long steps;            /* force steps taken                               */
    long long rebuilds;         /* contact-list rebuilds                           */
    long long n_clumps, n_spheres;
    long long n_pairs;          /* listed sphere-sphere pairs (current list)       */
    long long n_wall_contacts;  /* listed sphere-wall contacts (current list)      */
    long long bin_entries;      /* (bin, sphere) registrations of the last rebuild */
    long long pair_steps;       /* sum over steps of listed pairs + wall contacts  */
    long long active_last;      /* contacts with delta_n > 0 in the last step      */
    long long guard_violations; /* steps whose list failed the validity check      */
    long long rollbacks;        /* rollbacks to the last snapshot                   */
    long long missed_contacts;  /* touching contacts found missing by audits        */
    double margin;              /* current margin [m] (fixed policy)               */
    double time;                /* simulated time [s]                               */
    /* device time per phase [ms], accumulated while timing is on: list
     * rebuilds, sphere-sphere force kernel, sphere-wall force kernel, clump
     * update kernel; timed_steps counts the steps these cover. */
    double ms_detect, ms_pairs, ms_walls, ms_update;
    long long timed_steps;
    long long launches;         /* kernels this library launched                    */
    long long early_rebuilds;   /* learned-rule intervals cut short by a failed     */
                                /*   displacement certificate (see below)           */
    double ms_predict;          /* device time of the learned rule's margin        */
                                /*   predictions [ms], while timing is on           */
    long long outer_rebuilds;   /* detections of the outer list (dem_set_outer_list) */
} dem_stats;

typedef struct dem_ctx dem_ctx;

/* Creates a context.  Validates the parameters (DEM_ERR_INVALID_ARG), selects
 * params->device, copies the material table and walls, precomputes the pair
 * material table (section 2.1: pair stiffness and damping from each sphere's
 * E, nu, mu, CoR).  *out receives the context, or NULL on failure. */
int dem_create(const dem_params* params, dem_ctx** out);

/* Frees every device and host resource of the context.  NULL is accepted. */
void dem_destroy(dem_ctx* ctx);

/* Text of the last error on this context (or of the last failed dem_create
 * when ctx is NULL).  Valid until the next call on the context. */
const char* dem_last_error(const dem_ctx* ctx);

/* Loads the clump templates (section 2.1: a clump is a rigid union of
 * possibly overlapping spheres, each with its own material).
 *   n_tpl           number of templates (>= 1)
 *   sphere_offsets  n_tpl + 1 ints; template t owns spheres [off[t], off[t+1])
 *   local_pos       3 * S doubles: sphere centres in the template's principal
 *                   frame, centre of mass at the origin (S = off[n_tpl])
 *   radius          S doubles (> 0)
 *   material        S ints in [0, n_materials)
 *   mass            n_tpl doubles (> 0)
 *   inertia         3 * n_tpl doubles: principal moments (> 0)
 * Must precede dem_add_clumps; may be called once. */
int dem_load_clump_templates(dem_ctx* ctx, int n_tpl, const int* sphere_offsets,
                             const double* local_pos, const double* radius,
                             const int* material, const double* mass,
                             const double* inertia);

/* Adds a scene (an independent system sharing the templates, materials, dt
 * and g) with its own detection domain and bin size; scene 0 exists from
 * dem_create.  *scene_id receives the new id.  Bodies of different scenes
 * never interact.  Must precede the first dem_add_clumps into that scene. */
int dem_add_scene(dem_ctx* ctx, const double lo[3], const double hi[3], double bin_size,
                  int* scene_id);

/* Appends n clumps to a scene.
 *   tpl    n ints, template ids
 *   pos    3n doubles, centre of mass [m]
 *   quat   4n doubles, unit quaternions (w, x, y, z)
 *   vel    3n doubles [m/s]; angvel 3n doubles [rad/s], world frame
 * Clump i receives id (number of clumps before the call) + i; its spheres are
 * numbered consecutively in template order.  Rejects non-finite values.
 * Ids are also the order of the records in device memory: clumps added in a
 * spatially coherent order (e.g. along a Morton curve) keep the records of
 * touching spheres close together, and the force kernel then reads them from
 * L2 (about 1.6x faster on a 34M-sphere bed than a random order within
 * 0.25 m patches). */
int dem_add_clumps(dem_ctx* ctx, int n, const int* tpl, const double* pos,
                   const double* quat, const double* vel, const double* angvel, int scene);

/* Advances n_steps time steps: every step evaluates every listed contact
 * (section 2.2: deferred list, false positives give zero force), reduces the
 * forces and torques to the clumps and integrates Eq. (5); the list is
 * rebuilt when the rebuild rule says so.  Synchronises the stream before
 * returning and reports device-side failures (NONFINITE, CAPACITY, GUARD). */
int dem_step(dem_ctx* ctx, int n_steps);

/* Copies the clump state out.  on_device = 1: the four pointers are device
 * pointers on the context's device; 0: host pointers.  Sizes as in
 * dem_add_clumps, for all clumps in id order.  Any pointer may be NULL. */
int dem_get_state(dem_ctx* ctx, double* pos, double* quat, double* vel, double* angvel,
                  int on_device);

/* Overwrites the state of all clumps (host pointers, same layout as
 * dem_get_state; page-locked memory makes the copies DMA transfers).  The next
 * step rebuilds the list; tangential history is kept for pairs that stay
 * listed.  Once the context has stepped or rebuilt, the arrays are copied as
 * given into a device staging buffer (13 doubles per clump, kept by the
 * context) and validated and converted there; before that they are converted
 * on the host.  Errors: DEM_ERR_NONFINITE for a NaN or infinity,
 * DEM_ERR_INVALID_ARG (FP32_VOXEL) for a position more than 2e9 voxels from
 * its scene's corner; in both cases no clump record changes. */
int dem_set_state(dem_ctx* ctx, const double* pos, const double* quat, const double* vel,
                  const double* angvel);

/* Two-level contact list for the plain rule (no counterpart in the paper's
 * text; an acceleration of section 2.2's rebuild that keeps its result).
 * With n_inner >= 1 a rebuild detects an outer list with the wider margin
 * factor * m (factor > 1), whose wall candidates also cover the walls' travel
 * over n_inner rebuild intervals, and keeps the lattice point of every sphere
 * at that time.  The next n_inner rebuilds (that one included) take their
 * list from the outer one: each pair or wall candidate of the outer list is
 * kept when it passes the exact test of a fresh detection at margin m, which
 * gives exactly the fresh detection's list, in the same order, as long as no
 * sphere's lattice point moved further from its outer-list point than the
 * difference of its two enlarged radii; every rebuild checks this for every
 * sphere and detects a new outer list when one moved further.  Adding clumps
 * or changing a wall's motion also starts a new outer list; the learned rule
 * and dem_rebuild use full detections.  n_inner = 0 turns it off (default).
 * dem_get_bins then reports the bins of the last outer list detected on the
 * context stream.
 *
 * async_detect != 0 (section 2.2's kinematics thread building the next
 * contact list while the dynamics thread steps, on one GPU with two streams):
 * at the last rebuild an outer list serves, the next one is started from
 * that rebuild's state; the part that reads the state (lattice points, bin
 * counts, wall candidates) runs on the context stream in order with the
 * steps, the rest (bin scatter, narrow phase, the list's rows and the host's
 * waits for its sizes) on a second stream of the context while the
 * interval's steps run; the next rebuild adopts it.  Its wall candidates
 * cover n_inner + 1 intervals, since it is adopted one interval after its
 * state; the lists filtered from it are still exactly those of a fresh
 * detection (the allowance check holds them to that).  Off while the scene
 * has mesh facets (their registration reads the state in the second part).
 * dem_step returns with the second stream idle.  Needs the library's
 * stream-ordered allocator (not a dem_params.alloc).  Returns
 * DEM_ERR_INVALID_ARG for factor <= 1, n_inner < 0, or async_detect with a
 * custom allocator. */
int dem_set_outer_list(dem_ctx* ctx, double factor, int n_inner, int async_detect);

int dem_get_stats(dem_ctx* ctx, dem_stats* out);
int dem_reset_stats(dem_ctx* ctx);
/* timing = 1 records CUDA events around each phase of every step on the
 * context stream; they are read once at the end of each dem_step call, so
 * the steps themselves are not serialised. */
int dem_set_timing(dem_ctx* ctx, int timing);
/* on = 1: deterministic reduction.  Every contact writes its force and
 * moments to its own slot, and a per-clump pass adds the slots of each clump
 * in a fixed order (slot lists built with each contact list), so that runs
 * with the same inputs give bit-identical trajectories.  Costs one slot write
 * and read per contact per step.  on = 0 (default): vector reductions into
 * the accumulators, whose summation order varies from run to run.  The net
 * forces on the walls are summed by atomics in both modes. */
int dem_set_deterministic(dem_ctx* ctx, int on);

/* Bin-size autotuner (the paper fixes no bin size; this picks one by timing).
 * For each of the n factors, the bin edge of every scene becomes the factor
 * times the scene's base edge (its bin_size, else twice the largest enlarged
 * radius), the contact list is rebuilt once to size the buffers, then `reps`
 * more times under CUDA events.  The fastest factor is kept (*best) and the
 * list is rebuilt with it.  ms (n doubles, may be NULL) receives the mean
 * rebuild time per factor, -1 for a factor that gives no valid grid (more
 * than 2^21 bins along an axis or 2^32 in all).  The state is unchanged: a
 * rebuild carries the tangential history over. */
int dem_autotune_bins(dem_ctx* ctx, int n, const double* factors, int reps, double* best,
                      double* ms);

/* Launch shapes of the hot kernels.  None of them changes a result: every
 * per-contact and per-clump computation is the same whatever the grid, and
 * in deterministic mode the trajectory is bit-identical across shapes. */
typedef struct {
    int pairs_blocks_per_sm;  /* blocks of 256 threads per SM for the pair force kernels
                                 (grid-stride loop), 1..32; default 8 */
    int update_block;         /* clumps per block of the FP32_VOXEL update kernel: 64,
                                 128 (default) or 256 */
    int narrow_chunk;         /* bins a narrow-phase warp claims at a time, 1..64; default 8 */
} dem_tiles;
/* DEM_ERR_INVALID_ARG for a value out of range (nothing changes then). */
int dem_set_tiles(dem_ctx* ctx, const dem_tiles* tiles);
int dem_get_tiles(dem_ctx* ctx, dem_tiles* tiles);
/* Tile autotuner, one coordinate at a time: the narrow chunk over
 * {2, 4, 8, 16, 32} timed on `reps` rebuilds each, then the pair blocks per
 * SM over {2, 4, 8, 16} and the update block over {64, 128, 256}, each timed
 * on `steps` force + update steps from a snapshot of the state and the list
 * history taken at a fresh rebuild.  The snapshot is restored after the
 * trials, so the state, the step count and the counters are unchanged; the
 * fastest shapes are kept and written to *best.  Overwrites the rollback
 * snapshot of the learned rule (call it outside dem_step). */
int dem_autotune_tiles(dem_ctx* ctx, int steps, int reps, dem_tiles* best);

/* enabled = 1 runs the steps between two rebuilds of the plain rule as one
 * CUDA graph launch (captured on first use per list buffer, step count and
 * margin, and recaptured after any buffer is reallocated).  Results are those
 * of the ordinary launches.  Ignored while timing is on.  Default 0. */
int dem_set_graphs(dem_ctx* ctx, int enabled);

/* ---- inspection (tests, tools) ----------------------------------------- */

/* Rebuilds the contact list now from the current state (section 2.2), keeping
 * the tangential history of pairs present before and after. */
int dem_rebuild(dem_ctx* ctx);

/* Evaluates the contact forces of the current state with the current list
 * (rebuilding first if none exists) without integrating or advancing time;
 * updates the tangential history exactly as a step would.  The per-clump
 * totals are then readable with dem_get_forces. */
int dem_eval_forces(dem_ctx* ctx);

/* Net contact force and torque per clump from the last dem_eval_forces
 * (3 * n_clumps doubles each, host buffers).  Torque about the clump CoM. */
int dem_get_forces(dem_ctx* ctx, double* force, double* torque);

/* Net force on each wall from the last force evaluation (3 * n_walls). */
int dem_get_wall_forces(dem_ctx* ctx, double* force);

/* Co-simulation hook (boundaries driven by another solver, as the rover's
 * multibody model drives the wheels in section 5.2).  Loads: the net
 * force on each wall and its moment about the wall's reference point at the
 * time of the last force evaluation (p + vel t), each contact force acting at
 * its contact point (3 * n_walls doubles each, host buffers).  The sum over
 * the clumps of X x F + T plus the sum over the walls of p(t) x F_w + T_w is
 * zero up to rounding.  A mesh's load is the sum over its facets: the force
 * sum F_w, and about a point P (a wheel's hub) the sum of
 * T_w + (p_w(t) - P) x F_w, with p_w(t) the facet's first vertex at that time. */
int dem_get_wall_loads(dem_ctx* ctx, double* force, double* torque);
/* Motion: from the current time t on, wall `wall` (index in the walls given
 * at creation) moves as point + vel (t' - t), i.e. its stored reference
 * point becomes point - vel t.  The next step rebuilds the contact lists
 * (the listed wall candidates assumed the old motion); the wall's tangential
 * histories are kept for contacts that stay listed.  Errors:
 * DEM_ERR_INVALID_ARG (index out of range), DEM_ERR_NONFINITE. */
int dem_set_wall_motion(dem_ctx* ctx, int wall, const double* point, const double* vel);

/* Sizes of the current lists. */
int dem_num_contacts(dem_ctx* ctx, long long* n_pairs, long long* n_wall);

/* Copies the current lists (host buffers sized by dem_num_contacts): pairs
 * (a < b, sphere ids, sorted by (a, b)) with their tangential history u
 * (3 doubles each), and sphere-wall contacts (sphere, wall) with history.
 * In DEM_FP32_VOXEL the device keeps a pair's history components as
 * float-float (about 48 significant bits); u receives their sums. */
int dem_get_contacts(dem_ctx* ctx, int* a, int* b, double* u, int* wall_sphere, int* wall_id,
                     double* wall_u);

/* Bin registrations of the last rebuild sorted by (bin key, sphere id):
 * keys/ids hold up to cap entries; *n receives the total. */
int dem_get_bins(dem_ctx* ctx, long long cap, unsigned int* keys, int* ids, long long* n);

/* The exact missed-contact check: a fresh zero-margin detection of the
 * current state compared with the current list.  *missed receives the number
 * of touching sphere pairs and sphere-wall contacts that are not listed. */
int dem_audit(dem_ctx* ctx, long long* missed);

/* ---- learned list lifetime (an extension: the paper uses a fixed margin) --
 * A small regressor predicts, per detection bin, how many steps the contact
 * list built with a given margin stays valid for the clumps of that bin.
 * Inputs (dem_trace documents them): 6 floats per sample; output: the natural
 * log of the number of steps.  Network: 6 -> 64 -> 64 -> 64 -> 1 with ReLU,
 * BF16 weights and FP32 accumulation on the GPU; parameters are one flat
 * float vector, layer by layer, each layer W (row-major [out][in]) then b. */
typedef struct dem_mlp dem_mlp;

/* Number of parameters (8833). */
int dem_mlp_num_params(void);
/* Creates a regressor on `device` with a fixed-seed initialisation. */
int dem_mlp_create(int device, dem_mlp** out);
void dem_mlp_destroy(dem_mlp* mlp);
/* Sets / reads the FP32 master parameters (host arrays of num_params);
 * setting resets the Adam moments. */
int dem_mlp_set_params(dem_mlp* mlp, const float* params);
int dem_mlp_get_params(dem_mlp* mlp, float* params);
/* y[k] for k < n from x[6k .. 6k+5] (host arrays). */
int dem_mlp_forward(dem_mlp* mlp, long long n, const float* x, float* y);
/* The same forward pass on the tensor cores (tcgen05.mma, 128-row tiles):
 * every layer's input is rounded to bfloat16 and the products are summed in
 * FP32, so results differ from dem_mlp_forward by bfloat16 rounding of the
 * activations.  The learned rule's predictions use this pass.
 * DEM_ERR_TIMEOUT if a bounded wait on the tensor cores ran out. */
int dem_mlp_forward_tc(dem_mlp* mlp, long long n, const float* x, float* y);
/* Mean squared error of predictions against targets t (host), and its
 * gradient with respect to the parameters (host, may be NULL). */
int dem_mlp_loss_grad(dem_mlp* mlp, long long n, const float* x, const float* t, double* loss,
                      float* grad);
/* The same loss and gradient as dem_mlp_loss_grad, computed without any
 * device allocation: no cudaMalloc / cudaFree, no allocating library call.
 * The paper has no counterpart; this serves callers that cannot allocate,
 * e.g. a process whose device memory another allocator already holds in full,
 * or a host loop that must not wait on the device-wide synchronisation of a
 * free.  Rows, targets, the gradient and the loss sum live in one fixed
 * scratch array of the library (file-scope __device__ storage, about 7.4 MB
 * per device).
 *   - n > DEM_MLP_NOALLOC_MAX_ROWS returns DEM_ERR_CAPACITY (nothing runs).
 *   - The scratch address is looked up with cudaGetSymbolAddress on the first
 *     call on each device (DEM_ERR_CUDA if that fails); make that first call
 *     before any stream capture begins on the device.
 *   - The gradient and loss accumulators are cleared at the start of every
 *     call; rows past n are left as they were and never read.
 *   - There is one scratch array per device: calls on the same device that
 *     overlap in time (from several host threads, or several regressors)
 *     race on it; the caller serialises them.
 * Returns once the results are in the host arrays. */
#define DEM_MLP_NOALLOC_MAX_ROWS 262144
int dem_mlp_loss_grad_noalloc(dem_mlp* mlp, long long n, const float* x, const float* t,
                              double* loss, float* grad);
/* `steps` Adam steps (lr, beta 0.9/0.999, eps 1e-8) on minibatches of `batch`
 * samples drawn without replacement per epoch (seeded); *final_loss gets the
 * loss over all n samples after training. */
int dem_mlp_train(dem_mlp* mlp, long long n, const float* x, const float* t, int steps, int batch,
                  float lr, unsigned long long seed, double* final_loss);

/* Learned rebuild rule.  At each rebuild, for every occupied bin, the
 * regressor is queried at each candidate margin (ascending, in metres); the
 * clumps of the bin get the smallest candidate whose predicted lifetime is at
 * least interval * safety (the largest candidate otherwise), and the list is
 * rebuilt every `interval` steps.  Every step checks that no clump moved
 * further than its margin since the rebuild (a certificate that no contact is
 * missing from the list).  What a failed certificate does depends on mode:
 *   DEM_LEARNED_HALT (0): the failing step completes its integration, and
 *     every later step of the interval is skipped on the device before it
 *     computes a force (its kernels see the halt step and return); the list
 *     is rebuilt at once and stepping continues.  Nothing is rolled back; no
 *     force is ever computed with a list that lacks a contact.  The interval
 *     is launched in chunks of 8 steps and the host reads the halt step back
 *     one chunk behind, so at most about two chunks are launched past a halt.
 *   DEM_LEARNED_ROLLBACK (1): the interval runs to its end; it is then judged
 *     by the certificate and by the exact check against a fresh zero-margin
 *     detection (as dem_audit); on a failure or a missing contact the state
 *     and tangential history are rolled back to the rebuild and the interval
 *     is replayed with the plain rule (margin and rebuild_interval of
 *     dem_params), and with a rebuild every step if that fails too.
 * speed_floor (>= 0; 0 turns it off) keeps every clump's margin at least
 * speed_floor * h * interval * (|v| + |omega| b), b the template's largest
 * sphere-centre distance from its centre of mass, at the clump's speed when
 * the margins are chosen: the distance it covers in the interval at that
 * speed.  The regressor judges bins; a fast clump in a bin of slow ones would
 * otherwise end the interval early on the certificate.
 * mlp = NULL restores the plain rule.  The regressor must outlive its use. */
enum { DEM_LEARNED_HALT = 0, DEM_LEARNED_ROLLBACK = 1 };
typedef struct {
    int interval;
    double safety;
    int n_candidates;
    const double* candidates;
    int mode;                 /* DEM_LEARNED_HALT or DEM_LEARNED_ROLLBACK */
    double speed_floor;       /* 0: off; else the margin floor's factor (see above) */
} dem_learned_params;
int dem_set_learned_policy(dem_ctx* ctx, dem_mlp* mlp, const dem_learned_params* params);

/* Training traces from the plain rule.  Runs `windows` windows of `window`
 * steps; at the start of each window every occupied bin of the learned
 * rule's grid (cells of the scene's base bin edge: its bin_size, else twice
 * the largest enlarged radius, whatever edge dem_autotune_bins picks for
 * detection) yields, for each candidate margin m, the features
 *   x = [ln(1 + clumps in bin), ln(h vmax / m), ln(h vmean / m),
 *        ln(h^2 amax / m), ln(m / r_mean), ln(h^2 |g| / m)]
 * (vmax, vmean: largest and mean clump speed bound |v| + |w| r_bound; amax:
 * largest clump acceleration in the last step; r_mean: mean sphere radius)
 * and the target t = ln(T), T the first step of the window at which a clump
 * of the bin has moved further than m (T = window if none did).  Writes up
 * to cap samples into x (6 * cap) and t (cap); *n receives the count.
 * Samples are ordered by window, then occupied bin, then candidate (the
 * n_candidates samples of one bin are adjacent, in the given order). */
int dem_trace(dem_ctx* ctx, int windows, int window, int n_candidates, const double* candidates,
              long long cap, float* x, float* t, long long* n);

#ifdef __cplusplus
}
#endif
#endif
