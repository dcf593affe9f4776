/*
 * dem_oracle.h -- plain FP64 CPU oracle for the clump-of-spheres DEM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are written
 * independently from the paper (arXiv 2307.03445, "A GPU-accelerated simulator
 * for the DEM analysis of granular systems composed of clump-shaped elements").
 *
 * Equation numbering follows the paper's section 2.1 in reading order:
 *   Eq. (1a)-(1e)  normal / tangential force, f, effective radius and mass
 *   Eq. (2a)-(2c)  relative velocity at the contact point, its n and t parts
 *   Eq. (3)        tangential micro-displacement update and projection
 *   Eq. (4)        capping of the micro-displacement (Coulomb condition)
 *   Eq. (5a),(5b)  equations of motion of a clump
 * Section 2.2 ("DEM simulator overview") defines the enlarged-geometry contact
 * list, its deferred re-evaluation, and the zero force for false positives.
 *
 * Everything is double precision, single threaded, unblocked.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Detection lattice: coordinates are quantised to 2^-ORC_EPS_LOG2 metres. */
#define ORC_EPS_LOG2 24

enum { ORC_WALL_PLANE = 0, ORC_WALL_CYLINDER = 1, ORC_WALL_CONE = 2, ORC_WALL_TRIANGLE = 3 };
enum { ORC_MIX_MEAN = 0, ORC_MIX_MIN = 1, ORC_MIX_MAX = 2 };

typedef struct {
    int type;           /* ORC_WALL_* */
    int material;       /* material index of the wall surface */
    double p[3];        /* plane point | cylinder axis point | cone tip, at t = 0 */
    double n[3];        /* plane unit normal (towards the grains) | unit axis
                           (cone: from the tip towards the base) */
    double radius;      /* cylinder radius (grains inside) */
    double half_angle;  /* cone half angle [rad] (grains outside the solid cone) */
    double height;      /* cone height, tip to base plane */
    double vel[3];      /* prescribed translation velocity [m/s] */
    double b[3], c[3];  /* triangle: the other two vertices (p is the first);
                           n is its unit normal on the grains' side */
} orc_wall;

typedef struct {
    /* clump templates: template t owns spheres tpl_off[t] .. tpl_off[t+1]-1 */
    int n_tpl;
    const int* tpl_off;         /* n_tpl + 1 */
    const double* tpl_pos;      /* 3 * S, sphere centre in the clump principal frame */
    const double* tpl_rad;      /* S */
    const int* tpl_mat;         /* S, material per component sphere */
    const double* tpl_mass;     /* n_tpl */
    const double* tpl_inertia;  /* 3 * n_tpl, principal moments */
    /* per-material properties */
    int n_mat;
    const double *E, *nu, *mu, *cor;
    int mix_rule;               /* ORC_MIX_* for mu and CoR */
    /* boundaries */
    int n_walls;
    const orc_wall* walls;
    /* world */
    double h;                   /* time step */
    double g[3];
    double lo[3], hi[3];        /* detection domain */
    double bin_size;            /* bin edge [m] */
} orc_model;

/* ---- geometry and detection (section 2.2) ---------------------------- */
long long orc_num_spheres(const orc_model* m, int n, const int* tpl);
void orc_sphere_centres(const orc_model* m, int n, const int* tpl, const double* pos,
                        const double* quat, double* xs, int* owner, int* tsph);
void orc_detect_coords(const orc_model* m, long long ns, const double* xs, const int* tsph,
                       const double* margin, long long* qc, long long* rho);
void orc_grid_dims(const orc_model* m, long long dims[3], long long* bin_edge);
long long orc_bin_entries(const orc_model* m, long long ns, const long long* qc,
                          const long long* rho, long long cap, unsigned int* keys, int* ids);
long long orc_pairs_brute(long long ns, const int* owner, const long long* qc,
                          const long long* rho, long long cap, int* a, int* b);
long long orc_pairs_binned(const orc_model* m, long long ns, const int* owner,
                           const long long* qc, const long long* rho, long long cap,
                           int* a, int* b);
double orc_wall_distance(const orc_wall* w, double t, const double x[3], double nw[3]);
long long orc_wall_candidates(const orc_model* m, long long ns, const double* xs,
                              const int* tsph, const double* margin, double t,
                              double wall_travel_time, long long cap, int* s, int* w);

/* ---- contact law (Eq. 1-4) ------------------------------------------- */
void orc_pair_material(const orc_model* m, int mat_a, int mat_b, double* Estar,
                       double* Gstar, double* mu, double* cor);
/* One contact.  x*, X*: sphere centre and owner CoM; v*, w*: owner linear and
 * world angular velocity; r*: radii; m*: owner masses (mb <= 0: wall, i.e.
 * effective mass = ma and R = ra); u: tangential history in, out.
 * F: force acting on body b (body a receives -F); ca, cb: lever arms from each
 * owner CoM to the contact point.  Returns 1 if the contact is active. */
int orc_contact(const orc_model* m, int mat_a, int mat_b, const double xa[3],
                const double xb[3], const double Xa[3], const double Xb[3],
                const double va[3], const double wa[3], const double vb[3],
                const double wb[3], double ra, double rb, double ma, double mb,
                const double n_wall[3], double delta_wall, double u[3], double F[3],
                double ca[3], double cb[3]);

/* Forces and torques on every clump for one step (contacts given).  The
 * history arrays are updated in place.  F, T: 3 * n.  Fw: 3 * n_walls or NULL:
 * the force on each wall.  Tw: 3 * n_walls or NULL: the moment of those forces
 * about the wall's reference point at time t (p + vel t), each force acting
 * at its contact point.  mag: 2 * n or NULL; receives, per clump, the sums over its contacts of |F|
 * and of |lever arm| * |F| (the scales that bound the rounding of the force
 * and torque totals, including the cancellation inside each cross product).
 * Returns the number of active contacts. */
long long orc_forces(const orc_model* m, int n, const int* tpl, const double* pos,
                     const double* quat, const double* vel, const double* angvel,
                     double t, long long np, const int* pa, const int* pb, double* up,
                     long long nw, const int* ws, const int* ww, double* uw, double* F,
                     double* T, double* Fw, double* Tw, double* mag);

/* Explicit integration of Eq. (5) for every clump, in place. */
void orc_integrate(const orc_model* m, int n, const int* tpl, double* pos, double* quat,
                   double* vel, double* angvel, const double* F, const double* T);

/* ---- learned contact-list lifetime (not in the paper) ------------------ */
/* A per-bin regressor: ORC_MLP_IN features -> 3 hidden ReLU layers of width
 * ORC_MLP_H -> 1 output.  Parameters are one flat array, layer by layer,
 * each layer as W (row-major [out][in]) then b. */
#define ORC_MLP_IN 6
#define ORC_MLP_H 64
int orc_mlp_num_params(void);
void orc_mlp_forward(const double* params, long long n, const double* x, double* y);
/* As orc_mlp_forward with each layer's input rounded to bfloat16 (nearest,
 * ties to even) and double sums: the tensor-core arithmetic. */
void orc_mlp_forward_bf16act(const double* params, long long n, const double* x, double* y);
/* Mean squared error over n samples and (grad != NULL) its gradient. */
double orc_mlp_loss_grad(const double* params, long long n, const double* x, const double* t,
                         double* grad);
/* One Adam step (Kingma & Ba 2015) with bias correction; step counts from 1. */
void orc_mlp_adam(double* params, double* m, double* v, const double* grad, int step, double lr,
                  double beta1, double beta2, double eps);

/* ---- a whole simulation: deferred contact-list rebuilds ---------------- */
typedef struct orc_sim orc_sim;
orc_sim* orc_sim_create(const orc_model* m, int n, const int* tpl, const double* pos,
                        const double* quat, const double* vel, const double* angvel,
                        double margin, int rebuild_every);
/* Advances nsteps steps.  With audit != 0 every step also checks that each
 * touching pair/wall contact is in the list; returns the number of misses. */
long long orc_sim_step(orc_sim* s, int nsteps, int audit);
void orc_sim_get_state(const orc_sim* s, double* pos, double* quat, double* vel,
                       double* angvel);
long long orc_sim_num_contacts(const orc_sim* s, long long* n_wall);
void orc_sim_get_contacts(const orc_sim* s, int* a, int* b, double* u, int* ws, int* ww,
                          double* uw);
void orc_sim_last_forces(const orc_sim* s, double* F, double* T);
double orc_sim_time(const orc_sim* s);
long long orc_sim_active(const orc_sim* s);
void orc_sim_destroy(orc_sim* s);

#ifdef __cplusplus
}
#endif
#endif
