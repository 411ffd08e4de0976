/*
 * lbm.h -- C ABI of the B300 porous-media lattice Boltzmann library (liblbm.so).
 *
 * The library advances the monolithic one-domain porous-media LBM of Gusev &
 * Karlin, "Monolithic kinetic algorithm for heterogeneous porous media systems
 * using a continuous one-domain approach", Sec. 3: product-form equilibria
 * (Eqs. (1d_scaled_eq)-(P_aa_*)), the collide-and-stream update Eq.
 * (dicrete_scheme) with the Relax-to-Force source Eq. (momentum_rate) and
 * lambda = delta t, the three-step velocity solve Eqs. (v_(0))-(v_final), the
 * acceleration Eq. (accel) with the porosity correction Eq.
 * (porosity_correction_expanded), and the correction terms Eqs. (ex_corr),
 * (eta_corr).  Lattice units: delta t = delta x = 1.
 *
 * Conventions
 *   node index     n = x + nx*(y + ny*z), x fastest; D2Q9 uses nz = 1.
 *   velocities     D2Q9  i = ix + 3*iy,         c_i = (ix-1, iy-1)
 *                  D3Q27 i = ix + 3*iy + 9*iz,  c_i = (ix-1, iy-1, iz-1)
 *                  opposite(i) = Q-1-i.
 *   populations    the transformed populations f_bar of Eq. (f_bar_transform),
 *                  after streaming (the state the paper's flowchart collides).
 *   walls          link-wise halfway bounce-back half a spacing outside the
 *                  first and last node layer of an axis.
 *
 * Errors: every int-returning call returns LBM_OK (0) or a negative LBM_E_*
 * code and never throws across the ABI; lbm_last_error() describes the last
 * failure of the calling thread.  A context is used by one thread at a time.
 *
 * Memory: lbm_create copies every input array; the caller keeps ownership of
 * its buffers.  Device memory comes from the allocator callbacks of
 * lbm_params when set (so a host framework's caching allocator can own it),
 * else from cudaMalloc; lbm_destroy returns all of it.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* return codes */
#define LBM_OK 0
#define LBM_E_INVALID (-1)     /* argument out of range, rejected before any device work */
#define LBM_E_CUDA (-2)        /* a CUDA runtime call failed */
#define LBM_E_NOMEM (-3)       /* device allocation failed */
#define LBM_E_DIVERGED (-4)    /* sticky device flag: rho <= 0, NaN/Inf, or |v|/eps > 0.5 */
#define LBM_E_UNSUPPORTED (-5) /* valid but not built (e.g. a kernel for this lattice/storage) */
#define LBM_E_TIMEOUT (-6)     /* sticky device flag: a kernel gave up a bounded wait for its copies into
                                  shared memory and skipped its work; the state is invalid */

/* lattices (Sec. 3.1) */
#define LBM_D2Q9 0
#define LBM_D3Q27 1

/* population storage; arithmetic is FP64 for LBM_STORE_FP64 and FP32 otherwise.
   Reduced-precision forms store the deviation f_bar_i - eps(x) w_i rho0, scaled
   by 1/w_i for FP16/BF16. */
#define LBM_STORE_FP64 0
#define LBM_STORE_FP32 1
#define LBM_STORE_FP16 2
#define LBM_STORE_BF16 3

/* per-axis boundary (both faces of the axis) */
#define LBM_BC_PERIODIC 0
#define LBM_BC_WALL 1
/* x axis only: velocity inlet at x = 0 (inlet_v, uniform or the Poiseuille
   profile that inlet_profile selects) and an outlet at x = nx-1 (outlet: a
   prescribed density outlet_rho, or zero-gradient outflow), wet-node planes
   rebuilt after streaming by the boundary density of Eq.
   (bc_density_impermWall) and the reconstruction that plane_scheme selects
   (LBM_PLANES_*).  Porosity and permeability must be uniform over the three
   node layers next to each plane, and the outlet layers free fluid
   (permeability +INF): there the acceleration of Eq. (accel) is explicit
   (Sec. 3.4.1).  lbm_create returns LBM_E_UNSUPPORTED otherwise. */
#define LBM_BC_INFLOW_OUTFLOW 2
/* y axis: with z periodic and x periodic, LBM_BC_INFLOW_OUTFLOW or wet walls:
   wet-node walls on the node rows y = 0 and y = ny-1 that move tangentially
   with the superficial velocities wall_v_low and wall_v_high (the Couette
   walls of Sec. 5.1; at rest, the channel walls of Sec. 6.1).  After
   streaming every population of a wall node is rebuilt: the density by mass
   continuity, Eq. (bc_density_impermWall) with v_perp = 0 (or the bounce-back
   density), then the reconstruction that plane_scheme selects.  With inlet /
   outlet planes the four corner columns take the wall velocity and the
   density of their diagonal bulk neighbour (Sec. 6.1 extrapolates the corner
   density from neighbouring nodes) -- or, with the bounce-back density, their
   own --, rebuilt after the x sides and before the wall rows.
   x axis: wet-node walls at rest on the node columns x = 0 and x = nx-1 (the
   side walls of the cavity of Sec. 6.2), with y periodic or wet walls and z
   periodic.  Porosity and permeability must be uniform over the three node
   rows next to each wall (LBM_E_UNSUPPORTED otherwise). */
#define LBM_BC_MOVING_WALLS 3

/* reconstruction of every population of an inlet / outlet node (Sec. 3.4),
   with f_tgt = f_eq(eps_b, rho_b, v_b) and f_* = f_eq(eps_b, rho_b, v_b + a_b):
   NEEM: non-equilibrium extrapolation from the interior neighbour along the
         normal, Eqs. (NEEM_bc_f_bar), (zeta_beta_NEEM) (default);
   EQUILIBRIUM: f_bar = 1.5 f_tgt - 0.5 f_*, Eq. (eq_bc_f_bar);
   TMS: Tamm--Mott-Smith, Eq. (f_i_neq_TMS) by the three steps of Sec. 3.4
        (local rho and v from the known populations, their equilibrium f_loc,
        then (f_tgt - f_loc) / (1 - beta) added to 1.5 f_tgt - 0.5 f_* for the
        populations entering from outside and to the known ones otherwise). */
#define LBM_PLANES_NEEM 0
#define LBM_PLANES_EQUILIBRIUM 1
#define LBM_PLANES_TMS 2

/* density of a wet-node wall (moving walls):
   CONTINUITY: Eq. (bc_density_impermWall) from the known populations and the
               prescribed velocity (default);
   BOUNCE_BACK: Eq. (bc_density_BounceBack), the known post-advection
               populations plus the outgoing post-collision ones, which every
               kernel reflects into the unknown slots of the boundary node.
               The paper states it for solid boundaries: an inlet always takes
               the density by continuity. */
#define LBM_DENSITY_CONTINUITY 0
#define LBM_DENSITY_BOUNCE_BACK 1

/* outlet of LBM_BC_INFLOW_OUTFLOW:
   PRESSURE: prescribed density outlet_rho; the normal velocity from mass
             continuity, the tangential one from the interior neighbour
             (default);
   ZERO_GRADIENT: the populations entering from outside are copied from the
             interior neighbour, Eq. (f_bar_outflow_BC).  With a velocity inlet
             it fixes no density level: between walls the density of a steady
             flow grows by a constant factor per step (the flow needs a density
             drop against the wall friction that the copied outlet does not
             let out). */
#define LBM_OUTLET_PRESSURE 0
#define LBM_OUTLET_ZERO_GRADIENT 1

/* inlet velocity of LBM_BC_INFLOW_OUTFLOW:
   UNIFORM: inlet_v at every inlet node (default);
   POISEUILLE: v_x = 6 inlet_v[0] eta (1 - eta), v_y = v_z = 0, Eq.
             (cylinder_inlet_BC), eta across y between the walls (wet-node
             walls on the rows y = 0 and ny-1: eta = y / (ny-1); halfway
             bounce-back walls: eta = (y + 1/2) / ny); needs walls on y. */
#define LBM_INLET_UNIFORM 0
#define LBM_INLET_POISEUILLE 1

/* velocity of the moving y walls of a cavity (wet walls on x and y):
   UNIFORM: wall_v_low / wall_v_high (default);
   REGULARISED: their x component times S(min(x, L - x) / (lid_delta L)),
             L = nx - 1, with the smoothstep S of Eq. (s_cinf): Eq.
             (cavity_velocity_profile), which vanishes at the corners. */
#define LBM_LID_UNIFORM 0
#define LBM_LID_REGULARISED 1

/* correction terms (bit mask); LBM_CORR_FULL is the paper's model */
#define LBM_CORR_DELTA_NU 1 /* Eq. (porosity_correction) in Eqs. (v_final), (accel) */
#define LBM_CORR_PHI_EXT 2  /* Eq. (ex_corr) */
#define LBM_CORR_PHI_ETA 4  /* Eq. (eta_corr) */
#define LBM_CORR_FULL 7

/* kernel selection */
#define LBM_KERNEL_AUTO 0  /* split kernels where built, else the fused kernel, else the sweep kernels */
#define LBM_KERNEL_SWEEP 1 /* three sweeps per step through device scratch fields */
#define LBM_KERNEL_FUSED 2 /* one z-marching kernel per step (D3Q27, FP32-compute storages) */
#define LBM_KERNEL_SPLIT 3 /* three streaming kernels per step (moments, velocity, collide), through
                              scratch fields (D3Q27, FP32-compute storages, fewer than 2^31 nodes) */

/* population streaming of the split kernels (lbm_params.streaming):
   TWO_ARRAYS: push into a second population array (two arrays);
   IN_PLACE:   AA-pattern in-place streaming, ONE population array whose layout
               alternates between steps (every call below still sees the
               post-stream f_bar in the documented order); nx must be even.
               Measured on a B300 it halves the population memory and costs
               about 7 % (FP32) to 10 % (FP16) of step time: every other step
               reads and writes neighbour-shifted slots;
   AUTO:       IN_PLACE when two arrays would take more than half the device
               memory free at creation (or nx is odd: TWO_ARRAYS), else
               TWO_ARRAYS (default).  Other kernels always use two arrays. */
#define LBM_STREAM_AUTO 0
#define LBM_STREAM_TWO_ARRAYS 1
#define LBM_STREAM_IN_PLACE 2
/* forchheimer argument: pass a value < 0 to use the Ergun correlation
   F_eps = 1.75 / sqrt(150 eps^3), Eq. (F_eps_Ergun), per node */
#define LBM_F_ERGUN (-1.0)

typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* user);

typedef struct {
    int storage;     /* LBM_STORE_*, default LBM_STORE_FP32 */
    double RT;       /* lattice temperature RT (c_s^2), default 1/3 */
    double J_nu;     /* nu_eff / nu_f, default 1 (Eq. (ratios_def)) */
    double J_eta;    /* eta_eff / nu_f, default 1 */
    int corrections; /* LBM_CORR_* mask, default LBM_CORR_FULL */
    int bc[3];       /* LBM_BC_* per axis x, y, z; default periodic */
    double rho0;     /* initial intrinsic density, default 1; also the deviation reference */
    double v0[3];    /* initial superficial velocity, default 0 */
    void* stream;    /* cudaStream_t for all work of the context; NULL = a stream the library creates */
    int device;      /* CUDA device ordinal, default 0 */
    lbm_alloc_fn alloc; /* optional device allocator; both or neither of alloc/free */
    lbm_free_fn free;
    void* alloc_user;
    int kernel; /* LBM_KERNEL_*, default LBM_KERNEL_AUTO */
    double inlet_v[3];  /* superficial inlet velocity for LBM_BC_INFLOW_OUTFLOW, default 0 */
    double outlet_rho;  /* outlet intrinsic density for LBM_BC_INFLOW_OUTFLOW, default 1 */
    int picard_iters;   /* 0 (default): one-shot velocity, Eqs. (v_(0))-(v_final).  k > 0: refine it
                           by k Picard iterations of the implicit velocity equation (Appendix F),
                           sweep and split kernels (one more launch per iteration on the split path) */
    double picard_omega; /* under-relaxation of those iterations, (0, 1], default 1 */
    int plane_scheme;    /* LBM_PLANES_*, default LBM_PLANES_NEEM */
    double wall_v_low[3];  /* LBM_BC_MOVING_WALLS: velocity of the wall at y = 0 (y component 0), default 0 */
    double wall_v_high[3]; /* and of the wall at y = ny-1 */
    int plane_density;     /* LBM_DENSITY_*, default LBM_DENSITY_CONTINUITY */
    int outlet;            /* LBM_OUTLET_*, default LBM_OUTLET_PRESSURE */
    int inlet_profile;     /* LBM_INLET_*, default LBM_INLET_UNIFORM */
    int lid_profile;       /* LBM_LID_*, default LBM_LID_UNIFORM */
    double lid_delta;      /* relative width of each lid taper, (0, 0.5], default 0.1 */
    int wait_probe;        /* test only, default 0.  1: the first in-place split step makes one block of
                              its collide kernel wait on a barrier that no copy will complete, so that
                              its bounded wait runs out (about 20 us, nothing in flight) and the step
                              reports LBM_E_TIMEOUT, sticky.  It exercises the failure path of the
                              kernels' bounded waits without a fault. */
    int streaming;         /* LBM_STREAM_*, default LBM_STREAM_AUTO */
    int tile_y;            /* tile height of the split kernels on an all-periodic grid with even nx:
                              rows of 64 nodes per block, 2, 4 or 8 forced; 0 (default): 4, or
                              the autotuner's choice when autotune is set.  A forced height on a
                              grid the heights do not apply to is LBM_E_UNSUPPORTED. */
    int autotune;          /* 1: lbm_create times steps at every candidate tile height (2, 4, 8, at
                              most ny) with CUDA events on the context stream, keeps the fastest (4
                              unless another is faster by more than 1 %) and re-initialises the
                              state; default 0 */
    const char* tune_cache; /* path of a JSON-lines file of the autotuner's choices (one object per
                               line: key, tile_y, candidates, ms_per_step; the last line of a key
                               wins), read before timing and appended to after it; NULL: none */
} lbm_params;

/* Fills *p with the defaults listed above. */
void lbm_default_params(lbm_params* p);

/* Creates a simulation.
 *   lattice        LBM_D2Q9 or LBM_D3Q27
 *   nx, ny, nz     grid size; nz = 1 for D2Q9; >= 3 on a periodic axis, >= 4 on a wall axis
 *   porosity       host, N doubles, 0 < eps <= 1 (Sec. 2)
 *   permeability   host, N doubles, kappa > 0, +INF marks free fluid (mu_D = mu_F = 0)
 *   forchheimer    F_eps >= 0 of Eq. (mu_F_Ergun_perm), or LBM_F_ERGUN
 *   viscosity      nu_f > 0, the fluid viscosity of Eq. (mu_D_Ergun_perm);
 *                  nu_eff = J_nu nu_f sets beta by Eq. (nu_eff_def)
 *   force          host, 3 doubles, body acceleration b (z ignored for D2Q9)
 *   opt            NULL for defaults
 * Computes mu_D, mu_F, grad eps and the Hessian of eps, and initialises the
 * populations by Eq. (eq_bc_f_bar) from (rho0, v0) with a_0 and Phi_0 of the
 * initial fields (flowchart of Sec. 3.5).  Synchronous.  On failure *out is
 * NULL and nothing is leaked. */
int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, const double* porosity,
               const double* permeability, double forchheimer, double viscosity, const double force[3],
               const lbm_params* opt);

/* Re-initialises the populations from per-node initial fields: rho0 (host, N)
   and superficial v0 (host, 3*N, component-major: v0[a*N + n]), either may be
   NULL for the uniform defaults.  Synchronous. */
int lbm_init_fields(lbm_ctx* ctx, const double* rho0, const double* v0);

/* Advances n >= 0 steps, asynchronously on the context stream.  Returns a
   launch error at once, or LBM_E_DIVERGED / LBM_E_TIMEOUT if the sticky device
   flag was seen set at an earlier synchronisation. */
int lbm_step(lbm_ctx* ctx, long n);

/* Waits for the context stream; returns LBM_E_DIVERGED (or LBM_E_TIMEOUT) if any step so far
   produced rho <= 0, a non-finite value or |v|/eps > 0.5. */
int lbm_sync(lbm_ctx* ctx);

/* Intrinsic density rho (N) and superficial velocity v (3*N, component-major,
   z component zero for D2Q9) of the current state, Eqs.
   (transformed_density_moment), (v_(0))-(v_final).  Host buffers owned by the
   caller; either may be NULL.  Synchronous. */
int lbm_moments(lbm_ctx* ctx, double* rho, double* v);

/* The same fields written to caller-owned DEVICE buffers (FP64), enqueued on
   the context stream without synchronising. */
int lbm_moments_device(lbm_ctx* ctx, double* rho_dev, double* v_dev);

/* Copies the populations f_bar (Q*N doubles, f[i*N + n]) to / from host memory.
   Synchronous.  Setting encodes into the context's storage format. */
int lbm_get_populations(lbm_ctx* ctx, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Domain-wide FP64 reductions of the current state. */
typedef struct {
    double mass;        /* sum over nodes and populations of f_bar = sum eps rho */
    double mean_v[3];   /* mean superficial velocity over all nodes */
    double v2_sum;      /* sum |v|^2 over nodes */
    double dv2_sum;     /* sum |v - v_ref|^2 against the snapshot of lbm_reduce's last call with snapshot=1 */
    double residual;    /* sqrt(dv2_sum / v2 of the snapshot), Eq. (SS_convergence_L2) over the snapshot gap */
    double drag[3];     /* sum of the Darcy-Forchheimer sink rho (mu_D + mu_F |v|) v */
    double k_app[3];    /* apparent permeability nu_f <v_a> / b_a (0 where b_a = 0) */
    long steps;         /* steps taken since creation */
} lbm_stats;

/* Fills *st (synchronous).  snapshot = 1 also stores the current v as the
   reference for the next call's residual. */
int lbm_reduce(lbm_ctx* ctx, lbm_stats* st, int snapshot);

/* Bytes of population and static-field traffic one node update needs at
   minimum (populations read + written, porosity and permeability read), the
   number of kernel launches one step issues, the kernel in use and whether
   the populations stream in place (1: one array) or not (0).  Any output
   pointer may be NULL. */
int lbm_info(const lbm_ctx* ctx, double* bytes_per_node_update, int* launches_per_step, int* kernel_in_use,
             int* in_place);

/* The tile height the context's split kernels use and how it was chosen.
 *   *tile_y        rows of 64 nodes per block (4 where the heights do not apply)
 *   *n, tiles, ms  the candidates timed by the autotuner and their ms per step
 *                  (n = 0 unless timed now); tiles and ms hold up to 8 entries
 *   *source        0 default or forced, 1 timed at creation, 2 from the cache file
 * Any output pointer may be NULL.  The tile height changes no arithmetic: every
 * height computes the same values. */
int lbm_tuning(const lbm_ctx* ctx, int* tile_y, int* n, int* tiles, double* ms, int* source);

/* The autotuner's cache file, host only (no device work).  lookup sets
 * *tile_y to the choice stored for key (the last line that names it) or 0 when
 * the file or the key is absent; lines that do not parse are skipped.  store
 * appends one line for key.  key: printable, no '"' or '\\'.  Errors:
 * LBM_E_INVALID for a NULL argument, a bad key or height, or (store) a file
 * that cannot be opened for appending. */
int lbm_tune_cache_lookup(const char* path, const char* key, int* tile_y);
int lbm_tune_cache_store(const char* path, const char* key, int tile_y, int n, const int* tiles, const double* ms);

/* Measurement: advances n steps exactly like lbm_step, with a CUDA event
 * recorded on the context stream before the first kernel of every step and
 * after each of its kernels, then synchronises.  ms_per_launch[k] receives the
 * mean device time of the k-th kernel of a step (k < max_kernels) and
 * *kernels the number of kernels per step (fused: 1; split: 3; plus 1 when
 * inlet / outlet planes are rebuilt).  The sweep kernels are not covered
 * (LBM_E_UNSUPPORTED).  Not a physics operation of the paper. */
int lbm_time_kernels(lbm_ctx* ctx, long n, double* ms_per_launch, int max_kernels, int* kernels);

/* Continuous-batching server for many independent D3Q27 cases (a host-side
 * runtime around the split kernels; the paper describes single cases only).
 * Requests are queued by lbm_server_submit (inputs copied) and admitted in
 * arrival order while their device footprint fits under hbm_cap_bytes; each
 * case streams in place (one population array).  The admitted cases below
 * 2^20 nodes advance by one launch of each of the three split kernels per step
 * over all of them (a block finds its case in a device case table); a case of
 * 2^20 nodes or more, which fills the GPU on its own, runs the single-case
 * kernels.  The check_every steps of a batch, for every case, are captured in
 * one CUDA graph.  After each
 * batch every case's relative L2 velocity change over the batch
 * (Eq. (SS_convergence_L2) over check_every steps) is compared with its tol;
 * converged, floor-limited, diverged or step-capped cases retire, freeing
 * memory for the queue.  A case's arithmetic does not depend on the other
 * cases in the batch.  Cases are periodic boxes with nx a multiple of 8;
 * storage FP32, FP16 or BF16; defaults (RT, J_nu, J_eta, corrections, device,
 * rho0) come from `defaults` (NULL for the library defaults).  Synchronous on
 * the calling thread. */
typedef struct lbm_server lbm_server;
/* Status of a case whose residual stopped decreasing above tol while its mean
   flow has settled: the smallest residual of its last 5 batches is no better
   than 0.9x the smallest of the 5 before, and the mean superficial velocity
   along the force changed by at most 10 tol (relative) over the last batch.
   Storage rounding sets such a residual floor (about 3e-6 for FP32 and 5e-4
   for FP16 storage at |v| ~ 1e-3, proportionally higher for slower flows);
   the domain mean, hence K_app, is far less sensitive to it. */
#define LBM_RETIRED_AT_FLOOR 1
typedef struct {
    long long id;        /* ticket of lbm_server_submit */
    int status;          /* LBM_OK converged below tol, LBM_RETIRED_AT_FLOOR, LBM_E_DIVERGED,
                            LBM_E_INVALID step cap reached, LBM_E_NOMEM too large */
    long steps;          /* steps taken */
    double residual;     /* last relative L2 velocity change over check_every steps */
    double mean_v[3];    /* mean superficial velocity at retirement */
    double k_app;        /* apparent permeability nu_f <v . b/|b|> / |b| */
    double submit_time;  /* seconds on the server clock */
    double finish_time;
} lbm_case_result;

int lbm_server_create(lbm_server** out, int storage, double hbm_cap_bytes, int check_every, const lbm_params* defaults);
/* Queues one case; *ticket receives its id. */
int lbm_server_submit(lbm_server* server, int nx, int ny, int nz, const double* porosity, const double* permeability,
                      double forchheimer, double viscosity, const double force[3], double tol, long max_steps,
                      long long* ticket);
/* Admits what fits, runs up to `batches` batches, and returns the cases that
   retired (up to max_results; LBM_E_INVALID if more finished), the number still
   running and the number queued. */
int lbm_server_run(lbm_server* server, int batches, lbm_case_result* results, int max_results, int* n_results,
                   int* n_active, int* n_queued);
/* Seconds since the server was created (the clock of submit_time / finish_time). */
double lbm_server_clock(const lbm_server* server);
/* Device bytes admitted now, batched kernel launches and node updates so far. */
int lbm_server_stats(const lbm_server* server, double* used_bytes, long long* kernel_launches, long long* node_updates);
void lbm_server_destroy(lbm_server* server);

/* Checkpoint.  lbm_save writes the grid, the parameters, porosity,
 * permeability, the step count and the raw stored populations to `path`;
 * lbm_load re-creates the context from such a file and continues bit for bit
 * (the next steps equal those of the saved context).  `runtime` supplies the
 * stream, device and allocator of the new context (NULL for defaults); its
 * other fields are ignored.  Both synchronous.  The residual snapshot of
 * lbm_reduce is not saved. */
int lbm_save(const lbm_ctx* ctx, const char* path);
int lbm_load(lbm_ctx** out, const char* path, const lbm_params* runtime);

/* Population sums computed without allocating anything.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory -- code running while a CUDA stream is captured into a graph,
 * where allocation calls are not allowed, and applications that give all
 * device memory to their own pool and forbid libraries to take more.
 *   lattice   LBM_D2Q9 or LBM_D3Q27
 *   n_nodes   N, 1 <= N <= LBM_NOALLOC_MAX_NODES
 *   f_dev     device, Q*N doubles, f[i*N + n] in the velocity order above (the
 *             layout lbm_get_populations returns), owned by the caller
 *   out_dev   device, 4 doubles, owned by the caller: sum over nodes and
 *             populations of f (the mass lbm_reduce reports), then the sum of
 *             c_i f per axis (z component 0 for D2Q9)
 *   stream    cudaStream_t to enqueue on (NULL = legacy default stream); the
 *             call returns without waiting
 * The partial sums live in one fixed device array of LBM_NOALLOC_MAX_NODES/256
 * rows of 4 doubles (2 MiB), held by every GPU that loads the library until
 * the process exits.  Every call made while `stream` is not being captured
 * looks up that array's device address (so a device reset, which moves it,
 * needs no action from the caller); a call made during a capture uses the
 * address an earlier call on the same device found, so make one call before
 * any stream capture begins.  All calls share the array (each call overwrites
 * the rows it reads, so no clearing is needed); calls that overlap on the GPU
 * race and must be ordered by the caller.  Returns LBM_OK, LBM_E_INVALID (bad
 * lattice, N out of range, NULL pointer) or LBM_E_CUDA when one of its own
 * launches or lookups fails; it neither reads nor clears the CUDA runtime's
 * last-error state left by the caller's earlier work, and it does not set
 * lbm_last_error. */
#define LBM_NOALLOC_MAX_NODES 16777216LL
int lbm_population_sums_noalloc(int lattice, long long n_nodes, const double* f_dev, double* out_dev, void* stream);

/* Frees every resource of ctx; NULL is a no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failing call on this thread (empty string if none). */
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H_ */
