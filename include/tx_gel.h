/*
 * tx_gel.h -- C ABI of the GB300 gelpad IPC step library (libtxgel.so).
 *
 * One implicit time step of a GelSight gelpad pressed by a kinematic rigid indenter, solved as an
 * incremental-potential-contact minimisation.  TacEx (arXiv 2411.04776), Sec. "General GIPC
 * Simulation Pipeline": each GIPC step first sets the kinematic targets (here: the indenter pose)
 * and then runs the solver that computes the new positions of the free gel vertices; the solver
 * is IPC [Li et al. 2020] (TacEx App. A "Choice of the Simulation Methods": intersection- and
 * inversion-free).  Per step the library minimises
 *
 *   E(x) = sum_i m_i |x_i - xt_i|^2 / (2 h^2) + sum_t V_t Psi_NH(F_t) + kappa sum_k b(d_k),
 *   Psi_NH(F) = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 ln^2 J,   b(d) = -(d - dhat)^2 ln(d/dhat),
 *
 * (xt = x_n + h v_n) by projected Newton: PSD-projected per-tet and per-contact Hessians, a
 * block-Jacobi PCG direction, a step capped by additive CCD and det F > 0, and backtracking.
 *
 * Conventions (all entry points):
 *   - SI units, FP64 at the boundary; arrays are row-major AoS (vertex k at [3k, 3k+3)).
 *   - Host pointers unless an argument says "device".  The library copies every input it keeps;
 *     the caller keeps ownership of all arrays it passes.
 *   - A `stream` argument is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *     device work of a handle is ordered on that stream.  Calls on one handle must not overlap
 *     (thread-compatible, not thread-safe); distinct handles are independent.
 *   - Errors are returned as tx_status; no exception crosses the ABI.  A failed step leaves the
 *     state at x_n (steps are transactional).  TX_ERR_CUDA reports a CUDA runtime error; its text
 *     is available from tx_last_error().
 */
#ifndef TX_GEL_H
#define TX_GEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tx_status {
  TX_OK = 0,
  TX_ERR_ARG = 1,            /* invalid argument (null pointer, size, index out of range)      */
  TX_ERR_OOM = 2,            /* device or host allocation failed                               */
  TX_ERR_MESH_INVERTED = 3,  /* a rest tetrahedron has non-positive volume                     */
  TX_ERR_INFEASIBLE = 4,     /* indenter placement penetrates the gel even after step splitting */
  TX_ERR_NEWTON_MAXIT = 5,   /* Newton iteration cap reached                                   */
  TX_ERR_PCG_MAXIT = 6,      /* PCG iteration cap reached (only if params ask to fail on it)   */
  TX_ERR_LINESEARCH = 7,     /* backtracking found no energy decrease above 1e-12 alpha_0       */
  TX_ERR_CCD_MAXIT = 8,      /* ACCD iteration cap reached                                     */
  TX_ERR_CUDA = 9,           /* CUDA runtime error (see tx_last_error)                         */
  TX_ERR_DEVICE_TIMEOUT = 10 /* a bounded device-side wait gave up (kernel returned early)     */
} tx_status;

typedef enum tx_precision {
  TX_PREC_FP64 = 0,  /* every step of the solve in FP64                                         */
  TX_PREC_MIXED = 1  /* elastic Hessian blocks + PCG matvecs in FP32 with FP64 residual
                        refinement; gradient, barrier, CCD and line-search energy stay FP64      */
} tx_precision;

/* Solver parameters.  tx_params_default() fills the values used by the GelSight workloads. */
typedef struct tx_params {
  double dhat;          /* barrier activation distance d_hat [m] (default 1e-4)                 */
  double kappa;         /* barrier stiffness [N/m]; <= 0 selects E * mean gel surface edge length */
  double newton_tol;    /* stop when ||p||_inf / h < newton_tol * (rest bbox diagonal) [1/s]     */
  double pcg_rel_tol;   /* PCG stops at ||r|| <= pcg_rel_tol * ||g|| (inexact Newton, 1e-3) near
                           convergence: when the next ||p||_inf, predicted from the last one and
                           the last contraction ratio, is below twice the Newton tolerance, and
                           always for the direction that ends the solve                        */
  double pcg_rel_tol_far; /* forcing term of the other Newton iterations (default 0.1); values
                           at or below pcg_rel_tol give a fixed forcing term                  */
  double gravity[3];    /* body acceleration [m/s^2] (default 0)                                 */
  int32_t newton_max_iter;  /* default 200                                                     */
  int32_t pcg_max_iter;     /* default 2000; hitting it keeps the direction (still descent)     */
  int32_t ls_max_halvings;  /* default 60                                                      */
  int32_t accd_max_iter;    /* default 1000000                                                 */
  int32_t max_split_depth;  /* infeasible indenter moves are halved up to this depth (4)       */
  int32_t precision;        /* tx_precision                                                     */
  int32_t refine_max;       /* mixed precision: max FP64 residual refinement rounds (3)         */
  int32_t pcg_cta_slices;   /* PCG work split: at least this many 32-row slices per CTA; 0 picks
                               the default (4); -1 autotunes it per class of active gel sets
                               (timed on live Newton rounds; the split changes the order of the
                               PCG's sums, so tuned runs are not bitwise reproducible)          */
  int32_t pcg_plan;         /* PCG kernel family: 0 automatic (the resident kernels, which keep the
                               matrix in shared memory, whenever the gels fit them; otherwise the
                               streaming kernels, which stream it from HBM: per-gel CTA groups
                               below 32 gels being solved, the pool of one CTA per SM that
                               re-splits the gels still iterating from 32 on); 1 always the
                               per-gel-group streaming kernels; 2 always the pooled streaming
                               kernels (1 and 2: tests and measurements of one family).  A handle
                               takes the largest value any of its gels asks for.               */
  int32_t pcg_coarse_off;   /* 1: no coarse space in the streaming FP64 PCG.  0 (default): a
                               solve of one gel with a body held by no vertex adds an exact solve
                               on that body's six rigid motions to block-Jacobi (two-level additive
                               preconditioner for the free bodies of tx_gel_desc's meshes)      */
  double friction;          /* IPC lagged friction coefficient mu_f between gel and indenter
                               (0: frictionless, the default).  Pairs in contact at the start of a
                               (sub)step fix their closest points, tangent plane and normal force
                               lambda = kappa |b'(d)|; the step then adds
                               D = mu_f lambda f0(|tangential relative displacement|), f0 the
                               smoothed Coulomb law of IPC (TacEx App. A: IPC models static and
                               dynamic friction)                                               */
  double friction_eps_v;    /* velocity below which friction acts as a stiff spring (static
                               friction) [m/s] (default 1e-3)                                  */
  double kappa_adapt_max;   /* adaptive barrier stiffness (IPC's kappa update, applied between
                               steps: the indenter is placed before each solve, so pairs close in
                               between steps): 0 keeps kappa fixed (the default); else, after a
                               step whose final smallest pair distance is below kappa_adapt_dmin
                               and below that of the step before, kappa doubles for the next
                               steps, up to kappa_adapt_max times its initial value (>= 1).
                               Reset and set_state return kappa to its initial value           */
  double kappa_adapt_dmin;  /* that distance threshold [m] (> 0 when kappa_adapt_max > 0)     */
} tx_params;

void tx_params_default(tx_params* p);

/* One gel + indenter scene.  The gel is a tet mesh (rest positions, positively oriented tets,
 * Dirichlet mask: 1 = vertex held at its rest position).  The indenter is a rigid triangle mesh
 * given in its own frame, placed in the world by a pose (qw, qx, qy, qz, tx, ty, tz).
 * The tet mesh may hold up to 4 deformable bodies (its connected components through the tets,
 * numbered in the order of their first vertex; all of one material): their surfaces then also
 * touch each other through the same barrier (GIPC's soft-to-soft contact, TacEx Sec. 2: every
 * surface vertex against every surface triangle of another body, every two surface edges of
 * different bodies), without friction and without counting in contact_force.  Body 0 is the
 * gelpad: the marker and height-map readouts use its top surface only.  More than 4 bodies is
 * TX_ERR_ARG, and so is mixed precision for a mesh with a body held by no vertex (its rigid
 * motions, resisted by its mass alone, are beyond the FP32 inner solves: use FP64). */
typedef struct tx_gel_desc {
  int32_t n_verts;
  const double* verts;       /* n_verts x 3 rest positions [m]                                  */
  int32_t n_tets;
  const int32_t* tets;       /* n_tets x 4 vertex ids                                           */
  const uint8_t* dirichlet;  /* n_verts; may be NULL (no fixed vertex)                          */
  double young;              /* Young's modulus E [Pa]                                          */
  double poisson;            /* Poisson ratio nu (< 0.5)                                        */
  double density;            /* rho [kg/m^3]                                                    */
  int32_t n_ind_verts;
  const double* ind_verts;   /* n_ind_verts x 3, indenter frame [m]                             */
  int32_t n_ind_tris;
  const int32_t* ind_tris;   /* n_ind_tris x 3                                                  */
  double ind_pose[7];        /* initial indenter pose                                           */
  tx_params params;
} tx_gel_desc;

/* Per-step record (last completed step of a gel). */
typedef struct tx_step_stats {
  int32_t newton_iters;     /* accepted Newton updates over all substeps                        */
  int32_t pcg_iters;        /* total PCG iterations                                             */
  int32_t ls_halvings;      /* total line-search halvings                                       */
  int32_t substeps;         /* solves run (1 unless the indenter move had to be split)           */
  int32_t active_pairs;     /* contact pairs with d < d_hat at the final state                  */
  int32_t candidate_pairs;  /* broad-phase candidates at the final state                        */
  int32_t refine_rounds;    /* mixed precision: FP64 refinement rounds used                      */
  int32_t status;           /* tx_status of the step                                            */
  double energy;            /* E at the final state                                             */
  double min_distance;      /* smallest candidate-pair distance at the final state [m]          */
  double contact_force[3];  /* force of the indenter on the gel, -kappa sum grad b [N]           */
  double mean_position[3];  /* mean of the gel vertex positions (TacEx "object position") [m]    */
  double kappa;             /* barrier stiffness for the next step [N/m] (tx_params.kappa_adapt_max) */
  int32_t soft_pairs_cut;   /* several bodies: Newton assemblies of a soft-soft pair whose blocks
                               between the two bodies found no spare matrix position and were left
                               out (the matrix stays PSD; the solve only converges more slowly)  */
  int32_t reserved1;
} tx_step_stats;

typedef struct tx_gel tx_gel;     /* opaque single-gel handle                                  */
typedef struct tx_batch tx_batch; /* opaque many-gel handle                                    */

const char* tx_status_str(tx_status s);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* tx_last_error(void);

/* ---------------- single gel ---------------- */

/* TacEx Sec. "General GIPC Simulation Pipeline" (set-up: a simulated object becomes a GIPC object
 * from its tetrahedral mesh before the first step).  Validates and copies the description,
 * precomputes rest data (Dm^-1, volumes, lumped masses, surface, BSR pattern), allocates device
 * memory and uploads.  The handle owns everything it allocates until tx_gel_destroy.  Returns
 * TX_ERR_MESH_INVERTED if a rest tet has det(Dm) <= 0, TX_ERR_ARG on bad sizes/indices or
 * parameters, TX_ERR_OOM (nothing left allocated) if device or pinned host memory runs out. */
tx_status tx_gel_create(const tx_gel_desc* desc, void* stream, tx_gel** out);

/* TacEx Sec. "General GIPC Simulation Pipeline": one GIPC step -- the kinematic target (here the
 * indenter pose) is set, then the solver moves the free gel vertices (the incremental-potential
 * minimisation above; App. A "Choice of the Simulation Methods": intersection- and inversion-
 * free).  Advances one time step of length dt with the indenter moving (linearly in position,
 * along the short arc in rotation) from its current pose to `pose`; a move whose sweep would hit
 * the gel is split into half steps.  Blocks until the step has finished; on error the state stays
 * at the step's start. */
tx_status tx_gel_step(tx_gel* g, const double pose[7], double dt);

/* TacEx Sec. "General GIPC Simulation Pipeline" (GIPC attachments): each step first sets the
 * attachment targets from the sensor-case pose, then solves.  Like tx_gel_step, with the gel's
 * attached (Dirichlet) vertices also moving, with their frame, from the current case pose to
 * `case_pose`: at the end of the step each sits at its rest position carried by case_pose (a pose
 * (qw, qx, qy, qz, tx, ty, tz) of the frame the rest mesh is given in; the identity at create and
 * after a reset).  The attached vertices are placed before the indenter placement check; a split
 * step halves the case motion with the indenter's; their velocity is their displacement over the
 * step.  Blocks until the step has finished; on error the state, the indenter pose and the case
 * pose stay at the step's start. */
tx_status tx_gel_step_attached(tx_gel* g, const double pose[7], const double case_pose[7], double dt);

/* The current case pose of an attachment-driven gel (identity if none was ever given). */
tx_status tx_gel_case_pose(const tx_gel* g, double case_pose[7]);

/* TacEx Sec. "General GIPC Simulation Pipeline": after each step the vertex positions update the
 * rendered gel mesh and their mean is the object position.  Reads the state: x, v (n_verts x 3,
 * may be NULL), contact force (3, may be NULL) and the last step's statistics (may be NULL; its
 * mean_position is that mean).  If device_ptrs != 0, x and v are device pointers and the copy is
 * enqueued on the gel's stream (ordered after the last step); otherwise host pointers and the
 * call returns after the copy.  The caller owns the output arrays. */
tx_status tx_gel_state(const tx_gel* g, double* x, double* v, double f_contact[3],
                       tx_step_stats* stats, int32_t device_ptrs);

/* Checkpoint / restore of x, v (host arrays, n_verts x 3) and the indenter pose. */
tx_status tx_gel_get_state(const tx_gel* g, double* x, double* v, double pose[7]);
tx_status tx_gel_set_state(tx_gel* g, const double* x, const double* v, const double pose[7]);

/* TacEx Sec. "General GIPC Simulation Pipeline" (reset for RL): x = rest positions, v = 0, the
 * indenter back at its initial pose. */
tx_status tx_gel_reset(tx_gel* g);

void tx_gel_destroy(tx_gel* g);

/* Device bytes a gel created from `desc` will hold (for admission control). */
size_t tx_gel_footprint_bytes(const tx_gel_desc* desc);

/* Evaluates E at the positions x (host, n_verts x 3) with predictor xt (host), step h and the
 * indenter at `pose`, on the device.  parts = [inertia, elastic, barrier, min distance, active
 * pairs] (may be NULL).  Does not change the state. */
tx_status tx_gel_energy(tx_gel* g, const double* x, const double* xt, double h,
                        const double pose[7], double* energy, double parts[5]);

/* Gradient of E (host out, n_verts x 3, Dirichlet rows included) and contact force at x. */
tx_status tx_gel_gradient(tx_gel* g, const double* x, const double* xt, double h,
                          const double pose[7], double* grad, double f_contact[3]);

/* ---------------- many gels (batched, continuous) ---------------- */

/* Creates one handle over n gels of any sizes; all state stays resident on the device. */
tx_status tx_batch_create(const tx_gel_desc* descs, int32_t n, void* stream, tx_batch** out);
void tx_batch_destroy(tx_batch* b);
int32_t tx_batch_size(const tx_batch* b);

/* Steps every gel once (poses: n x 7, dts: n) and blocks until all finished.  statuses: n. */
tx_status tx_batch_step(tx_batch* b, const double* poses, const double* dts, tx_status* statuses);
/* tx_batch_step with every gel attachment-driven as in tx_gel_step_attached (case_poses: n x 7;
 * NULL: a plain tx_batch_step). */
tx_status tx_batch_step_attached(tx_batch* b, const double* poses, const double* case_poses, const double* dts,
                                 tx_status* statuses);

/* Continuous batching.  submit() queues one step request for each listed gel (a gel may hold
 * at most one request in flight: TX_ERR_ARG otherwise); the request is admitted at the next
 * Newton-iteration boundary.  advance() runs one Newton iteration for every admitted gel and
 * reports the gels whose step finished (done_ids/done_status: capacity n each). */
tx_status tx_batch_submit(tx_batch* b, int32_t count, const int32_t* ids, const double* poses,
                          const double* dts);
tx_status tx_batch_advance(tx_batch* b, int32_t* n_done, int32_t* done_ids,
                           tx_status* done_status);
/* Number of gels with a request submitted or in flight. */
int32_t tx_batch_pending(const tx_batch* b);

tx_status tx_batch_state(const tx_batch* b, int32_t gel, double* x, double* v,
                         double f_contact[3], tx_step_stats* stats);
tx_status tx_batch_set_state(tx_batch* b, int32_t gel, const double* x, const double* v,
                             const double pose[7]);
tx_status tx_batch_reset(tx_batch* b, int32_t gel);

/* ---------------- gel-surface readout ----------------
 * For the tactile simulation that consumes the physics state (TacEx, Sec. "Tactile Simulation":
 * height maps of the gel surface feed the optical simulation; App. "Marker Simulation": markers
 * tied to faces of the tet mesh follow the vertex positions of their facet).  The top surface is
 * the set of boundary triangles whose rest outward normal points up (+z).  Both calls read the
 * gel's current state (not while a request of the gel is in flight: TX_ERR_ARG), run on the
 * device and return when the host arrays are filled.
 *
 * Markers: n markers at rest points rest_xy (n x 2, [m]) of the top surface; each lies in a top
 * triangle of the rest mesh (the first in the surface order whose xy barycentric coordinates are
 * all >= -1e-12) and is carried by them to the current positions: out (n x 3); found[i] = 0 (and
 * out zero) for a point off the top surface.  n times the gel's top triangles must not exceed
 * 2^38 (TX_ERR_ARG). */
tx_status tx_gel_markers(tx_gel* g, int32_t n, const double* rest_xy, double* out, int32_t* found);
tx_status tx_batch_markers(tx_batch* b, int32_t gel, int32_t n, const double* rest_xy, double* out, int32_t* found);

/* Height map of the deformed top surface seen from above: out (ny x nx, row j = y) at pixel
 * centres (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy) holds the largest z [m] of the top triangles
 * covering the centre in the xy projection (barycentric coordinates >= -1e-12), NaN where none
 * does.  Rasterised by a CUDA kernel (no graphics API); nx * ny <= 2^26. */
tx_status tx_gel_height_map(tx_gel* g, int32_t nx, int32_t ny, double x0, double y0, double dx, double dy,
                            double* out);
tx_status tx_batch_height_map(tx_batch* b, int32_t gel, int32_t nx, int32_t ny, double x0, double y0, double dx,
                              double dy, double* out);

/* ---------------- per-phase device timing ----------------
 * With profiling enabled the library brackets each phase of the step with CUDA events on the
 * handle's stream and accumulates, per phase, the device time, the number of kernel launches and
 * the algorithmic work the phase performed (FP64-equivalent flops, counted per unit as documented
 * for each phase name).  tx_*_profile(h, enable, out): copies the counters accumulated since the
 * previous call into `out` (may be NULL), resets them and sets profiling on (enable = 1) or off. */
#define TX_PROFILE_MAX 12
typedef struct tx_profile {
  int32_t n_phases;
  int32_t reserved;
  const char* names[TX_PROFILE_MAX];
  double ms[TX_PROFILE_MAX];        /* summed event time per phase                               */
  int64_t launches[TX_PROFILE_MAX]; /* kernel launches per phase                                 */
  double flops[TX_PROFILE_MAX];     /* algorithmic flops per phase (0 where not counted)         */
  double bytes[TX_PROFILE_MAX];     /* algorithmic DRAM/L2 bytes per phase (0 where not counted) */
  int64_t pcg_iters;                /* PCG iterations (summed over gels)                         */
  int64_t newton_iters;             /* Newton iterations run (summed over gels)                  */
  int64_t kernel_launches;          /* every kernel this library launched (all handles)          */
  int64_t pcg_resident_launches;    /* PCG launches of the resident kernels (matrix in shared
                                       memory; counted whether or not profiling is on)            */
  int64_t pcg_streaming_launches;   /* PCG launches of the streaming kernels (matrix from HBM),
                                       both forms                                                */
  int64_t pcg_pool_launches;        /* of which launches of the pooled form                      */
} tx_profile;

tx_status tx_batch_profile(tx_batch* b, int32_t enable, tx_profile* out);
tx_status tx_gel_profile(tx_gel* g, int32_t enable, tx_profile* out);

/* ---------------- measurement ----------------
 * Peak rate of the plain (non-tensor) FMA pipe in FP64 (bits = 64) or FP32 (bits = 32): one launch
 * over every SM in which each thread runs four independent chains of `iters` FMAs, timed with
 * CUDA events on `stream` (the call waits for it).  *flops = 2 x the FMAs executed, *ms = the
 * launch's event time; flops / ms is the roofline denominator of the FP64-bound solver kernels.
 * No counterpart in the paper: it measures the device the solver runs on. */
tx_status tx_peak_fma(int32_t bits, int32_t iters, double* flops, double* ms, void* stream);

/* ---------------- fault injection (test hook) ----------------
 * Makes the library's own failure paths run without faulting the device.  kind 1: the device or
 * pinned-host allocation `count` allocations from now fails before it reaches the CUDA runtime
 * (the call that makes it returns TX_ERR_OOM and frees what it had allocated); kind 2: the PCG
 * launches of the next `count` Newton iterations (any handle) wait at their group barriers for an
 * arrival that never comes, with a short poll limit, so that every wait gives up and the step
 * returns TX_ERR_DEVICE_TIMEOUT with the state rolled back.  count 0 disarms a kind.  Returns
 * TX_ERR_ARG for an unknown kind or a negative count.  Process-wide; not for production use. */
#define TX_INJECT_ALLOC_FAIL 1
#define TX_INJECT_WAIT_TIMEOUT 2
tx_status tx_debug_inject(int32_t kind, int32_t count);

/* ---------------- unit-level kernels (device pointers, for parity checks and reuse) --------- */

/* Per-tet elastic energy V Psi, gradient (12) and Hessian (144, row-major; PSD-projected in the
 * deformation-gradient space if project != 0).  X, x: n x 12 (4 corners x 3), rest and current.
 * e: n, g: n x 12, H: n x 144; g and H may be NULL (energy only).  All device pointers. */
tx_status tx_eval_tets(int32_t n, const double* X, const double* x, double mu, double lambda,
                       int32_t project, double* e, double* g, double* H, void* stream);

/* Per-pair barrier b (without kappa), gradient (12) and Hessian (144) w.r.t. the 4 points of
 * each pair; kind 0: point P0 vs triangle P1..P3, kind 1: segment P0P1 vs segment P2P3 (IPC
 * edge-edge mollifier with threshold eps_x[i]).  If free_mask[i] != 0, the Hessian block on the
 * points whose bit is set is PSD-projected.  dtype[i] = [formula, i0..i3] (5 ints) of the closest
 * feature pair.  All device pointers; free_mask, dtype may be NULL. */
tx_status tx_eval_pairs(int32_t n, const int32_t* kind, const double* P, double dhat,
                        const double* eps_x, const int32_t* free_mask, double* b, double* g,
                        double* H, int32_t* dtype, void* stream);

/* Additive CCD per pair along P + t dP (n x 12 each), s = gap fraction (0.1), t in [0, tc].
 * hit[i]: 0 no hit, 1 hit (toi[i] set), 2 iteration cap.  Device pointers. */
tx_status tx_eval_accd(int32_t n, const int32_t* kind, const double* P, const double* dP,
                       double s, double tc, int32_t max_iter, double* toi, int32_t* hit,
                       void* stream);

/* Block-Jacobi preconditioned conjugate gradient for A x = b -- the linear solve of the projected
 * Newton step on its own.  A is symmetric positive definite with 3x3 blocks in block-CSR form:
 * row_ptr (n + 1), col_idx (nnzb), vals (9 nnzb, row-major blocks; every block row holds its
 * diagonal block).  b and x are 3n vectors; x0 = 0.  All array arguments are device pointers.
 * Stops when |r| <= rel_tol |b| or after max_iter iterations.  Allocates its scratch (~21 n
 * doubles of device memory) for the call, runs on `stream` and returns after the solve; the
 * iteration count and the final relative residual go to *iters and *rel_res (host, may be NULL).
 * TX_ERR_DEVICE_TIMEOUT if a bounded grid-wide wait gave up. */
tx_status tx_bsr_pcg(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                     const double* b, double* x, double rel_tol, int32_t max_iter, int32_t* iters,
                     double* rel_res, void* stream);

/* tx_bsr_pcg without any device allocation.  (This entry point has no counterpart in the paper; it
 * exists for callers of this library that must not allocate device memory while they run: a host
 * framework that owns every device allocation of a simulation step through its own pool or a
 * fixed memory budget, or a real-time control loop where cudaMalloc/cudaFree would synchronise
 * the device and stall the other streams.)  Same arguments and results as tx_bsr_pcg, for
 * n <= 65536 block rows; larger systems are rejected with TX_ERR_ARG (tx_last_error says why).
 * Like tx_bsr_pcg it waits for its stream to finish before returning (it reads the iteration
 * count back).  The scratch is one fixed array of about 11 MB inside the library's device module,
 * held by every GPU that loads the library until the process exits.  The first call in a CUDA
 * context (each device's primary context; a device reset makes a new one) looks up that array's
 * device address (cudaGetSymbolAddress) with the context current and keeps it for that context;
 * make that first call before any stream capture.  All calls on a device share the array: calls
 * that overlap on the GPU (on different streams or from different threads) race and give wrong
 * results; the counters a call needs zeroed are cleared by the call itself. */
tx_status tx_bsr_pcg_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                             const double* vals, const double* b, double* x, double rel_tol,
                             int32_t max_iter, int32_t* iters, double* rel_res, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TX_GEL_H */
