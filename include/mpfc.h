/*
 * mpfc.h -- C ABI of libmpfc, a GB300 (sm_103a) solver for the Modified Phase
 * Field Crystal equation by the convex-splitting finite-difference schemes of
 * Baskaran, Zhou, Hu, Wang, Wise and Lowengrub (arXiv:1208.2643), each time step
 * solved by a nonlinear FAS multigrid V-cycle.
 *
 * Problem (Sec. 2, (2.4) and (2.9)): d_tt phi + beta d_t phi = M Delta mu,
 *   mu = phi^3 + alpha phi + 2 Delta phi + Delta^2 phi, alpha = 1 - epsilon,
 * on a periodic m x n cell-centred grid of spacing h (App. A).
 *
 * Conventions for every entry point:
 *  - return value: MPFC_OK (0) or a negative MPFC_ERR_* status;
 *  - grid functions are double arrays of m*n values, row-major, f[j*m + i], i the
 *    x index; pointers are device pointers unless an argument says otherwise;
 *  - calls are ordered on the CUDA stream given to mpfc_create; entry points that
 *    return host results (mpfc_step, mpfc_step_cycles, mpfc_mass, mpfc_energy,
 *    mpfc_get_state to host memory) synchronise that stream before returning;
 *  - a handle allocates no device memory: everything lives in the workspace the
 *    caller passes to mpfc_create (size from mpfc_workspace_bytes), which the
 *    caller owns and must keep alive until mpfc_destroy.
 */
#ifndef MPFC_H
#define MPFC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPFC_OK 0
#define MPFC_ERR_INVALID (-1)       /* bad argument, grid size or parameter            */
#define MPFC_ERR_WORKSPACE (-2)     /* workspace too small or misaligned                */
#define MPFC_ERR_CUDA (-3)          /* a CUDA runtime call failed                       */
#define MPFC_ERR_NOT_CONVERGED (-4) /* max_cycles V-cycles without reaching tol         */
#define MPFC_ERR_DIVERGED (-5)      /* residual became non-finite or grew by > 1e10     */
#define MPFC_ERR_TOO_LARGE (-6)     /* grid larger than mpfc_mass_noalloc's static scratch allows */

#define MPFC_FP64 0       /* every V-cycle kernel in FP64                                  */
#define MPFC_FP32_INNER 1 /* FP64 outer defect correction around FP32 inner V-cycles       */

#define MPFC_LAUNCH_GRAPH 0  /* a time step is one CUDA graph with a device-side loop (default) */
#define MPFC_LAUNCH_STREAM 1 /* kernels launched one by one, loop decided on the host           */

#define MPFC_GUESS_PREV 0    /* phi^(0) = phi^k                                            */
#define MPFC_GUESS_EXTRAP 1  /* phi^(0) = 2 phi^k - phi^{k-1}                              */
#define MPFC_GUESS_LEARNED 2 /* extrapolation plus the learned correction (mpfc_set_guess_model),
                                 behind a residual gate on FP64 handles (mpfc_set_guess_gate)   */

/* Boundary conditions (App. A): periodic in both directions, (A.8)-(A.9); or, as in the
 * polycrystal run of Sec. 4.5, periodic in x and homogeneous Neumann in y with the ghost
 * rule (A.7), phi_{i,0} = phi_{i,1}, phi_{i,n+1} = phi_{i,n}, applied to phi, mu, kappa
 * on every multigrid level.  The Neumann rule is available for MPFC_FP64 handles with
 * the PREV or EXTRAP guess (not in batches). */
#define MPFC_BC_PERIODIC 0
#define MPFC_BC_NEUMANN_Y 1

/* Model: the MPFC damped wave equation (Sec. 1, (2)), or its purely parabolic special
 * case, the PFC equation d_t phi = M Delta mu (Sec. 1, (1)), solved by the same
 * convex-splitting schemes: row 1 of N reads phi - s M Delta_h mu and S1 = phi^k (no
 * velocity term); psi then holds the discrete velocity (phi^{k+1} - phi^k)/s. */
#define MPFC_MODEL_MPFC 0
#define MPFC_MODEL_PFC 1

typedef struct {
  int m, n;          /* cells in x and y; the hierarchy halves both while they stay even
                        and at least `coarsest` cells per side remain; m n <= 2^30 (the
                        kernels index cells in 32-bit ints) and n <= 65535 (rows are a
                        launch grid's y dimension)                                       */
  double h;          /* grid spacing (App. A), L_x = m h, L_y = n h                      */
  double M;          /* mobility (Sec. 2)                                                 */
  double epsilon;    /* alpha = 1 - epsilon (Sec. 2, (2.1))                               */
  double beta;       /* damping (Sec. 2, (2.4))                                           */
  double dt;         /* time step s (Sec. 3)                                              */
  int nu1, nu2;      /* red-black sweeps before / after the coarse-grid correction        */
  int coarsest;      /* minimum cells per side on the coarsest level (default 4)          */
  double omega;      /* relaxation of the smoother's cell update: 1 = App. B as printed   */
  double tol;        /* stop when sqrt(sum_{c,i,j} r_c^2 / (3 m n)) <= tol; both forms reach
                        the FP64 roundoff floor of the residual (about 1e-15 at h = 0.5,
                        1e-13 at h = 1/16 for O(0.1) fields): smaller tol cannot be met  */
  int max_cycles;    /* V-cycle limit per step                                            */
  int precision;     /* MPFC_FP64 or MPFC_FP32_INNER                                      */
  int guess;         /* MPFC_GUESS_*                                                      */
  int inner_cycles;  /* MPFC_FP32_INNER: FP32 V-cycles per FP64 outer iteration (0 = 2)   */
  int bc;            /* MPFC_BC_PERIODIC (default) or MPFC_BC_NEUMANN_Y                   */
  int pinning;       /* 1: reserve the pinning weight and target of Sec. 4.6 in the
                        workspace (mpfc_set_pinning); PREV/EXTRAP guess only (FP64 or
                        FP32-inner)                                                      */
  int model;         /* MPFC_MODEL_MPFC (default) or MPFC_MODEL_PFC                        */
} mpfc_params;

typedef struct {
  int cycles;        /* V-cycles taken (outer iterations for MPFC_FP32_INNER)             */
  int status;        /* MPFC_OK, MPFC_ERR_NOT_CONVERGED or MPFC_ERR_DIVERGED              */
  double res0;       /* scaled residual of the initial guess                              */
  double res_final;  /* scaled residual when the step stopped                             */
} mpfc_step_info;

typedef struct {
  double F;          /* F(phi^k), Sec. 3 (3.1)                                            */
  double pseudoF;    /* F + ||psi^k||_{-1}^2 / (2M), Sec. 3 (3.2); F for the PFC model     */
  double tildeF;     /* pseudoF + ||grad_h(phi^k - phi^{k-1})||^2 / 2, Sec. 3.4 (3.26)     */
  double pinning;    /* h^2 sum W (phi^k - phihat)^2, the pinning energy of Sec. 4.6 (0 if
                        pinning is off); not included in F, pseudoF, tildeF              */
} mpfc_energy_t;

typedef struct mpfc_s mpfc_t;

/* Fills p with the defaults: 64 x 64, h = 0.5, M = 1, epsilon = 0.025, beta = 0.9,
 * dt = 0.01, V(2,2), coarsest 4, omega = 0.8, tol = 1e-10, max_cycles = 100, FP64,
 * extrapolated guess. */
void mpfc_default_params(mpfc_params* p);

/* Workspace bytes a handle with these parameters needs (0 if the parameters are
 * invalid).  The workspace must be device memory aligned to 256 bytes. */
size_t mpfc_workspace_bytes(const mpfc_params* p);

/* Creates a solver handle on `cuda_stream` (a cudaStream_t; NULL = legacy stream).
 * The state is phi = 0, psi = 0 until mpfc_set_state.  Returns MPFC_ERR_INVALID for
 * bad parameters, MPFC_ERR_WORKSPACE if `bytes` is short or d_workspace misaligned. */
int mpfc_create(const mpfc_params* p, void* d_workspace, size_t bytes, void* cuda_stream, mpfc_t** out);

/* Releases the handle (its CUDA graphs and host memory; not the workspace). */
void mpfc_destroy(mpfc_t* h);

/* Sets the time-level state (phi^k, phi^{k-1}, psi^k) of Sec. 3.1/3.2 by copying.
 * phi_prev NULL means phi^{-1} = phi^0 and psi NULL means psi^0 = 0, the start-up
 * rule of Sec. 3.2.  Pointers may be host or device memory. */
int mpfc_set_state(mpfc_t* h, const double* phi, const double* phi_prev, const double* psi);

/* Copies the state out; any pointer may be NULL; host or device memory. */
int mpfc_get_state(mpfc_t* h, double* phi, double* phi_prev, double* psi);

/* Advances nsteps steps of scheme 1 (first order, Sec. 3.1, (3.6)-(3.9)) or scheme 2
 * (second order, Sec. 3.2, (3.12)-(3.15)).  Each step builds the FAS source S of
 * App. B.1/B.2, runs V-cycles until the scaled residual is at or below tol, and
 * updates psi by (3.9) or (3.15).  A step that ends NOT_CONVERGED or DIVERGED leaves
 * the state at the last good step and stops the remaining steps of the call; the
 * first such status is returned.  per_step (nullable, nsteps entries, host memory)
 * receives each step's record.  Synchronises the stream. */
int mpfc_step(mpfc_t* h, int scheme, int nsteps, mpfc_step_info* per_step);

/* Enqueues nsteps steps on the handle's stream and returns without synchronising.
 * Each step appends its record to a device-side log of 1024 entries (later records
 * are counted but not kept); a failing step halts the steps after it until
 * mpfc_records or mpfc_set_state.  Graph construction on the first call of a scheme
 * must not happen inside a stream capture. */
int mpfc_step_async(mpfc_t* h, int scheme, int nsteps);

/* Synchronises, copies up to max_records step records (oldest first) to `out`
 * (host, nullable), stores the number of steps logged since the last call in
 * *count (nullable), clears the log and the halt flag, and returns the first
 * failing status among the copied records (MPFC_OK if none). */
int mpfc_records(mpfc_t* h, mpfc_step_info* out, int max_records, int* count);

/* Chooses how steps are launched.  MPFC_LAUNCH_GRAPH replays one CUDA graph per step
 * whose conditional WHILE node runs the V-cycles until the device-side residual test
 * fails.  MPFC_LAUNCH_STREAM launches the same kernels in the same order on the
 * stream and reads the loop decision back after each cycle (for profilers and
 * debuggers that cannot look inside conditional graph nodes); with it mpfc_step_async
 * synchronises once per V-cycle. */
int mpfc_set_launch_mode(mpfc_t* h, int mode);

/* Kernel launches of one FP64 time step (handles with precision MPFC_FP64 and an
 * analytic guess; MPFC_ERR_INVALID otherwise): *per_step launches besides the
 * V-cycles, plus *per_cycle for each V-cycle, under the handle's current launch shape.
 * Either pointer may be null. */
int mpfc_launch_counts(const mpfc_t* h, int scheme, int* per_step, int* per_cycle);

/* Measurement helper of the mixed-precision form: times `sweeps` red-black FP32
 * sweeps of the correction equation (as the inner cycles run them, mpfc_set_fp32_sweep)
 * on level `level` of a handle
 * created with precision MPFC_FP32_INNER, whatever its planes hold, between CUDA events
 * on the handle's stream, and writes the milliseconds to *ms (host).  Synchronises.
 * The planes' contents change; call mpfc_set_state before stepping again. */
int mpfc_fp32_time_smooth(mpfc_t* h, int level, int sweeps, float* ms);

/* How the mixed-precision form's inner red-black sweeps run on levels launched per
 * level (a tuning choice: results do not depend on it, bit for bit).  tile_rows 0: each
 * sweep is two launches, one per colour, updating e in place.  tile_rows 4, 8, 16 or
 * 32: on levels of at least min_cells cells whose width is a multiple of 4, each sweep
 * is one launch over tiles of 64 x tile_rows cells staged in shared memory (e with a
 * two-cell halo), reading e from one copy in the workspace and writing the other, in
 * pairs so that e ends where it started.  Default: 16 rows on levels of at least
 * 2048 x 2048 cells, whose planes do not stay in L2 between sweeps (there the tiled
 * sweep reads each plane once instead of twice; smaller levels, served from L2, run
 * faster as two launches).  Drops
 * the handle's captured graphs.  MPFC_ERR_INVALID for other values or handles that are
 * not MPFC_FP32_INNER. */
int mpfc_set_fp32_sweep(mpfc_t* h, int tile_rows, int min_cells);

/* Test hook of the tiled FP32 sweep's failure handling (no counterpart in the paper; for
 * tests of its bounded waits without a GPU fault).  withhold = 1: in every following
 * tiled sweep, the tensor copies that stage tile (1, 1) (columns 64..127, the second
 * row of tiles) are not issued (no memory is touched out of bounds) when that tile is
 * staged by tensor copies, so the owning CTA's wait runs out after spin_cycles clock
 * cycles; the CTA then writes NaN into all its remaining output tiles and returns, and
 * the step's defect is not finite: the step reports MPFC_ERR_DIVERGED and keeps its
 * state.  withhold = 0, spin_cycles = 0 restore normal operation (waits limited to about
 * 1 s).  Process-wide, synchronous.  MPFC_ERR_INVALID for other values. */
int mpfc_fp32_test_withhold_copy(int withhold, long long spin_cycles);

/* Launch shapes of the time step's per-cell kernels (a tuning choice: results do not
 * depend on it).  Launches of at least small_cells cells use blocks of 32 x rows
 * threads (rows 1, 2, 4 or 8), smaller ones one-warp blocks; grids of at most
 * pdl_blocks blocks are launched with programmatic dependent launch (0: none).  The
 * V-cycle's levels of at most tail_cells cells (0: none) run as one launch: for the
 * FP64 path of one CTA (tail_ctas 1) or of a thread-block cluster of tail_ctas CTAs (8,
 * or 16 where the GPU can hold such a cluster), for the FP32 inner cycles of one CTA
 * with the levels in shared memory.  Drops the handle's captured graphs (rebuilt on the
 * next step).  Returns MPFC_ERR_INVALID for other values. */
int mpfc_set_launch_shape(mpfc_t* h, int rows, int small_cells, int pdl_blocks, int tail_cells, int tail_ctas);

/* Thread layout of the FP64 V-cycle's grid transfers (App. B: the FAS restriction of u and
 * of the residual, and the bilinear prolongation of the correction; a tuning choice:
 * results do not depend on it, bit for bit).  Onto or from fine levels of at most
 * fine_cells cells that run as per-level launches, the restriction takes four threads per
 * coarse cell and the prolongation one thread per fine cell, which shortens each thread's
 * FP64 chain on small levels; larger levels keep one thread per coarse cell.  0: never.
 * Default 256 x 256 (65536) for FP64 handles.  Kept by mpfc_set_launch_shape.  Drops the handle's captured graphs.  MPFC_ERR_INVALID
 * for a negative value. */
int mpfc_set_transfer_split(mpfc_t* h, int fine_cells);

/* One step with exactly ncycles V-cycles (no tolerance test), for lockstep
 * comparisons.  Same state update and synchronisation as mpfc_step. */
int mpfc_step_cycles(mpfc_t* h, int scheme, int ncycles, mpfc_step_info* info);

/* Loads the learned initial guess model (host or device pointer to
 * MPFC_CNN_PARAM_COUNT fp32 values, layout in mpfc_cnn.h) into the handle's workspace.
 * The handle must have been created with guess = MPFC_GUESS_LEARNED (its workspace
 * then holds the network's weights and activations).  The guess uses phi^{k-2}, which
 * the handle keeps from mpfc_set_state on (phi^{-2} = phi^{-1} at the start).
 * Synchronises. */
int mpfc_set_guess_model(mpfc_t* h, const float* params, size_t count);

/* When the learned guess runs (FP64 handles with guess = MPFC_GUESS_LEARNED; no
 * counterpart in the paper): each step forms the extrapolated guess and its scaled
 * residual first, and the network corrects the guess only if that residual is at least
 * res0_threshold (kappa, mu and the residual are then formed again from the corrected
 * phi); elsewhere the step is the extrapolated guess's, bit for bit.  0 runs the network
 * on every step.  Default: 2.6e4 tol, the residual above which the extrapolated guess
 * needs more V-cycles than the network's corrected one on the 1024^2 headline workload.
 * Drops the handle's captured graphs.  MPFC_ERR_INVALID for other handles or a
 * negative or NaN threshold. */
int mpfc_set_guess_gate(mpfc_t* h, double res0_threshold);

/* The learned guess's correction on the current state, for tests of the inference
 * against the network's definition (no counterpart in the paper): d_out (m*n device
 * doubles, overwritten) receives what the guess adds to the extrapolation 2 phi^k -
 * phi^{k-1} at the next step, sy times the network's output on the features of
 * (phi^k, phi^{k-1}, phi^{k-2}).  Handle created with MPFC_GUESS_LEARNED and a model
 * loaded, else MPFC_ERR_INVALID.  Asynchronous on the handle's stream. */
int mpfc_guess_correction(mpfc_t* h, double* d_out);

/* Mass h^2 sum phi^k (conserved, Sec. 3.3, first theorem).  Synchronises. */
int mpfc_mass(mpfc_t* h, double* out);

/* Discrete energies of Sec. 3 at the current state.  The -1 norm of App. A,
 * (A.16)-(A.18), comes from a Poisson multigrid solve (under the handle's boundary
 * rule) to 1e-13 relative residual.  Synchronises. */
int mpfc_energy(mpfc_t* h, mpfc_energy_t* out);

/* Pinning of Sec. 4.6: the second-order scheme then solves with the pinned potential
 * mu~ = mu + 2 (phi^{k+1/2} - phihat) W, i.e. row 2 of N gains -W phi (a pointwise
 * linear term of the cell system) and S2 gains W (phi^k - 2 phihat); coarse levels
 * use the 2x2 averages of W.  weight (W >= 0) and target (phihat): m*n doubles, host
 * or device, copied.  weight NULL switches pinning off.  The handle must have been
 * created with pinning = 1 (else MPFC_ERR_INVALID).  While pinning is on, steps of
 * scheme 1 return MPFC_ERR_INVALID.  The step's mu is the pinned potential mu~.
 * Synchronises. */
int mpfc_set_pinning(mpfc_t* h, const double* weight, const double* target);

/* Mass h^2 sum phi of a caller's device array, without any device allocation and
 * without a handle.  The paper has no counterpart.  It serves callers that cannot let
 * a library allocate device memory and hold only a field, not a solver workspace: an
 * application whose own memory pool has reserved all of the GPU's memory (a cudaMalloc
 * would then fail or fragment that pool), or a plug-in whose host forbids device
 * allocation outside the host's allocator.  Its scratch (8.2 KB: 1024 block partial
 * sums, a counter and the result) is a static array in the library's device image,
 * present on every GPU that loads the library until the process exits.  The first
 * call on a device looks up the array's device address (once per device); make that
 * first call before any stream capture.  Every call shares the array and starts by
 * clearing its counter, so calls whose kernels overlap on the GPU race: serialise them
 * (one stream, or synchronise between calls).  At most 2048 x 2048 = 4 194 304 cells:
 * larger grids are rejected with MPFC_ERR_TOO_LARGE before anything is launched.
 * d_phi: m*n doubles on the current device; out: host.  The call waits for
 * `cuda_stream` (a cudaStream_t; NULL = legacy stream) to finish and copies the sum to
 * host memory before it returns.  MPFC_ERR_INVALID for null pointers, m or n <= 0 or
 * h <= 0; MPFC_ERR_CUDA if a CUDA call fails. */
int mpfc_mass_noalloc(const double* d_phi, int m, int n, double h, void* cuda_stream, double* out);

/* ---------------------------------------------------------------------------
 * Batched ensemble: `count` independent instances, each with its own grid size and
 * physical parameters (m, n, h, M, epsilon, beta, dt), advanced together.  The solver
 * settings (nu1, nu2, coarsest, omega, tol, max_cycles, guess) must agree, the
 * precision must be MPFC_FP64 and the guess not learned.  Every V-cycle kernel runs
 * as one persistent launch per level over a work list of (instance, tile) items;
 * instances are aligned at their coarsest grids; each instance has its own residual
 * test and drops out of the work once converged; a step is one CUDA graph that loops
 * while any instance is active.  One caller-owned workspace, as for mpfc_create.
 * ------------------------------------------------------------------------- */
typedef struct mpfc_batch_s mpfc_batch_t;

/* Workspace bytes for the batch (0 if any instance is invalid or the settings differ). */
size_t mpfc_batch_workspace_bytes(int count, const mpfc_params* each);

int mpfc_batch_create(int count, const mpfc_params* each, void* d_workspace, size_t bytes, void* cuda_stream,
                      mpfc_batch_t** out);
void mpfc_batch_destroy(mpfc_batch_t* b);

/* State of instance `inst` (copies; host or device pointers; NULL as in mpfc_set_state). */
int mpfc_batch_set_state(mpfc_batch_t* b, int inst, const double* phi, const double* phi_prev, const double* psi);
int mpfc_batch_get_state(mpfc_batch_t* b, int inst, double* phi, double* phi_prev, double* psi);

/* Advances every instance nsteps steps of scheme 1 or 2.  An instance whose step fails
 * keeps its last good state and sits out the rest of the call; statuses[i] (nullable)
 * gets its first failing status (MPFC_OK if none), cycles[i] (nullable) its V-cycles
 * over the call.  Returns the first failing status of any instance.  Synchronises. */
int mpfc_batch_step(mpfc_batch_t* b, int scheme, int nsteps, int* statuses, int* cycles);

/* One step with exactly ncycles V-cycles for every instance (lockstep tests). */
int mpfc_batch_step_cycles(mpfc_batch_t* b, int scheme, int ncycles, int* statuses);

/* Number of aligned levels (the largest instance's hierarchy). */
int mpfc_batch_levels(const mpfc_batch_t* b);

/* Tile shape (threads, tx * ty a multiple of 32 in [64, 1024]) of the smoother's
 * work items on aligned level `level`; rebuilds the work lists.  Used by the tile
 * autotuner, which times candidates with mpfc_batch_time_smooth (milliseconds per full
 * red-black sweep of that level, all instances, averaged over `reps`). */
int mpfc_batch_set_tile(mpfc_batch_t* b, int level, int tx, int ty);
int mpfc_batch_time_smooth(mpfc_batch_t* b, int scheme, int level, int reps, float* ms);

/* Message for a status code. */
const char* mpfc_strerror(int status);

/* Number of grid levels of the handle's hierarchy and the size of one level. */
int mpfc_levels(const mpfc_t* h);
int mpfc_level_size(const mpfc_t* h, int level, int* m, int* n, double* hl);

/* ---------------------------------------------------------------------------
 * Component entry points.  Each runs one building block of the V-cycle on caller
 * arrays of the given level's size (device pointers, asynchronous on the handle's
 * stream), with the handle's coefficients.  `phik` is phi^k on that level and is
 * read only by scheme 2 (pass NULL for scheme 1).
 * ------------------------------------------------------------------------- */

/* S of App. B.1 (scheme 1) or App. B.2 (scheme 2) on the finest level. */
int mpfc_op_source(mpfc_t* h, int scheme, const double* phik, const double* phikm1, const double* psik,
                   double* S1, double* S2, double* S3);

/* `sweeps` nonlinear red-black block Gauss-Seidel sweeps (App. B), red cells
 * ((i+j) even) first; each cell: one local Newton linearisation of the cubic and a
 * 3x3 solve by Cramer's rule for the correction of the cell's residual, applied
 * with relaxation omega (u <- u + omega A^-1 r). */
int mpfc_op_smooth(mpfc_t* h, int scheme, int level, double* phi, double* mu, double* kappa, const double* S1,
                   const double* S2, const double* S3, const double* phik, int sweeps);

/* r = S - N(u), N of App. B.1/B.2. */
int mpfc_op_residual(mpfc_t* h, int scheme, int level, const double* phi, const double* mu, const double* kappa,
                     const double* S1, const double* S2, const double* S3, const double* phik, double* r1,
                     double* r2, double* r3);

/* FAS restriction from `level` to level+1: u_c = R u (2x2 average) and
 * S_c = N_c(u_c) + R(S - N(u)).  phik_c is phi^k on level+1 (scheme 2). */
int mpfc_op_restrict(mpfc_t* h, int scheme, int level, const double* phi, const double* mu, const double* kappa,
                     const double* S1, const double* S2, const double* S3, const double* phik,
                     const double* phik_c, double* phi_c, double* mu_c, double* kappa_c, double* S1_c,
                     double* S2_c, double* S3_c);

/* FAS correction of `level` from level+1: u += P(u_c_new - u_c_old), P the
 * cell-centred bilinear interpolation. */
int mpfc_op_prolong(mpfc_t* h, int level, const double* phi_c_new, const double* mu_c_new,
                    const double* kappa_c_new, const double* phi_c_old, const double* mu_c_old,
                    const double* kappa_c_old, double* phi, double* mu, double* kappa);

/* Runs the learned guess alone on the current state: the network's correction is
 * added to the finest level's phi array (handle created with MPFC_GUESS_LEARNED and a
 * model loaded).  For timing the network; asynchronous. */
int mpfc_op_learned_guess(mpfc_t* h);

/* Exact solve of N(u) = S on the coarsest level (Newton on the eliminated
 * equation for phi; mu, kappa recovered from the second and third rows). */
int mpfc_op_coarse_solve(mpfc_t* h, int scheme, double* phi, double* mu, double* kappa, const double* S1,
                         const double* S2, const double* S3, const double* phik);

#ifdef __cplusplus
}
#endif

#endif /* MPFC_H */
