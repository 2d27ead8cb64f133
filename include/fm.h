/*
 * fm.h -- C ABI of the GB300 (sm_103a) implicit time step for the hydrodynamic
 * freezing models of Baskaran, Guan and Lowengrub, "Energy Stable Multigrid
 * Method for Local and Non-local Hydrodynamic Models for Freezing".
 *
 * One call of fm_step advances (rho^k, u^k) by one step of the fully discrete
 * convex-splitting scheme, Sec. 5, Eqs. (discrete_a)-(discrete_d):
 *
 *   rho^{k+1} - rho^k = -s div_h(rho^k u^{k+1/2}),
 *   rho^k (u^{k+1} - u^k) = s [ -rho^k omega^k x u^{k+1/2}
 *        - (rho^k/2) grad_h |u^{k+1}|^2 - rho^k grad_h mu^{k+1}
 *        + gamma Lap_h u^{k+1/2} ],
 *   mu^{k+1} = dF_c[rho^{k+1}] - dF_e[rho^k],   omega^k = curl_h u^k,
 *
 * with the PFC functional (Sec. 5.3, Lemma 5.4) or the non-local CDFT
 * functional (Sec. 5.2, Lemma 5.2, kernel J of Sec. 6, convolution of
 * Eq. (discrete_convolution) evaluated by a hand-written FFT).  The implicit
 * system N(g) = S of App. G is solved by FAS multigrid (Sec. 6) with a
 * red-black point-block Gauss-Seidel smoother (App. G.1, G.2), damping
 * (App. G.3) and the positive projection of Sec. 6.
 *
 * Conventions shared by every entry point:
 *  - Return 0 (FM_OK) on success or a negative FM_E* code; nothing throws.
 *  - Grids are periodic with cubic cells of side h.  Fields are stored
 *    row-major with x fastest: index (k*ny + j)*nx + i.  Velocities are passed
 *    as `dim` separate arrays (structure of arrays), all float64.
 *  - `where` says whether caller pointers are host (FM_HOST) or device
 *    (FM_DEVICE) memory; device pointers must be on the current CUDA device.
 *  - The caller owns the handle and its own arrays; the library allocates
 *    (cudaMalloc at fm_create) and owns every device buffer of the solver and
 *    frees them in fm_destroy.
 *  - All work is issued on the stream given to fm_set_stream (default: the
 *    legacy default stream).  Calls that return values to the host (fm_step's
 *    convergence test, fm_energy, fm_mass) synchronise that stream.
 *  - On a nonzero return from fm_step the state is left at time level k,
 *    unchanged.
 */
#ifndef FM_H
#define FM_H

#ifdef __cplusplus
extern "C" {
#endif

#define FM_OK        0
#define FM_EINVAL   (-1)  /* invalid argument (sizes, parameters, null pointers) */
#define FM_ENOMEM   (-2)  /* device allocation failed */
#define FM_ECUDA    (-3)  /* a CUDA runtime call failed */
#define FM_ENOCONV  (-4)  /* residual above tol after max_cycles V-cycles */
#define FM_ENONPOS  (-5)  /* CDFT: a density <= 0 where ln rho is needed -- an input
                             rho^k <= 0, or (delta = 0, no projection floor) an
                             update that left rho <= 0; the state is unchanged */
#define FM_ENAN     (-6)  /* non-finite residual */
#define FM_ETIMEOUT (-7)  /* a bounded wait inside a kernel ran out (a tensor copy that
                             did not complete within 1 s); the state is unusable */

#define FM_PFC   1        /* local phase-field-crystal functional, Sec. 2.2 / 5.3 */
#define FM_CDFT  2        /* non-local CDFT functional, Sec. 2.1 / 5.2 */

#define FM_FP64  0        /* every sweep in float64 */
#define FM_MIXED 1        /* float32 smoothing and transfers inside a float64
                             outer residual / defect-correction loop */

#define FM_HOST   0
#define FM_DEVICE 1

#define FM_WALLS_NONE 0   /* periodic in every direction (default) */
#define FM_WALLS_Y    1   /* 2-D PFC channel: periodic in x, no-slip walls at
                             y = 0 and y = n_y h (App. E.2, Sec. 6.3) */

#define FM_INIT_PREVIOUS    0  /* initial iterate of a step: the previous time level (default) */
#define FM_INIT_EXTRAPOLATE 1  /* the linear extrapolation in time of the last two converged iterates */

#define FM_HYDRO    0     /* the hydrodynamic scheme of Sec. 4-5 (default) */
#define FM_GRADFLOW 1     /* the conservative gradient-flow scheme of Sec. 3,
                             Thm 3.3: rho^{k+1} - rho^k = s Lap_h (dF_c[rho^{k+1}]
                             - dF_e[rho^k]); no velocity */

/* Periodic grid: dim = 2 or 3; n[d] points along x, y, z (n[2] ignored in
 * 2-D); spacing h.  Every n[d] must be even (red-black ordering). */
typedef struct {
    int dim;
    int n[3];
    double h;
} fm_grid;

/* kind = FM_PFC: alpha = 1 - eps (App. B).  kind = FM_CDFT: nu is the spatial
 * scale of the kernel J(x) = sqrt(2) exp(-pi^2 |x|^2/(2 nu^2))
 * - exp(-pi^2 |x|^2/(4 nu^2)) (Sec. 6). */
typedef struct {
    int kind;
    double alpha;
    double nu;
} fm_functional;

/* Solver parameters (fm_default_params fills the defaults in brackets). */
typedef struct {
    double gamma;   /* viscosity [2], Sec. 6 */
    double w_damp;  /* damping weight of the point block [0.5], App. G.3 */
    double delta;   /* projection rho <- sqrt(rho^2 + delta^2) [0], Sec. 6 */
    double tol;     /* stop when max_c sqrt(h^d sum r_c^2) <= tol [1e-10] */
    double sigma;   /* sign of the vorticity term [+1 = vector form of Eq.
                       (discrete_b)]; -1 reproduces the App. G printing */
    int nu1, nu2;   /* pre- and post-smoothing iterations [2, 2] */
    int max_cycles; /* [50] */
    int coarsest;   /* coarsen while every n[d]/2 >= coarsest and is even [16] */
    int ncoarse;    /* smoothing iterations on the coarsest grid [4] */
    int precision;  /* FM_FP64 or FM_MIXED [FM_FP64] */
    int model;      /* FM_HYDRO or FM_GRADFLOW [FM_HYDRO].  The gradient flow
                       has the unknowns (rho, mu, kappa) (PFC) or rho (CDFT),
                       solved by the same FAS cycle with a point block of its
                       own (damping w_damp = 0.5 is needed for PFC); its state
                       has no velocity: fm_set_fields / fm_step_host accept
                       null velocity arrays, fm_get_fields returns zeros,
                       fm_smooth and the batch calls return FM_EINVAL. */
    int walls;      /* FM_WALLS_NONE or FM_WALLS_Y [FM_WALLS_NONE].  Walls
                       (2-D hydrodynamic PFC only): the n_y rows are cells
                       whose centres lie at (j + 1/2) h, the walls half a cell
                       beyond the first and last rows, with the ghost rules of
                       App. E.2 -- rho, mu, kappa mirrored (no flux), v odd,
                       u = 2 u_wall - u (no slip on a wall moving along x);
                       the multigrid transfers are cell-centred in y.  fm_smooth
                       and the batch calls return FM_EINVAL. */
    double u_wall[2]; /* speeds along x of the walls at y = 0 and y = n_y h [0, 0];
                       with both at rest the step is energy stable (Thm 5.1) */
    int init;       /* initial iterate of a step [FM_INIT_PREVIOUS] (periodic
                       hydrodynamic solver; FM_EINVAL elsewhere).  The paper
                       fixes only the solution, not the iterate that reaches
                       it: FM_INIT_PREVIOUS starts from (rho^k, u^k) with
                       kappa^0 = Lap_h rho^k and mu^0 the mu row at rho^k, so
                       a step depends on (rho^k, u^k) alone; FM_INIT_EXTRAPOLATE
                       starts from 2 g^k - g^{k-1}, the converged iterates
                       of the last two steps of this state, which fewer
                       V-cycles then correct.  The history is kept across
                       fm_step and fm_step_host calls and cleared by
                       fm_set_fields, fm_prepare, fm_residual, a change of
                       the step size and a failed step; the converged
                       solution is the same either way (to the tolerance). */
    int coarse_precision; /* precision of the coarsest-grid solve when
                       precision = FM_MIXED [FM_FP64]: FM_FP64 solves it in
                       float64 (the levels the single-block V-cycle or the
                       coarsest multi-block sweeps handle, on float64 copies
                       of their data), FM_MIXED in the cycle's float32.  The
                       periodic hydrodynamic solver; the gradient flow, the
                       channel and batches solve it in the cycle's
                       precision. */
} fm_params;

typedef struct {
    int cycles;     /* V-cycles taken */
    double res0;    /* residual norm of the initial iterate */
    double res;     /* final residual norm (float64) */
} fm_step_info;

typedef struct fm_state fm_state;

/* Fill *p with the defaults listed in fm_params. */
void fm_default_params(fm_params* p);

/* Create a solver for one grid.  Validates the sizes and parameters
 * (FM_EINVAL), builds the multigrid hierarchy, and for CDFT samples J,
 * computes c_e = (J_e * 1) = h^d sum J_e (Lemma 5.2) and the transform of J
 * on the device.  The state starts at rho = 0, u = 0: call fm_set_fields. */
int fm_create(const fm_grid* grid, const fm_params* prm,
              const fm_functional* fn, fm_state** out);

/* Free every device buffer and the handle (null is accepted). */
void fm_destroy(fm_state* st);

/* Issue all further work on `stream` (a cudaStream_t). */
int fm_set_stream(fm_state* st, void* stream);

/* Copy rho and the dim velocity components (vel[0..dim-1]) into the state.
 * Each array holds nx*ny*nz float64 values. */
int fm_set_fields(fm_state* st, const double* rho, const double* const* vel, int where);

/* Copy the current rho and velocity out of the state. */
int fm_get_fields(fm_state* st, double* rho, double* const* vel, int where);

/* Advance one time step of size dt (the paper's s) with FAS V(nu1, nu2)
 * cycles until the float64 residual norm is <= tol, then re-evaluate
 * rho^{k+1} from the continuity equation with the final velocity (mass exact
 * to round-off) and project.  info may be null.  FM_ENOCONV / FM_ENAN /
 * FM_ENONPOS leave the state unchanged. */
int fm_step(fm_state* st, double dt, fm_step_info* info);

/* One step for a caller that keeps the fields in host memory: copies rho_in
 * and vel_in[0..dim-1] (host arrays, nx*ny*nz float64 each; pinned memory
 * lets the copies run asynchronously) into the state, runs fm_step's step on
 * the state's stream and copies the new rho and velocity to rho_out and
 * vel_out (host), with a single host synchronisation at the end.  The same
 * arithmetic as fm_set_fields + fm_step + fm_get_fields.  On FM_ENOCONV /
 * FM_ENAN / FM_ENONPOS the state and the outputs hold the inputs (time level
 * k). */
int fm_step_host(fm_state* st, double dt, const double* rho_in, const double* const* vel_in,
                 double* rho_out, double* const* vel_out, fm_step_info* info);

/* Total energy E = 1/2 (rho u || u) + F[rho] (Thm 5.1) of the current state,
 * with F the discrete PFC energy (Eq. CS_PFC_discrete) or the CDFT energy
 * (Eq. CS_DFT_discrete); F and KE separately.  Float64 deterministic
 * reductions.  Any output pointer may be null. */
int fm_energy(fm_state* st, double* E, double* F, double* KE);

/* Components of the energy of the current state (the quantities the paper
 * plots in its freezing and convergence figures, Sec. 6.1-6.2), float64
 * deterministic reductions, into terms[0..4]:
 *   terms[0] = KE = 1/2 (rho u || u);
 *   PFC (Eq. CS_PFC_discrete): terms[1..4] = h^d sum psi^4/12,
 *        h^d sum alpha psi^2/2, h^d sum (Lap_h rho)^2/2, h^d sum rho Lap_h rho
 *        (psi = rho - 3/2; F is their sum);
 *   CDFT (Eq. CS_DFT_discrete): terms[1] = F_id = (rho || ln rho - 1),
 *        terms[2] = F_ex = -1/2 (rho || J * rho), terms[3] = terms[4] = 0.
 * terms must hold 5 doubles (host memory).  Synchronises the state's stream. */
int fm_energy_terms(fm_state* st, double* terms);

/* Mass (rho || 1) = h^d sum rho (Thm 5.1). */
int fm_mass(fm_state* st, double* M);

/* Human-readable message for a return code. */
const char* fm_strerror(int code);

/* ---- Row-level entry points (each is one step of fm_step, exposed so that
 * every part of the hot path can be checked on its own). ---- */

/* What fm_get_aux reads (all float64, nx*ny*nz values per component). */
#define FM_AUX_OMEGA   1  /* omega^k components (1 in 2-D, 3 in 3-D), Eq. (discrete_d) */
#define FM_AUX_SOURCE  2  /* S components of App. G (1+dim, +2 for PFC) */
#define FM_AUX_CONV    3  /* J * rho^k (CDFT), Eq. (discrete_convolution) */
#define FM_AUX_ITERATE 4  /* the current iterate g (rho, u.., mu, kappa) */

/* Compute omega^k, J*rho^k (CDFT), the source S and the initial iterate g^0
 * for a step of size dt from the current fields (the first stage of
 * fm_step). */
int fm_prepare(fm_state* st, double dt);

/* Read component `comp` of an auxiliary field after fm_prepare or fm_step. */
int fm_get_aux(fm_state* st, int what, int comp, double* out, int where);

/* Float64 residual r = S - N(g) of App. G for a caller-supplied iterate g
 * (g[0..nu-1] with nu = 1 + dim (+2 for PFC)) against the source of the last
 * fm_prepare; writes r (r may be null) and its norm max_c sqrt(h^d sum r_c^2). */
int fm_residual(fm_state* st, const double* const* g, double* const* r,
                double* norm, int where);

/* Periodic convolution out = J * rho (Eq. (discrete_convolution)) with the
 * state's kernel J (CDFT states only), by FFT. */
int fm_convolve(fm_state* st, const double* rho, double* out, int where);

/* Nodal full-weighting restriction of one float64 field from the state's
 * finest grid to the next coarser grid (coarse sizes n[d]/2). */
int fm_restrict(fm_state* st, const double* fine, double* coarse, int where);

/* fine += bilinear (trilinear) prolongation of one float64 coarse field. */
int fm_prolong_add(fm_state* st, const double* coarse, double* fine, int where);

/* Number of multigrid levels of the state. */
int fm_levels(const fm_state* st);

/* Smoother row (App. G.1-G.3 and the red-black ordering of the solver):
 * `sweeps` red-black sweeps of the damped point-block Gauss-Seidel smoother,
 * in the state's precision, on the finest grid for the correction equation
 * M(e) = N(g + e) - N(g) = f, with g the iterate of the last fm_prepare or
 * fm_step as coefficient.  e (in/out) and f are nu float64 arrays each
 * (nu = 1 + dim, +2 for PFC; host or device per `where`), rounded to the
 * state's precision on entry.  variant: FM_SWEEP_AUTO runs the sweeps exactly
 * as fm_step does (2-D: the autotuned fused sweep over the largest even
 * number of sweeps, an odd last sweep as two colour launches);
 * FM_SWEEP_TWO_COLOUR runs every sweep as a red launch and a black launch;
 * 0 .. FM_SWEEP_VARIANTS - 1 fixes the fused variant (encoding as fm_tuning;
 * in 3-D 0 .. 4, a z-marching variant falling back to the colour launches on
 * a level it does not fit).  FM_EINVAL before the first fm_prepare, for
 * sweeps < 0, an unknown variant or a 2-D variant that does not fit in
 * shared memory. */
#define FM_SWEEP_AUTO (-1)
#define FM_SWEEP_TWO_COLOUR (-2)
int fm_smooth(fm_state* st, double* const* e, const double* const* f, int sweeps, int variant,
              int where);

/* ---- Batched ensembles (2-D) ---- */

/* A set of independent 2-D instances (uneven grid sizes allowed) stepped
 * together: every stage of the step -- including each multigrid level of the
 * V-cycle -- is one kernel launch over all instances, and the whole step is
 * one CUDA graph whose WHILE loop runs until every instance has converged
 * (each instance stops iterating at its own convergence).  Same scheme and
 * solver as fm_step, per instance. */
typedef struct fm_batch fm_batch;

/* count instances with grids[0..count-1] (all dim = 2), shared parameters
 * and functional.  FM_EINVAL for 3-D grids or invalid sizes. */
int fm_create_batch(int count, const fm_grid* grids, const fm_params* prm,
                    const fm_functional* fn, fm_batch** out);

/* Free the batch and all its instances (null accepted). */
void fm_destroy_batch(fm_batch* b);

/* Issue all further work on `stream`. */
int fm_batch_set_stream(fm_batch* b, void* stream);

/* Instance i as an fm_state, owned by the batch: use fm_set_fields,
 * fm_get_fields, fm_energy, fm_mass on it (not fm_destroy). */
fm_state* fm_batch_instance(fm_batch* b, int i);

/* One time step of every instance, instance i with step dt[i] > 0; info
 * (nullable) receives count records.  Returns the first non-zero instance
 * status (instances that failed are left at their time level k). */
int fm_step_batch(fm_batch* b, const double* dt, fm_step_info* info);

/* Kernels launched by the batch since creation. */
long long fm_batch_launches(const fm_batch* b);

/* Autotuner choice of the fused-sweep variant for multigrid level `level` of
 * the batch (same encoding and timings as fm_tuning). */
int fm_batch_tuning(const fm_batch* b, int level, int* variant, float* ms_per_variant);

/* Measurement (no counterpart in the paper): mean duration (ms, CUDA events)
 * of one launch of the fused red-black sweep variant the autotuner chose for
 * the finest level, over all instances (one sweep, or two for the two-sweep
 * variants 18..23; see fm_batch_tuning), timed over `iters` back-to-back
 * launches after one warm-up launch, and the number of finest-level points
 * one launch covers.  Overwrites only solver scratch (the corrections), which
 * the next fm_step_batch resets. */
int fm_batch_time_smoother(fm_batch* b, int iters, double* ms_per_launch, long long* points);

/* Measurement (no counterpart in the paper): as fm_batch_time_smoother for
 * fused-sweep variant `variant` (0 .. FM_SWEEP_VARIANTS - 1, encoding as
 * fm_tuning) instead of the autotuned one.  FM_EINVAL for an unknown variant
 * or one that does not fit in shared memory. */
int fm_batch_time_sweep_variant(fm_batch* b, int variant, int iters, double* ms_per_launch, long long* points);

/* ---- Measurement (no counterpart in the paper). ---- */

/* Number of variants of the 2-D fused red-black sweep. */
#define FM_SWEEP_VARIANTS 36

/* Variant of the 2-D fused red-black sweep the autotuner chose for `level`
 * at fm_create, and its timings of all FM_SWEEP_VARIANTS variants in ms per
 * sweep (ms_per_variant may be null; 0 for levels that were not tuned and for
 * variants that do not fit in shared memory).  Variants 0..11 are the tile
 * form (v >> 2: tile 32x16, 64x8 or 32x32; bit 1: right-hand side staged in
 * shared memory; bit 0: persistent double-buffered blocks); 12..17 the
 * row-marching form (strip width 64 for 12..14, 128 for 15..17; 16, 32 or 64
 * rows per block); 18..23 the row-marching form that runs two sweeps in one
 * pass (strips and rows as 12..17); 24..26 the tile form that runs two sweeps
 * per tile (tiles 32x16, 64x8, 32x32, halo of four, f and omega from global
 * memory); 27..29 the tile form with each tile staged by tensor copies (TMA)
 * instead of cp.async: 27 as 24, 28 as 0, 29 as 26 (the same updates; on a
 * level whose rows are not a whole number of 16 bytes they run the cp.async
 * staging; batches run them as 24, 0 and 26 and do not time them); 30..33
 * the tile form on small tiles, for the coarse levels: 30 one sweep and 31
 * two sweeps per launch on 16 x 16 tiles, 32 and 33 the same on 16 x 8
 * (single-instance solver; batches run them as 0, 24, 0, 24 and do not time
 * them); 34 all the sweeps of a smoothing step (red and black passes over
 * the whole level, in place) in one cooperative launch whose blocks meet at
 * a grid-wide barrier between passes, timed with two sweeps per launch
 * (single-instance solver; batches run it as 24); 35 as 24 on 32 x 14 tiles
 * (592 tiles at 512^2, so that four blocks on each of 152 multiprocessors
 * take nearly all of them in one wave; single-instance solver, batches run
 * it as 24).  The time per launch of a two-sweep variant is halved to give
 * its time per sweep.  In 3-D the variants are 0 (a red and a black launch,
 * 256-thread blocks, the compiler's register count), 1 (the same bounded to
 * six resident blocks per multiprocessor) and 2 (the sweep in z-chunks sized
 * to stay in L2: red over a chunk, then black over the planes whose
 * neighbours are red by then; levels whose arrays fit in 48 MB are not
 * chunked and report 0 for it), 3 and 4 (one launch per sweep, marching up
 * the planes of 32 x 8 or 32 x 16 point tiles staged plane by plane in
 * shared memory by bulk copies; levels whose sides are not multiples of the
 * tile report 0 for them and sweep with variant 1); their times are per
 * sweep.  Setting the environment variable
 * FM_RB_VARIANT=v before fm_create fixes the variant (no timing); a
 * comma-separated list fixes one per level from the finest (the last one
 * repeats; batches take the first). */
int fm_tuning(const fm_state* st, int level, int* variant, float* ms_per_variant);

/* Enable (1) or disable (0) CUDA-event timing of every finest-level smoother
 * launch issued by fm_step, and reset the accumulated totals. */
int fm_profile(fm_state* st, int enable);

/* Accumulated finest-level smoother time (ms) and launch count since the last
 * fm_profile call, and the total number of kernels this state has launched
 * since fm_create.  Any output pointer may be null. */
int fm_profile_read(const fm_state* st, double* smoother_ms, long long* smoother_launches,
                    long long* launches);

/* Diagnostic (no counterpart in the paper): out[i] = in[i] narrowed from
 * float64 to float32 exactly as the float64 residual kernels narrow the
 * right-hand side and coefficients they hand to the float32 cycle (round to
 * nearest, ties to even, computed with integer instructions); in and out are
 * device arrays of n values, the work is issued on `stream` and synchronised.
 * Exposed so that it can be compared bit for bit with the CUDA conversion. */
int fm_narrow(const double* in, float* out, long long n, void* stream);

/* Diagnostic (no counterpart in the paper): out[i] = in[i] widened from
 * float32 to float64 (exact) with integer instructions, as the float64
 * update g += e widens the float32 correction; device arrays, n values, on
 * `stream`, synchronised.  For a bit-for-bit comparison with the CUDA
 * conversion. */
int fm_widen(const float* in, double* out, long long n, void* stream);

/* Diagnostic (no counterpart in the paper): runs the bounded mbarrier wait
 * of the tensor-copy tile smoother in a one-block kernel on `stream`, on a
 * barrier that one thread completes (complete = 1) or that nothing completes
 * (complete = 0), giving up after limit_us microseconds (1 .. 1000000), and
 * synchronises.  FM_OK when the wait saw the barrier complete, FM_ETIMEOUT
 * when the limit ran out (the kernel then returns normally and the device
 * stays usable), FM_EINVAL for a limit out of range.  Not reentrant: calls
 * that overlap on the GPU share one status word. */
int fm_wait_selftest(int complete, int limit_us, void* stream);

/* Measurement (no counterpart in the paper): the bounded wait of the
 * grid-wide barrier of the cooperative sweep (fused-sweep variant 34), on
 * `stream`: a cooperative launch of all the blocks the device holds at once,
 * each arriving once and then waiting for every block (complete = 1) or for
 * an arrival count nothing reaches (complete = 0), giving up after limit_us
 * microseconds (1 .. 1000000), and synchronises.  FM_OK when every block
 * passed, FM_ETIMEOUT when the limit ran out (every block then returns and
 * the device stays usable), FM_EINVAL for a limit out of range.  Not
 * reentrant: calls share one barrier and status word. */
int fm_grid_barrier_selftest(int complete, int limit_us, void* stream);

/* ---- Allocation-free entry point (the paper has no counterpart). ---- */

/* Largest grid fm_mass_noalloc accepts: 4096 blocks x 1024 points. */
#define FM_NOALLOC_MAX_POINTS (4096LL * 1024LL)

/* Mass h^d sum rho of the caller's float64 device array `rho` (dim = 2 or 3,
 * n[0..dim-1] points, spacing h), written to the caller's device double
 * `out`, issued on `stream` (a cudaStream_t; null = legacy default stream).
 * It allocates no device memory: for callers that cannot call cudaMalloc
 * (a host application whose device memory is reserved by its own allocator,
 * or a time-critical loop that must not take cudaMalloc's implicit
 * synchronisation).  Its 32 KiB reduction scratch is a static device array
 * that every GPU loading libfm holds until exit; all calls share it, so calls
 * that overlap on the GPU race.  The first call on each device looks up the
 * scratch address (cudaGetSymbolAddress) and must come before any stream
 * capture.  Returns FM_EINVAL for null pointers, bad dim/h or more than
 * FM_NOALLOC_MAX_POINTS points; asynchronous (read `out` after the stream). */
int fm_mass_noalloc(const double* rho, int dim, const int* n, double h, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FM_H */
