/*
 * sve.h -- C ABI of libsve, the GB300 (sm_103a) time stepper for the
 * Saint-Venant--Exner system with the relaxation-solver interface fluxes of
 * Audusse, Delestre, Le, Masson-Fauchier, Navaro, Serra, "Parallelization of
 * a relaxation scheme modelling the bedload transport of sediments in shallow
 * water flow" (arXiv:1307.0491).
 *
 * One step (Sec. 3, the procedure stated after the list of properties of the
 * relaxation model): project the auxiliary variables to equilibrium
 * (Pi = g h^2/2, Omega = q_b; lambda -> 0 in Eqs. relaxpi, relaxqs), solve
 * the homogeneous relaxation Riemann problem (Eqs. relaxh--relaxqs) at every
 * interface, and average the juxtaposed Riemann solutions over each cell
 * (Godunov); then apply semi-implicit friction (S_f laws of Sec. 2).  The 2D
 * step is the unsplit method of lines on a structured grid (Sec. 4).  The time
 * step is the global CFL step of the current state.
 *
 * Conventions
 *   - State: four fields h, hu, hv, zb (water depth, x and y discharge, bed
 *     elevation), each nx*ny values, row-major [ny][nx] with x fastest.  In
 *     1D (dim = 1) ny = 1 and hv is ignored (pass NULL).
 *   - Precision: SVE_FP64 state arrays are double; SVE_FP32 state arrays are
 *     float (the time, time step and mass sums stay double).
 *   - where = SVE_HOST: pointers are host memory; SVE_DEVICE: pointers are
 *     device memory of the current device, contiguous, of the state type.
 *   - Ownership: the caller owns every buffer it passes; the library copies on
 *     set and writes into the caller's buffers on get.  The library owns its
 *     device state, scratch, status word and CUDA graph.
 *   - Streams: all device work is enqueued on the handle's stream (default:
 *     the legacy default stream; see sve_set_stream).
 *   - Errors: every int-returning call returns SVE_OK (0) or a negative
 *     SVE_ERR_* code; sve_strerror names it.  Device-detected errors (a
 *     Riemann solve that does not converge, a non-positive depth, a NaN, a bad
 *     time step) are latched in a device status word; the step calls return
 *     the latched code.  A handle is not thread-safe.
 */
#ifndef SVE_H
#define SVE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- codes -------------------------------------------------------------- */
enum {
  SVE_OK = 0,
  SVE_ERR_ARG = -1,       /* invalid argument or configuration */
  SVE_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  SVE_ERR_OOM = -3,       /* device allocation failed */
  SVE_ERR_NEG_DEPTH = -4, /* a depth became <= 0 */
  SVE_ERR_RIEMANN = -5,   /* an interface Riemann problem had no solution with positive specific volumes */
  SVE_ERR_NAN = -6,       /* a non-finite value appeared in the state */
  SVE_ERR_DT = -7,        /* a time step was <= 0 or non-finite */
  SVE_ERR_STATE = -8,     /* no state has been set on the handle */
  SVE_ERR_NOALLOC_SIZE = -9, /* the grid does not fit the static scratch of sve_step_noalloc */
  SVE_ERR_SYNC = -10        /* a grid-wide wait of the persistent small-grid step ran out (the
                               context stays usable; latched until the next sve_set_state) */
};

enum { SVE_FP64 = 0, SVE_FP32 = 1 };                       /* state precision */
enum { SVE_SCHEME_COUPLED = 0, SVE_SCHEME_SPLIT = 1 };      /* step scheme (sve_set_scheme) */
/* bedload law: Grass, or a Shields-parameter law of Sec. 2 */
enum { SVE_GRASS = 0, SVE_MPM = 1, SVE_FLVB = 2, SVE_NIELSEN = 3, SVE_RIBBERINK = 4, SVE_CAMENEN = 5 };
enum { SVE_FRIC_NONE = 0, SVE_FRIC_DARCY = 1, SVE_FRIC_STRICKLER = 2 };
enum { SVE_BC_PERIODIC = 0, SVE_BC_FREE = 1, SVE_BC_INFLOW_Q = 2, SVE_BC_INFLOW_QH = 3, SVE_BC_WALL = 4,
       SVE_BC_EXTERNAL = 5 /* ghost ring set by the caller: a side of a block of a decomposed grid */ };
enum { SVE_HOST = 0, SVE_DEVICE = 1 };
enum { SVE_W = 0, SVE_E = 1, SVE_S = 2, SVE_N = 3 };

/* ---- configuration -------------------------------------------------------
 * dim           1 or 2.
 * nx, ny        cells (ny = 1 in 1D).
 * lx, ly        domain lengths [m]; dx = lx/nx, dy = ly/ny.
 * g             gravity [m/s^2].
 * cfl           CFL number of the time step: dt = cfl dx / Sx (1D),
 *               dt = cfl / (Sx/dx + Sy/dy) (2D), S = max over interfaces of
 *               the extreme relaxation wave speeds |u - a/h|, |u + a/h|.
 * precision     SVE_FP64 or SVE_FP32 (state storage and arithmetic).
 * bedload       SVE_GRASS: q_b = A_g u |u|^(m_g - 1) (Eq. bedload Grass, 2D:
 *               vector u).  The Shields-parameter laws (non-dimensional form
 *               of Sec. 2: q_b = sqrt((s-1) g d_s^3) q*(tau*) along u/|u|,
 *               tau* from the friction law), x = (tau* - tau_cr)_+:
 *               SVE_MPM 8 x^1.5 (Eq. MPM); SVE_FLVB 5.7 x^1.5 (Eq. FLVB);
 *               SVE_NIELSEN 12 sqrt(tau*) x (Eq. Nielsen); SVE_RIBBERINK
 *               11 x^1.65 (Eq. Ribberink); SVE_CAMENEN 12 tau*^1.5
 *               exp(-4.5 tau_cr / tau*) (Eq. Camenen).  They need a friction
 *               law.
 * A_g, m_g      Grass constants (1 <= m_g <= 4).
 * s, d_s, tau_cr  Shields laws: relative density, grain diameter [m],
 *               critical Shields number.
 * friction      SVE_FRIC_NONE / _DARCY (f_dw) / _STRICKLER (K_st = 1/n).
 * bc[4]         W, E, S, N ghost rules: PERIODIC (both sides of an axis),
 *               FREE (copy), INFLOW_Q (inward normal discharge q_in, h and
 *               zb copied), INFLOW_QH (h = h_in as well), WALL (mirror),
 *               EXTERNAL (the ghost ring of that side is set by the caller,
 *               sve_block_set_ghosts; not for batches, the adjoint or
 *               sve_step_noalloc).
 * q_in, h_in    inflow data.
 * kappa_a, beta_min, gamma_z  relaxation celerities of one interface:
 *               a = max(kappa_a max(a0, b0), sqrt(b^2 + 2 g gamma_z |dzb| hmax^2)),
 *               b = max(b0, beta_min a0), with a0 = max h sqrt(g h) and
 *               b0 = max sqrt((h u)^2 + g h^2 dq_b/du) the bounds of Eq. (ab).
 * newton_tol, newton_maxit   stopping rule of the scalar Newton iteration of
 *               each Riemann solve: stop after the update with |dp| <= tol p
 *               (quadratic convergence leaves ~(tol p)^2 |F''/2F'| behind:
 *               1e-9 puts that below FP64 rounding).
 */
typedef struct sve_config {
  int dim;
  int nx, ny;
  double lx, ly, g;
  double cfl;
  int precision;
  int bedload;
  double A_g, m_g;
  double s, d_s, tau_cr;
  int friction;
  double f_dw, K_st;
  int bc[4];
  double q_in, h_in;
  double kappa_a, beta_min, gamma_z;
  double newton_tol;
  int newton_maxit;
} sve_config;

typedef struct sve_handle sve_handle;

/* Fill *cfg with the defaults (2D, FP64, g = 9.81, cfl = 0.9, Grass A_g = 1e-3,
 * m_g = 3, MPM s = 2.65, d_s = 1e-3, tau_cr = 0.05, no friction, periodic in
 * x, free in y, kappa_a = 1.1, beta_min = 0.01, gamma_z = 2, newton_tol =
 * 1e-9, newton_maxit = 30).  Sizes must still be set. */
int sve_config_default(sve_config* cfg);

/* Validate cfg, allocate the device state and scratch on the current device
 * and return a handle in *out.  SVE_ERR_ARG on an invalid configuration,
 * SVE_ERR_OOM if device memory runs out. */
int sve_create(const sve_config* cfg, sve_handle** out);

/* Use the CUDA stream `stream` (a cudaStream_t, NULL = legacy default) for
 * all later work of the handle. */
int sve_set_stream(sve_handle* h, void* stream);

/* Copy a state in (t is reset to 0).  hv may be NULL in 1D.  The state is
 * checked on the device (depth > 0, finite): the first failing check is
 * returned. */
int sve_set_state(sve_handle* h, const void* depth, const void* hu, const void* hv, const void* zb, int where);

/* Advance nsteps CFL steps.  *t_out (nullable) receives the simulated time.
 * Blocks until the steps are done and returns the first latched device
 * error, if any.  With the FP32 state in 2D a call of several steps (this
 * one, sve_step_dt, sve_step_async, sve_advance) carries each step's update
 * into the next step's solve pass, which applies it as it reads the state,
 * and runs the update pass once after the last solve pass: the same states,
 * time steps and mass sums as one-step calls, bit for bit, with one trip of
 * the state through device memory per step instead of two. */
int sve_step(sve_handle* h, int nsteps, double* t_out);

/* Advance nsteps steps of the given sizes dts[0..nsteps-1] (host memory). */
int sve_step_dt(sve_handle* h, int nsteps, const double* dts);

/* Copy the state out (interior cells only).  hv may be NULL in 1D.  Blocks
 * until the copy is done. */
int sve_get_state(sve_handle* h, void* depth, void* hu, void* hv, void* zb, int where);

/* From a caller's state to a caller's state in one call: sve_set_state of
 * (depth_in, hu_in, hv_in, zb_in), nsteps >= 1 CFL steps (Sec. 3: the time
 * step of each from the CFL condition of its state), then the interior state
 * into (depth_out, hu_out, hv_out, zb_out); row-major ny x nx arrays of the
 * handle's precision, all in the memory `where` names (SVE_HOST or
 * SVE_DEVICE; hv_in / hv_out may be NULL in 1D).  The caller owns all eight
 * buffers; in and out may be the same buffers.  Output buffers in device
 * memory, and in page-locked host memory (cudaHostAlloc, cudaHostRegister)
 * for the two-kernel step (FP64, and FP32 in 1D), are written by the last
 * step's cell update itself, so that with host buffers the result crosses
 * the host link while that kernel computes; other host buffers (pageable,
 * or for the FP32 2D step, whose memory-bound update pass the link would
 * slow down) are copied after the last step.  *t_out (nullable)
 * receives the simulated time (the state's time starts at 0).  Blocks until
 * the result is in place.  Returns SVE_ERR_ARG for a NULL handle or buffer,
 * nsteps < 1 or an unknown `where`, SVE_ERR_CUDA for a failed CUDA call,
 * else the first device error latched by the upload checks or the steps
 * (SVE_ERR_NEG_DEPTH, SVE_ERR_NAN, SVE_ERR_RIEMANN, SVE_ERR_DT); the output
 * buffers then hold the state the steps reached. */
int sve_advance(sve_handle* h, int nsteps, const void* depth_in, const void* hu_in, const void* hv_in,
                const void* zb_in, void* depth_out, void* hu_out, void* hv_out, void* zb_out, int where,
                double* t_out);

/* Diagnostics after the last step: mass_h = sum h dx dy, mass_z = sum zb dx dy
 * (FP64, summed in a fixed order), the simulated time and the last time step.
 * Any pointer may be NULL.  Blocks. */
int sve_get_diag(sve_handle* h, double* mass_h, double* mass_z, double* t, double* last_dt);

/* Time steps of the last sve_step / sve_step_dt call: copies min(n, steps of
 * that call) values into dts (host).  Returns the number copied (>= 0) or an
 * error code. */
int sve_get_dts(sve_handle* h, double* dts, int n);

/* Per-step history (off by default).  sve_set_history(h, capacity) keeps,
 * after every later step, one record of six doubles in a device ring of
 * `capacity` records: t after the step, its dt, mass_h and mass_z of the new
 * state (as sve_get_diag sums them) and the step's extreme wave speeds Sx,
 * Sy (0 in 1D).  capacity 0 switches it off; every call empties the ring,
 * and so does sve_set_state.  Each step then launches one more small kernel,
 * and FP32 2D calls of several steps run their steps one at a time (each
 * step's mass sums are needed).  SVE_ERR_ARG for capacity < 0, SVE_ERR_OOM.
 * sve_get_history copies the last min(n, steps recorded, capacity) records,
 * oldest first, into records (host, 6 doubles each) and returns how many
 * (blocks); SVE_ERR_STATE while the history is off. */
int sve_set_history(sve_handle* h, int capacity);
int sve_get_history(sve_handle* h, double* records, int n);

/* Release everything the handle owns.  NULL is accepted. */
void sve_destroy(sve_handle* h);

/* Static text for a code. */
const char* sve_strerror(int code);

/* Number of kernel launches the last sve_step / sve_step_dt /
 * sve_step_async call enqueued (inside graphs or not). */
long long sve_last_launch_count(sve_handle* h);

/* Enqueue nsteps CFL steps on the handle's stream and return without waiting
 * (the step of Sec. 3, as in sve_step).  Device errors are latched and
 * returned by sve_sync or by any later blocking call. */
int sve_step_async(sve_handle* h, int nsteps);

/* Wait for the handle's enqueued work; return the latched device status. */
int sve_sync(sve_handle* h);

/* Kernel timing.  on != 0: later steps are launched one by one (no graph)
 * and bracketed by CUDA events on the handle's stream; the totals restart
 * at 0.  on == 0 switches it off. */
int sve_profile(sve_handle* h, int on);

/* Device time [ms] and launch count accumulated since sve_profile(h, 1):
 * index 0 = interface kernel or solve pass (Riemann solves), 1 = cell
 * kernel or update pass (in an FP32 2D call of several steps the solve
 * passes, which carry the updates, count under 0 and the call's one update
 * pass under 1).  ms and launches point to two elements each.  Blocks. */
int sve_profile_read(sve_handle* h, double* ms, long long* launches);

/* Counters since the last sve_set_state: steps taken and Newton updates
 * summed over all interface Riemann solves.  Either pointer may be NULL.
 * Blocks; returns the latched device status. */
int sve_get_counters(sve_handle* h, long long* steps, unsigned long long* newton_iters);

/* Safeguards of the Riemann solves taken since the last sve_set_state,
 * summed over all interfaces and steps (Sec. 3: the relaxation solver is
 * well defined for celerities that satisfy the bounds of Eq. (ab), and
 * stronger bounds may be needed):
 *   halvings  Newton steps of the scalar equation in p = tau1 + tau4 that
 *             were halved because the full step made a specific volume
 *             tau_k non-positive (each halving counts one; a halved step
 *             never ends the iteration);
 *   raised    solves whose celerity a was raised by the bed-jump bound
 *             a^2 >= b^2 + 2 g gamma_z |dzb| hmax^2;
 *   retries   doublings of a in solves whose celerities admitted no
 *             solution with positive tau_k (at most 3 per solve; the
 *             solve's wave speeds, and so the CFL step, use the final a;
 *             past the third the step latches SVE_ERR_RIEMANN).
 * Any pointer may be NULL.  Blocks; returns the latched device status
 * (SVE_ERR_STATE without a state, SVE_ERR_ARG for a NULL handle). */
int sve_get_safeguards(sve_handle* h, unsigned long long* halvings, unsigned long long* raised,
                       unsigned long long* retries);

/* ---- launch shape of the two-kernel step -------------------------------------
 * Threads per block of the step's two kernels (interface kernel, cell
 * kernel): 128 (measured fastest on large grids), 256, or 32 (one warp per
 * block) so that a small grid's work is spread over more SMs -- GB300
 * issues ~2 FP64 operations per clock per SM, and a grid of a few thousand
 * interfaces in large blocks would occupy a handful of SMs.  threads = 0
 * (the default at sve_create) picks 32 while a 256-thread interface launch
 * would give fewer than two blocks per SM, else 128.  Results do not depend
 * on it beyond the order of the mass sums.  The 2D FP32 step (column strips
 * marching over runs of rows, with its own launch shape) does not use it.  The step is
 * that of Sec. 3 for every shape; the paper has no counterpart of this
 * choice.  SVE_ERR_ARG for other values. */
int sve_set_block_size(sve_handle* h, int threads);

/* ---- the splitting scheme (comparison) ------------------------------------
 * The end of Sec. 2 of the paper contrasts its coupled method with the usual
 * splitting approach -- a shallow-water step over the time step, then the
 * Exner equation updates the bed -- which it says can create spurious
 * oscillations.  sve_set_scheme(h, SVE_SCHEME_SPLIT) makes the handle's
 * steps that scheme (the paper gives no discretisation of it; this library
 * takes): (1) the coupled step with the transport switched off (Grass law
 * with A_g = 0: the relaxation solver for shallow water over the bed; its
 * CFL time step; friction as configured), the bed held at z^n; (2) the bed
 * updated by a first-order finite-volume Exner step with the configured
 * transport law evaluated on the new flow, the flux through each interface
 * taken from the cell upwind of it by the sign of the sum of the two cells'
 * normal velocities (their mean where that sum is 0: a wall passes no
 * sediment).  SVE_SCHEME_COUPLED (the default) restores the paper's step.
 * FP64 handles without external sides only (SVE_ERR_ARG otherwise); the
 * current state, if any, is re-projected for the new scheme (blocks).  Not
 * for the adjoint (sve_record_forward returns SVE_ERR_ARG while it is on).
 * sve_get_scheme returns the scheme, SVE_ERR_ARG for a NULL handle. */
int sve_set_scheme(sve_handle* h, int scheme);
int sve_get_scheme(sve_handle* h);

/* ---- persistent step of small grids (opt-in) -------------------------------
 * With on = 1 the steps of one call run as cooperative launches of one-warp
 * blocks (all co-resident, spread over the SMs), up to 4096 steps each:
 * per step every interface is solved, a grid-wide barrier, every block
 * takes the same CFL dt, every cell is updated, a grid-wide barrier (Sec.
 * 3's step with the same per-interface and per-cell functions as the
 * two-kernel form: the states and time steps agree to round-off, each kernel
 * being compiled on its own).  Eligible: the two-kernel form (FP64, or FP32
 * in 1D) with at most 4 x SMs one-warp blocks of 32 interfaces or cells,
 * co-resident; otherwise, and for profiled steps (sve_profile), the
 * two-kernel form runs.  on = 0 (the default) restores the two kernels from
 * CUDA graphs, which measured as fast on GB300 (a step of a small grid is
 * bound by one warp's chain of FP64 instructions, not by its launches).
 * Every barrier wait is bounded (~0.5 s of polling); past it the step ends
 * with SVE_ERR_SYNC.  SVE_ERR_ARG for other values.  sve_get_persistent
 * returns 1 if the next steps use it, else 0.
 *
 * sve_check_sync_timeout checks that bounded wait: one persistent launch
 * whose barrier expects one block more than it has, each wait bounded by
 * `polls` polls (~100 ns each); returns SVE_ERR_SYNC as the step would
 * (the state is not advanced), SVE_ERR_ARG if the grid is not eligible,
 * SVE_ERR_STATE without a state. */
int sve_set_persistent(sve_handle* h, int on);
int sve_get_persistent(sve_handle* h);
int sve_check_sync_timeout(sve_handle* h, long long polls);

/* Threads per block the next step call will use (32, 128 or 256). */
int sve_get_block_size(sve_handle* h);

/* ---- batches of independent runs ------------------------------------------
 * An ensemble of runs, each with its own configuration (grid size, bedload
 * and friction parameters, boundaries; all of one precision), its own CFL
 * time step, time and mass sums, stepped together: every step is one launch
 * over all runs' interfaces and one over all their cells, cut into tiles of
 * one run each (a tile table in a schedule order), captured in CUDA graphs.
 * With the FP32 state and every run 2D, the interface launch is the fused
 * FP32 step's solve pass (column strips marching over runs of rows, four
 * strip-runs of one run per block) and the cell launch its update pass;
 * a call of several steps carries each run's update into its next solve
 * pass (as a single handle's call does), one launch a step and one update
 * pass a call.
 * Each run advances as a single handle with the same configuration would:
 * the same per-interface and per-cell code, compiled into other kernels, so
 * results agree to round-off (FMA contraction may differ).  Run r's state
 * arrays follow the single-run conventions with its own nx, ny. */
typedef struct sve_batch sve_batch;

/* cfgs[0..nruns-1]: one validated configuration per run (same precision).
 * Allocates every run's device state; SVE_ERR_ARG / SVE_ERR_OOM. */
int sve_batch_create(const sve_config* cfgs, int nruns, sve_batch** out);
int sve_batch_set_stream(sve_batch* b, void* stream);
/* Copy run `run`'s state in (t of that run reset to 0); checked as in
 * sve_set_state.  Every run needs a state before the first step. */
int sve_batch_set_state(sve_batch* b, int run, const void* depth, const void* hu, const void* hv, const void* zb,
                        int where);
/* Every run advances nsteps of its own CFL steps.  Blocks; returns the first
 * latched device error of any run.  _async: enqueue only. */
int sve_batch_step(sve_batch* b, int nsteps);
int sve_batch_step_async(sve_batch* b, int nsteps);
int sve_batch_get_state(sve_batch* b, int run, void* depth, void* hu, void* hv, void* zb, int where);
int sve_batch_get_diag(sve_batch* b, int run, double* mass_h, double* mass_z, double* t, double* last_dt);
/* Steps and Newton updates summed over all runs since their states were set. */
int sve_batch_get_counters(sve_batch* b, long long* steps, unsigned long long* newton_iters);
/* Time trial_steps steps of every candidate tile size (128, 256 work items)
 * and schedule (0: run after run, largest first; 1: round robin over the
 * runs) -- for the fused FP32 2D form also the rows of a strip-run (8, 16,
 * 32, 64) -- and keep the fastest; the runs' states are restored afterwards.
 * Reports the choice in *tile, *schedule (nullable). */
int sve_batch_autotune(sve_batch* b, int trial_steps, int* tile, int* schedule);
/* The last autotune's candidates: copies min(n, count) entries (tile,
 * schedule, rows -- 0 outside the fused form -- and the mean time of a trial
 * step [ms]) into the nullable arrays and returns the count. */
int sve_batch_autotune_trials(sve_batch* b, int n, int* tile, int* schedule, int* rows, double* ms_per_step);
/* Rows of a strip-run of the fused FP32 2D form (8, 16, 32 or 64; SVE_ERR_ARG
 * otherwise or for another form); sve_batch_get_rows returns the current
 * value (0 outside the fused form). */
int sve_batch_set_rows(sve_batch* b, int rows);
int sve_batch_get_rows(sve_batch* b);
/* Select a tile size and schedule directly. */
int sve_batch_set_schedule(sve_batch* b, int tile, int schedule);
long long sve_batch_last_launch_count(sve_batch* b);
void sve_batch_destroy(sve_batch* b);

/* ---- discrete adjoint ------------------------------------------------------
 * Gradients through nsteps steps of the scheme, with the time steps of the
 * forward run recorded and held fixed: the adjoint of the discrete map
 * U^n -> U^{n+1} (the paper gives the scheme, Sec. 3; its adjoint is this
 * library's addition).  FP64 state; every transport law (Grass, and the
 * Shields-parameter laws with tau* through the friction law).
 *
 * sve_record_forward advances the handle's current state by nsteps CFL
 * steps (as sve_step) and records the time steps and a checkpoint of the
 * conserved state every checkpoint_every steps.  With checkpoint_every <= 0
 * the choice is automatic, within a memory budget (sve_set_adjoint_budget;
 * by default half of the device memory free when the recording starts):
 * when every step's forward data -- its padded state, convected
 * (pre-friction) state and Newton roots, 2 x 32 bytes a cell and 9 bytes an
 * interface a step in 2D -- fit, all of them are kept and the adjoint
 * recomputes nothing; otherwise a checkpoint every ceil(sqrt(nsteps)) steps,
 * and the last segments' forward data are kept as far as the rest of the
 * budget allows (the adjoint recomputes only the earlier segments).  The
 * handle then holds U^N.
 *
 * sve_adjoint propagates a cotangent of the final state back to the
 * recorded run's initial state: lam_h, lam_hu, lam_hv, lam_z = dL/dU^N
 * (nx*ny doubles each, NULL = zero; hv ignored in 1D) in memory `where`;
 * g_h0 .. g_z0 (nullable, same layout and memory) receive dL/dU^0 and
 * g_params[3] (host, nullable) = dL/dA_g, dL/dm_g, dL/d(friction
 * coefficient: K for Strickler, f for Darcy-Weisbach; 0 without friction);
 * with a Shields-parameter law the first two are 0 and the third includes
 * the coefficient's effect through tau*.
 * The forward states are recomputed per checkpoint segment unless the
 * recording kept them all.  Afterwards the handle holds the recorded run's
 * initial state.  SVE_ERR_STATE if nothing was recorded; SVE_ERR_ARG for
 * FP32 handles.
 *
 * sve_get_checkpoint_every returns the recording's checkpoint interval
 * (nsteps when every step was kept), SVE_ERR_STATE if nothing was recorded,
 * SVE_ERR_ARG for a NULL handle.
 *
 * sve_set_adjoint_budget sets the bytes of forward data that the handle's
 * next automatic recordings may keep in device memory (bytes >= 0; -1: half
 * of the free device memory, the default); SVE_ERR_ARG for a NULL handle or
 * bytes < -1.  sve_get_adjoint_kept_steps returns how many of the recorded
 * steps' forward data the recording kept (nsteps when all, 0 with
 * checkpoints only), SVE_ERR_STATE if nothing was recorded. */
int sve_record_forward(sve_handle* h, int nsteps, int checkpoint_every);
int sve_get_checkpoint_every(sve_handle* h);
int sve_set_adjoint_budget(sve_handle* h, long long bytes);
int sve_get_adjoint_kept_steps(sve_handle* h);
int sve_adjoint(sve_handle* h, const void* lam_h, const void* lam_hu, const void* lam_hv, const void* lam_z,
                int where, void* g_h0, void* g_hu0, void* g_hv0, void* g_z0, double* g_params);

/* ---- one block of a decomposed grid ----------------------------------------
 * The domain decomposition of Sec. 4: the grid is cut into blocks, each with
 * one ghost layer filled from the neighbouring blocks before every step, and
 * the time step is the CFL step of the extreme wave speeds over all blocks.
 * A handle for a block is created with the block's cell counts and lengths
 * (the whole grid's dx, dy) and SVE_BC_EXTERNAL on every side that borders
 * another block (the other sides keep their boundary rules).  A step of a
 * decomposed run, after sve_set_state on every block:
 *   1. each block's edge cells to its neighbours: sve_block_get_edge on the
 *      block, sve_block_set_ghosts on the neighbour (the opposite side);
 *   2. sve_block_speeds on every block; the caller takes the maximum of Sx
 *      and of Sy over all blocks (an all-reduce across processes);
 *   3. sve_block_advance on every block with those maxima.
 * The kernels are those of a whole-grid step, so with the same launch shape
 * of the two-kernel step (sve_set_block_size) the decomposed run equals the
 * whole-grid run cell for cell.  The block's own boundary rules refill its
 * other ghosts at every update; external ghosts keep what was set last.
 *
 * sve_block_get_edge copies the interior cells along side (SVE_W: column 0,
 * SVE_E: column nx - 1, SVE_S: row 0, SVE_N: row ny - 1) into edge: four
 * consecutive planes (h, hu, hv, zb) of n values of the state type, n = ny
 * for W/E and nx for S/N (hv zeros in 1D), in memory `where`.  Blocks.
 * sve_block_set_ghosts sets the ghost ring of an EXTERNAL side from the same
 * layout (the neighbour's edge), projecting it as the step projects its
 * ghosts; a non-finite value or a depth <= 0 is latched (SVE_ERR_NAN,
 * SVE_ERR_NEG_DEPTH at the next blocking call).  SVE_ERR_ARG for a side that
 * is not EXTERNAL.  Returns once a host buffer may be reused.
 * sve_block_speeds solves every interface of the block (Sec. 3) and returns
 * its extreme wave speeds max(|lambda1|, |lambda5|) over the x- and the
 * y-interfaces (*sy = 0 in 1D; sy may be NULL); the fluctuations wait for
 * the update.  Blocks; returns the latched device status.
 * sve_block_advance updates the block's cells (Godunov average, friction,
 * checks, boundary-rule ghosts) with the CFL step of the given maxima,
 * dt = cfl dx / sx (1D) or cfl / (sx / dx + sy / dy) (2D): the one every
 * block computes alike.  SVE_ERR_DT if that step is not positive and finite.
 * Blocks; returns the latched device status. */
int sve_block_get_edge(sve_handle* h, int side, void* edge, int where);
int sve_block_set_ghosts(sve_handle* h, int side, const void* ghosts, int where);
int sve_block_speeds(sve_handle* h, double* sx, double* sy);
int sve_block_advance(sve_handle* h, double sx, double sy);

/* ---- stepping without device allocation ----------------------------------
 * The paper has no counterpart of this entry point: it serves callers that
 * cannot call cudaMalloc -- code living under a framework's caching allocator
 * that owns (or has reserved all of) the device memory, real-time loops that
 * must not pay allocation latency or fail for lack of memory mid-run, and
 * plug-ins that are handed device buffers but no allocator.
 *
 * sve_step_noalloc advances the caller's state by nsteps CFL steps with the
 * kernels and arithmetic of sve_create + sve_set_state + sve_step for the
 * same configuration: the two-kernel step in FP64 and in 1D, the marching
 * solve pass and the update pass for the FP32 state in 2D (128-thread blocks for the
 * two-kernel step at every grid size, so the mass sums may be added in
 * another order than a small grid's regular handle adds them).  The caller
 * passes its state as device arrays (depth, hu, hv, zb: nx*ny values of the
 * configured precision, row-major [ny][nx], hv NULL in 1D), updated in
 * place, and the simulated time in *t_inout (host; read, then overwritten
 * with the time after the steps).  stream: a cudaStream_t or NULL (legacy
 * default stream).  The call is host-synchronous: it waits for the input
 * checks, for the steps and for the copy back, reading the device status
 * after each.
 *
 * No memory is allocated: every other buffer (padded state and projection,
 * fluctuations or net fluctuations, block partials, scalars) lives in one
 * file-scope device array of SVE_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until the process exits.  A configuration
 * whose buffers do not fit returns SVE_ERR_NOALLOC_SIZE without touching
 * the state: in FP64 a step needs about 232 bytes per cell (13 padded
 * fields + 8 fluctuation planes per interface), so grids up to about
 * 36 000 cells fit (e.g. 180 x 180); the 2D FP32 state about 68 bytes per
 * cell (about 120 000 cells, e.g. 340 x 340).
 *
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress, with that device current) and the fused step's
 * launch shape; make that first call before any stream capture.  All calls
 * share the array and it keeps the previous call's contents (each call
 * clears what must start at zero): two calls that overlap on the GPU -- on
 * different streams or devices' threads sharing one device -- race on it and
 * must be serialised by the caller.
 * Errors: SVE_ERR_ARG (bad config or pointers), SVE_ERR_NOALLOC_SIZE,
 * SVE_ERR_CUDA, the device errors of the input checks (SVE_ERR_NAN,
 * SVE_ERR_NEG_DEPTH: returned before any step) and of the steps (the first
 * latched one).  On any error the caller's arrays and *t_inout keep their
 * input values. */
#define SVE_NOALLOC_SCRATCH_BYTES (8u << 20)
int sve_step_noalloc(const sve_config* cfg, void* depth, void* hu, void* hv, void* zb, int nsteps, double* t_inout,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SVE_H */
