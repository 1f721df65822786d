/*
 * hydro.h -- C-ABI of the GB300 CTU + PPMC + exact-Riemann hydrodynamics library.
 *
 * One call of hydro_step() advances the 3D Euler equations of an ideal gas
 * (Schneider & Robertson, "Cholla", Sec. 2.1, Eqs. mass_cons ... energy_cons)
 * by one unsplit six-solve Corner Transport Upwind step on a static Cartesian
 * mesh (Sec. 2.3): ghost cells from the boundary conditions (Sec. 3.1), the
 * CFL time step (Eq. calc_dt_3D), PPMC reconstruction with characteristic
 * tracing per axis (App. A.3), the exact Riemann solver (App. B.1), the
 * transverse half-step (Eq. transverse_evolution), a second set of exact
 * Riemann solves and the conserved update (Eq. conserved_update).
 *
 * Conventions for every function below:
 *  - Conserved state arrays are five planes [5][nz][ny][nx] of float64 real
 *    cells, x fastest: rho, rho*u, rho*v, rho*w, E (Sec. 2.1, Eq.
 *    conserved_variables).  There are no ghost cells in caller-visible arrays.
 *  - Cells are cubic (dx = dy = dz).  An axis with one cell is inactive: no
 *    ghost cells, no sweep and no transverse term, so the step reduces to 2D or
 *    1D CTU (Sec. 2.3).  Active axes need at least 4 cells.
 *  - Functions returning int return HYDRO_OK (0) or a negative HYDRO_E* code.
 *    Functions returning double return a value >= 0 on success and a negative
 *    value on error; hydro_last_error() then gives the code.  No function
 *    aborts, traps or waits on the device without a bound.
 *  - The library owns all device memory it allocates (hydro_init .. hydro_free).
 *    Buffers passed by the caller stay owned by the caller; the library copies
 *    from or into them, in order on the handle's stream, and returns only when
 *    the copy has completed.
 *  - Device pointers are plain CUDA device addresses in the current context;
 *    streams are cudaStream_t values passed as void*.  No torch types appear in
 *    this interface.
 *  - A handle must not be used from two host threads at the same time.
 */
#ifndef HYDRO_H
#define HYDRO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hydro_s* hydro_t;

/* Boundary condition of one face (Sec. 3.1): periodic wrap; reflective (mirror
 * copy, normal momentum negated); transmissive/outflow (every ghost copies the
 * outermost real cell); inflow (every ghost holds a prescribed state); Noh
 * (Sec. 4.3.1: every ghost holds the analytic Noh solution at the time t of
 * the step's start and the ghost's centre x, r = |x| over the n active axes:
 * rho = rho0 (1 + V t / r)^(n-1), velocity V toward the origin, E = p0/(gamma-1)
 * + rho V^2/2, with (rho0, V, -, -, p0) given by hydro_set_inflow; single grids
 * only).  Ghosts are filled as passes along x, then y, then z would fill them.
 * Both faces of an axis must be periodic or neither. */
enum {
  HYDRO_BC_PERIODIC = 0,
  HYDRO_BC_REFLECT = 1,
  HYDRO_BC_OUTFLOW = 2,
  HYDRO_BC_INFLOW = 3,
  HYDRO_BC_NOH = 4
};

/* Arithmetic of the step.
 * HYDRO_FP64 (default): every operation in float64; the printed formulas are
 *   evaluated through exact algebraic identities (k-th roots in place of pow,
 *   reciprocals in place of divisions), each result within a few ulp of the
 *   formula as printed.
 * HYDRO_MIXED: reconstruction, Riemann solves and the transverse half-step
 *   (written for the increments of the face states, so that its pressure
 *   recovery has no cancellation) in float32; the conserved update (flux
 *   accumulation), the recovery of the internal energy from E minus the kinetic
 *   energy, the positivity floors and the time step stay float64.
 * HYDRO_FP64_STRICT: float64 with every formula evaluated operation by
 *   operation as printed (divisions, pow, conserved face states between the
 *   reconstruction and the Riemann solver as in App. B.1), for bit-level
 *   reproducibility against a plain CPU implementation; slower. */
enum { HYDRO_FP64 = 0, HYDRO_MIXED = 1, HYDRO_FP64_STRICT = 2 };

/* Reconstruction of the face states (Sec. 2.2.1, App. A).  HYDRO_RECON_PPMC
 * (default): PPM in characteristic variables with characteristic tracing
 * (App. A.3).  HYDRO_RECON_PPMP: PPM in primitive variables with contact
 * steepening, shock flattening and CW84 characteristic tracing (App. A.4; the
 * contact test is d2rho_{i-1} d2rho_{i+1} < 0, as in the method the paper
 * follows, which reproduces its Sod result).  HYDRO_RECON_PLMC: piecewise
 * linear, characteristic limiting and tracing (App. A.2).  HYDRO_RECON_PLMP:
 * piecewise linear, primitive limiting, half-step flux evolution (App. A.1).
 * HYDRO_RECON_PCM: piecewise constant (Sec. 2.2.1).  PPMP needs three cells on
 * each side of a cell, the others one or two; every mode fits the 4 ghost
 * layers. */
/* Riemann solver (Sec. 2.2.2).  HYDRO_RIEMANN_EXACT (default): the exact
 * solver of App. B.1.  HYDRO_RIEMANN_ROE: the Roe solver with the HLLE
 * fallback for negative intermediate states (App. B.2) in both sets of solves
 * and the H correction (App. C) in the second; its eta is half the largest
 * jump of u + a and u - a across a face (the paper prints the u + a term). */
enum { HYDRO_RIEMANN_EXACT = 0, HYDRO_RIEMANN_ROE = 1 };

enum {
  HYDRO_RECON_PPMC = 0,
  HYDRO_RECON_PPMP = 1,
  HYDRO_RECON_PLMC = 2,
  HYDRO_RECON_PLMP = 3,
  HYDRO_RECON_PCM = 4
};

enum {
  HYDRO_OK = 0,
  HYDRO_EINVAL = -1,    /* invalid argument (sizes, bc, gamma, dx, null pointer, face) */
  HYDRO_ENOMEM = -2,    /* device or host allocation failed */
  HYDRO_ECUDA = -3,     /* a CUDA runtime call failed (see hydro_cuda_error_string) */
  HYDRO_ENONPHYS = -4,  /* after a step some real cell has rho <= 0 or a NaN */
  HYDRO_ENEWTON = -5,   /* a Riemann solve reached the 50-iteration Newton cap */
  HYDRO_ENOSTATE = -6   /* a step or dt was requested before hydro_set_state */
};

/* Create a grid of nx*ny*nz real cells of width dx for an ideal gas of index
 * gamma (> 1).  bc[6] lists the faces x-, x+, y-, y+, z-, z+.  Allocates all
 * device memory the step needs (about 450 bytes per padded cell in float64).
 * The padded grid ((n+8) cells along each active axis) must have fewer than
 * 2^31 cells (about 1290^3, more than the device holds), else HYDRO_EINVAL.
 * On success *out holds the handle; on error *out is NULL. */
int hydro_init(hydro_t* out, int nx, int ny, int nz, double dx, double gamma, const int bc[6]);

/* Prescribed primitive state (rho, u, v, w, p) of an HYDRO_BC_INFLOW face, or
 * (rho0, V, -, -, p0) of an HYDRO_BC_NOH face (0..5 in the order of bc[]).  Host
 * pointer, copied.  HYDRO_EINVAL unless rho > 0 and p >= 0. */
int hydro_set_inflow(hydro_t h, int face, const double prim[5]);

/* Time t at the start of the next step, which the Noh boundary reads: 0 after
 * hydro_init, advanced by every step's dt on the device (hydro_set_state leaves
 * it).  Set it (t >= 0, else HYDRO_EINVAL) to start a run at another time; read
 * it back after steps. */
int hydro_set_time(hydro_t h, double t);
/* The time (see hydro_set_time); waits for the handle's stream.  A negative
 * value is an error code. */
double hydro_get_time(hydro_t h);

/* Select HYDRO_FP64 (default), HYDRO_MIXED or HYDRO_FP64_STRICT for the
 * following steps. */
int hydro_set_precision(hydro_t h, int mode);

/* Threads a block of the HYDRO_FP64 and HYDRO_MIXED launches: 128 or 256, or 0
 * for the library's choice (the default, 128: never slower than 256 in
 * measurements from a 512-cell tube to 256^3, faster on small grids, which
 * spread over more SMs).  The arithmetic per cell does not depend on it and the
 * dt is a maximum over cells, so FP64 results are the same bit for bit; in
 * HYDRO_MIXED the cell whose signal speed is evaluated in FP64 is picked per
 * block, so dt can differ within 10 * 2^-24 relative where two cells' float
 * estimates tie.  HYDRO_EINVAL for other values.  HYDRO_FP64_STRICT always
 * uses 256. */
int hydro_set_block_size(hydro_t h, int bs);
/* The block size in use (128 or 256), or a negative error code. */
int hydro_block_size(hydro_t h);

/* Stream on which all following work of this handle is ordered (a
 * cudaStream_t; NULL = the legacy default stream). */
int hydro_set_stream(hydro_t h, void* stream);

/* Copy a conserved state [5][nz][ny][nx] float64 into the handle.  u is a
 * device pointer if on_device != 0, else a host pointer. */
int hydro_set_state(hydro_t h, const double* u, int on_device);

/* Copy the current conserved state out, same layout as hydro_set_state. */
int hydro_get_state(hydro_t h, double* u, int on_device);

/* Advance one CTU step with dt = cfl * min over real cells and active axes of
 * dx/(|v_d| + a), a = sqrt(gamma p / rho) (Eq. calc_dt_3D; the paper requires
 * cfl < 0.5 for the six-solve CTU).  Returns the dt used, or a negative value
 * on error (then hydro_last_error() is HYDRO_ENONPHYS, HYDRO_ENEWTON, ...; the
 * state is the result of the step even then). */
double hydro_step(hydro_t h, double cfl);

/* Advance one CTU step with a caller-chosen dt (> 0), e.g. to land exactly on a
 * final time.  Returns dt, or a negative value on error. */
double hydro_step_dt(hydro_t h, double dt);

/* The dt that hydro_step(h, cfl) would use now, without changing the state. */
double hydro_compute_dt(hydro_t h, double cfl);

/* Asynchronous forms, for pipelines that overlap one handle's copies with
 * another's steps: each enqueues its work on the handle's stream and returns
 * without waiting.  A host pointer must stay valid until the copy has run and
 * should be page-locked memory (cudaHostAlloc, a pinned torch tensor): copies
 * from pageable memory do not overlap.  hydro_step_async takes one CFL step as
 * hydro_step does but leaves dt and the status word on the device; it is not
 * timed by the tracing (its launches are counted).  The status word of async
 * steps accumulates until hydro_sync reads it; a synchronous hydro_step,
 * hydro_step_dt or hydro_advance clears it first, so call hydro_sync before
 * them.  Return HYDRO_OK, HYDRO_EINVAL, HYDRO_ENOSTATE or HYDRO_ECUDA. */
int hydro_set_state_async(hydro_t h, const double* u, int on_device);
int hydro_get_state_async(hydro_t h, double* u, int on_device);
int hydro_step_async(hydro_t h, double cfl);
/* Wait for the handle's stream.  Returns HYDRO_OK, or HYDRO_ENONPHYS /
 * HYDRO_ENEWTON if a step since the last synchronous step or hydro_sync raised
 * that status (then cleared); *dt_out (may be NULL) receives the last step's
 * dt. */
int hydro_sync(hydro_t h, double* dt_out);

/* Advance with CFL steps (as hydro_step(h, cfl)) until the time (see
 * hydro_set_time) reaches t_end, or max_steps steps were taken, without a host
 * round trip per step: the steps run as a loop inside one CUDA graph (a
 * conditional WHILE node), whose dt kernel shortens the step that would pass
 * t_end to t_end - t and then sets the time to t_end exactly -- the same dt
 * sequence and final time as a host loop of hydro_compute_dt / hydro_step_dt
 * that does so.  t_end = +INFINITY takes exactly max_steps steps.  A graph
 * launch runs at most about 2^26 cell updates (>= 1 step); the host relaunches
 * until done, reading the 88-byte step record once per launch.  The graph is
 * captured on the first call and again when cfl, the precision, reconstruction
 * or Riemann solver, or an inflow state changed.  Steps are counted in the launch
 * counter of hydro_profile_read but get no per-stage times.
 * Returns HYDRO_OK, HYDRO_EINVAL (cfl <= 0, t_end NaN, max_steps < 0 or
 * > 2^52), HYDRO_ENOSTATE, or the error of a step (HYDRO_ENONPHYS,
 * HYDRO_ENEWTON): the run stops after that step and the state is its result.
 * *steps_out (may be NULL) receives the number of steps taken, also on error. */
int hydro_advance(hydro_t h, double cfl, double t_end, long long max_steps, long long* steps_out);

/* Code of the last error on this handle (HYDRO_OK if the last call succeeded). */
int hydro_last_error(hydro_t h);

/* Static description of a HYDRO_E* code. */
const char* hydro_error_string(int code);

/* Text of the last CUDA runtime error seen by this handle ("" if none). */
const char* hydro_cuda_error_string(hydro_t h);

/* ---- tracing -----------------------------------------------------------------
 * Stages of a step, in launch order: 0 ghost remap + primitives (+ dt minimum),
 * 1 dt, 2 limited slopes (per axis), 3 PPMC face states (per axis), 4 first
 * Riemann fluxes (per axis), 5 transverse half-step + CTU fluxes (per axis),
 * 6 conserved update.  The paper times the GPU hydro step as a whole (Sec.
 * 3.5.3); this adds the per-stage split. */
#define HYDRO_NUM_STAGES 7

/* Enable (1) or disable (0) per-stage timing: each kernel launch of a step is
 * bracketed by CUDA events on the handle's stream.  Either call resets the
 * accumulated totals and the launch counter. */
int hydro_profile(hydro_t h, int enable);

/* Totals since the last hydro_profile() call, for the first nstages stages
 * (<= HYDRO_NUM_STAGES): device milliseconds, number of launches and number of
 * cells or faces processed, per stage; plus the total number of kernel launches
 * (counted whether or not timing is enabled).  Any output pointer may be NULL. */
int hydro_profile_read(hydro_t h, int nstages, double* ms, long long* launches, long long* units,
                       long long* launches_total);

/* Select the reconstruction (HYDRO_RECON_*) of the following steps.  The
 * non-default modes run in HYDRO_FP64 and HYDRO_FP64_STRICT; with HYDRO_MIXED
 * they are rejected (HYDRO_EINVAL), as is an unknown mode. */
int hydro_set_reconstruction(hydro_t h, int recon);

/* Select the Riemann solver (HYDRO_RIEMANN_*) of the following steps.  The Roe
 * solver runs in HYDRO_FP64 and HYDRO_FP64_STRICT (HYDRO_EINVAL with
 * HYDRO_MIXED or an unknown solver); selecting it allocates one plane per
 * active axis for the H correction (HYDRO_ENOMEM if that fails). */
int hydro_set_riemann_solver(hydro_t h, int solver);

/* Release the handle and all device memory it owns.  NULL is accepted. */
void hydro_free(hydro_t h);

/* ---- batches of independent grids ----------------------------------------------
 * Many grids of uneven sizes (and boundary conditions, gamma, dx) advanced
 * together: each stage of the step is one kernel launch over all grids, every
 * grid keeps its own CFL time step, and the steps of one hydro_batch_step call
 * are captured once into a CUDA graph and replayed with one graph launch (the
 * paper suggests running many problems at once, Sec. 5).  Conventions as for
 * single grids; `grid` indexes 0..ngrids-1. */
typedef struct hydro_batch_s* hydro_batch_t;

/* dims: [ngrids][3] (nx, ny, nz); dx, gamma: [ngrids]; bc: [ngrids][6].
 * Each grid obeys the size rules of hydro_init (HYDRO_EINVAL otherwise).
 * Allocates the device memory of all grids (one allocation). */
int hydro_batch_init(hydro_batch_t* out, int ngrids, const int* dims, const double* dx,
                     const double* gamma, const int* bc);
int hydro_batch_set_inflow(hydro_batch_t h, int grid, int face, const double prim[5]);
/* HYDRO_FP64 (default) or HYDRO_MIXED. */
int hydro_batch_set_precision(hydro_batch_t h, int mode);
/* A non-default stream (graph capture needs one); the batch creates its own
 * otherwise. */
int hydro_batch_set_stream(hydro_batch_t h, void* stream);
int hydro_batch_set_state(hydro_batch_t h, int grid, const double* u, int on_device);
int hydro_batch_get_state(hydro_batch_t h, int grid, double* u, int on_device);
/* Advance every grid by nsteps CTU steps, each with its own dt = cfl * min
 * dx/(|v_d| + a) of that grid.  dt_out (host, may be NULL): [nsteps][ngrids].
 * The first call with a given (nsteps, cfl, precision, schedule) captures the
 * graph; later calls replay it.  Returns HYDRO_OK or an error code (a
 * non-physical state or a Newton cap in any grid is reported after the call). */
int hydro_batch_step(hydro_batch_t h, double cfl, int nsteps, double* dt_out);
/* Asynchronous forms of hydro_batch_set_state, hydro_batch_get_state and
 * hydro_batch_step (as for single grids: enqueued on the batch's stream, no
 * wait; host buffers should be page-locked and stay valid until the copy has
 * run).  Each graph launch starts from a cleared status word, so
 * hydro_batch_sync reports the status of the last hydro_batch_step_async:
 * call it after each one (a pipeline syncs one batch while the next one's work
 * is queued).  No dt history is returned. */
int hydro_batch_set_state_async(hydro_batch_t h, int grid, const double* u, int on_device);
int hydro_batch_get_state_async(hydro_batch_t h, int grid, double* u, int on_device);
int hydro_batch_step_async(hydro_batch_t h, double cfl, int nsteps);
/* Wait for the batch's stream; HYDRO_OK, or HYDRO_ENONPHYS / HYDRO_ENEWTON if
 * a grid of the last step call raised that status. */
int hydro_batch_sync(hydro_batch_t h);

/* Choose the launch schedule -- threads per block (128 or 256) and the order of
 * the grids' blocks (as given, or largest grid first) -- by timing one step of
 * each candidate from the current states (restored afterwards).  With
 * use_cache != 0 a previous choice for the same grid sizes, precision and
 * device is read from the cache file ($HYDRO_TUNE_CACHE, else
 * ~/.cache/hydro_gb300_batch_tune.txt) instead; every new choice is appended
 * there.  Outputs (may be NULL): the chosen block size and order, and its
 * measured ms a step (-1 when taken from the cache). */
int hydro_batch_autotune(hydro_batch_t h, int use_cache, int* block_size, int* order,
                         float* ms_per_step);
/* Reconstruction of every grid of the batch (as hydro_set_reconstruction). */
int hydro_batch_set_reconstruction(hydro_batch_t h, int recon);
/* Riemann solver of every grid of the batch (as hydro_set_riemann_solver). */
int hydro_batch_set_riemann_solver(hydro_batch_t h, int solver);
int hydro_batch_last_error(hydro_batch_t h);
const char* hydro_batch_cuda_error_string(hydro_batch_t h);
void hydro_batch_free(hydro_batch_t h);

/* ---- time step without allocation ---------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc (their device memory is owned by another allocator, or
 * an allocation's possible device synchronization is not acceptable).
 *
 * dt = cfl * min over cells and active axes of dx/(|v_d| + a) for a state held
 * by the caller: u is a device pointer to [5][nz][ny][nx] float64 conserved
 * variables, dt_out a device pointer to one double.  Enqueued on `stream`; the
 * result is valid once the stream reaches it.  Allocates nothing: its scratch is
 * a static device array of 65536 doubles (512 KiB) that every GPU loading the
 * library holds until exit, so states of more than 2^24 cells are rejected with
 * HYDRO_EINVAL.  Calls share that array: calls overlapping on the GPU race.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and should come before any stream capture; the address is kept for the life of
 * the process, so the entry point must not be used across a cudaDeviceReset.
 * The state is not checked on the host: a cell with rho <= 0, or a NaN in any
 * cell, gives *dt_out = NaN (the call still returns HYDRO_OK), so test the
 * result; the handle path rejects such states in hydro_set_state instead.  The
 * result equals hydro_compute_dt's in HYDRO_FP64_STRICT bit for bit and agrees
 * with HYDRO_FP64's to a few ulp.  Returns HYDRO_OK, HYDRO_EINVAL or HYDRO_ECUDA. */
int hydro_compute_dt_noalloc(const double* u, int nx, int ny, int nz, double dx, double gamma,
                             double cfl, double* dt_out, void* stream);

/* ---- building blocks of the step, exposed on device arrays ------------------
 * Both read and write device memory laid out as structure-of-arrays planes of
 * n entries each, enqueue on `stream` and return after the launch has been
 * enqueued (they do not wait for completion). */

/* Exact Riemann solver (App. B.1) on n interfaces.  UL, UR: conserved states
 * [5][n] in sweep order (rho, normal momentum, two transverse momenta, E); the
 * pressure derived from them is floored at 1e-20.  F: fluxes [5][n] in the same
 * order.  flags: one int on the device, OR-ed with 1 when a solve hits the
 * Newton cap. */
int hydro_riemann_exact(int n, const double* UL, const double* UR, double gamma, double* F,
                        int* flags, void* stream);

/* PPMC reconstruction with characteristic tracing (App. A.3) of n cells.
 * w: primitive stencils [5 cells][5 variables][n] (cells i-2..i+2; variables
 * rho, normal velocity, two transverse velocities, p); dtdx = dt/dx.  WsL, WsR:
 * the time-evolved primitive states [5][n] at the left and right face of cell i. */
int hydro_ppmc(int n, const double* w, double dtdx, double gamma, double* WsL, double* WsR,
               void* stream);

/* ---- library self-check ---------------------------------------------------------
 * The paper has no counterpart to this entry point.  The mixed-precision kernels
 * convert between float and double with integer arithmetic instead of the
 * hardware conversion instructions (which run at the FP64 rate); this compares
 * those conversions with the hardware ones on the current device: the widening
 * for all 2^32 float bit patterns, the narrowing (round to nearest even) for
 * 2^30 double bit patterns drawn from a counter-based hash, concentrated on the
 * float range's edges and on rounding ties.  Expected: the hardware's bits for
 * normal values, zeros and infinities; a zero of the same sign where the value
 * (or, narrowing, the double operand) lies below the float normal range; NaN
 * for NaN.  mismatches: host array of two counts (widening, narrowing), both 0
 * when every case agrees.
 * Runs on `stream` and waits for it; allocates 16 bytes of device memory.
 * Returns HYDRO_OK, HYDRO_EINVAL (mismatches NULL) or HYDRO_ECUDA. */
int hydro_check_conversions(unsigned long long* mismatches, void* stream);

/* Self-check of the integer-pipe FP64 helpers of the kernels (GB300 issues
 * FP64 adds, multiplies and compares on its FP64 pipe at 1/64 of the float
 * rate): halving and doubling by moving the exponent field (shifting the
 * magnitude at the subnormal edge, rounding to even), the sign tests of a
 * product x*y from the factors' bits and of a product of differences
 * (a-b)(c-d) from the operands' order, against the FP64 arithmetic; and the
 * mixed update's conversion of a float-float sum to one double, against the
 * FP64 add (within one ulp).  2^30 counter-hashed cases, concentrated on the
 * exponent range's edges.  mismatches: host array of four counts (halving,
 * doubling, sign tests, float-float sums; the sign tests skip products that
 * underflow to zero or are NaN and differences of +0 and -0), all 0 when every
 * case agrees.  Runs on `stream` and waits for it; allocates 32 bytes of device
 * memory.  Returns HYDRO_OK, HYDRO_EINVAL (mismatches NULL) or HYDRO_ECUDA. */
int hydro_check_scaling(unsigned long long* mismatches, void* stream);

/* Self-check of the kernels' FP64 operations refined from hardware seeds by
 * Newton-type iterations (the fast FP64 path replaces IEEE division and square
 * root, about ten FP64 issue slots each on GB300, by three to eight): the
 * reciprocal, the quotient and the square root against CUDA's correctly rounded
 * __drcp_rn, __ddiv_rn and __dsqrt_rn; the reciprocal square root, and the
 * reciprocal roots sigma^(-1/5) and sigma^(-1/2) of the exact solver's pressure
 * function (sigma in [1e-30, 1e30]), against the nearest double to the exact
 * value (a correction with the residual 1 - sigma t^m in double-double
 * arithmetic).  2^26 counter-hashed positive normal operands each (binades
 * -500..500 for the reciprocal, square root and reciprocal square root,
 * -200..200 for the quotient's operands).  max_ulp: host array of six largest
 * distances in ulps (reciprocal, quotient, square root, reciprocal square root,
 * fifth root, square-root form).  Runs on `stream` and waits for it; allocates
 * 48 bytes of device memory.  Returns HYDRO_OK, HYDRO_EINVAL (max_ulp NULL) or
 * HYDRO_ECUDA. */
int hydro_check_newton(unsigned long long* max_ulp, void* stream);

/* The paper has no counterpart to this entry point.  Measured FP64 throughput
 * of the current device, the ceiling of the FP64 path (bound by its FP64 pipe):
 * a kernel of independent fused multiply-add chains on every SM (152 x 8
 * blocks of 256 threads, 8 chains of 4096 FMAs a thread), timed with CUDA
 * events on `stream`, the fastest of three launches after a warm-up.
 * flops_per_s: host double receiving 2 flops per FMA over that time.  Waits
 * for the stream; allocates nothing.  Returns HYDRO_OK, HYDRO_EINVAL
 * (flops_per_s NULL) or HYDRO_ECUDA. */
int hydro_probe_fp64_rate(double* flops_per_s, void* stream);

/* Host-only self-check of the integer division the kernels' index arithmetic
 * uses (a multiply-high and a shift by constants formed per grid, in place of
 * an integer division; valid for numerators below 2^31, which the size rules
 * above guarantee): compares it with plain division for every divisor up to
 * 2^16 and 200000 hashed divisors up to 2^31 - 1, at edge and hashed
 * numerators.  Needs no GPU.  Returns the number of mismatches (0 expected). */
long long hydro_check_fastdiv(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
