/*
 * teno7.h -- C ABI of the GB300 (sm_103a) implementation of the extended
 * seventh-order TENO scheme ("TENO7-ext") of F. Zhang, J. Liu, H. Zhang and
 * C. Xu, "An extending strategy based on TENO framework for hyperbolic
 * conservation laws", arXiv:1808.00037.
 *
 * The method (the paper's Sections 2-4):
 *   - conservative finite differences, du_i/dt = -(f_{i+1/2} - f_{i-1/2})/dx
 *     (Eq. app), with global Lax-Friedrichs flux splitting and Roe-averaged
 *     characteristic projection for the Euler equations (Remark 3; Sec.
 *     "One dimensional Euler equations");
 *   - per face, the five-point TENO smoothness measure on three 3-point
 *     stencils (Eqs. smooth_expl, tau5, TENO1 with C = 1, q = 6, norm,
 *     seclect with C_T = 1e-5, epsilon = dx^3);
 *   - the binary vector Delta_i built from this face's and the two neighbouring
 *     faces' cutoff bits (Eq. vec), which selects one of 13 polynomials
 *     (Table co3) whose coefficients are Table co2;
 *   - the third-order SSP Runge-Kutta method in time (Sec. 2.1).
 *
 * Conventions for every call:
 *   - Device arrays are caller-owned, contiguous, and hold `double` for
 *     T7_F64 and `float` for T7_F32 contexts.  Conserved variables are
 *     variable-major ("SoA"): 1D [m][nx], 2D [m][ny][nx] with x fastest;
 *     (rho, rho u, E) for 1D Euler, (rho, rho u, rho v, E) for 2D Euler, u for
 *     the scalar laws.
 *   - The library owns only the workspace inside a t7_ctx (two stage buffers,
 *     a host-API state buffer and a small control block).
 *   - Calls are asynchronous on the context's stream unless stated.  Device-
 *     side errors (non-physical or non-finite states) are latched in the
 *     control block and returned by the next synchronising call (t7_sync,
 *     t7_cfl_dt, t7_run, t7_run_host), which clears them.  A cell holding
 *     Inf or NaN gives T7_ENONFINITE; a finite one with rho <= 0 or p <= 0, or
 *     a Roe frame with c^2 <= 0, gives T7_ENONPHYSICAL, which wins when both
 *     occurred (a state that went non-physical and then produced NaN).
 *     t7_last_error() names the lowest flat cell index (1D: i; 2D: y nx + x;
 *     batches: the index in the concatenated array) near which one was met.
 *   - Checked build (libteno7_checked.so, compiled with T7_CHECKED=1, a
 *     stand-in for a memory checker): every cell, row and column index a
 *     kernel forms for a global-memory access is tested against the extent of
 *     the array; a failing one is latched, the access is clamped into the
 *     array, and the next synchronising call returns T7_EINDEX (before any
 *     other status) with the lowest failing index in t7_last_error().  The
 *     release build never returns T7_EINDEX.
 *   - A call never aborts the process; it returns a t7_status and, on
 *     failure, t7_last_error() describes the cause.
 */
#ifndef TENO7_H
#define TENO7_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    T7_OK = 0,
    T7_EINVAL = -1,       /* bad argument: null pointer, size, enum value    */
    T7_ECUDA = -2,        /* a CUDA runtime call failed                       */
    T7_ENONPHYSICAL = -3, /* rho <= 0, p <= 0 or Roe c^2 <= 0 was met          */
    T7_ENONFINITE = -4,   /* Inf/NaN met (or the "no exist" pattern of Table co3) */
    T7_ETIMEOUT = -5,     /* a bounded device wait gave up                    */
    T7_ENOMEM = -6,       /* workspace allocation failed                      */
    T7_EINDEX = -7        /* checked build only: an array index failed its check */
} t7_status;

typedef enum { T7_BC_PERIODIC = 0, T7_BC_ZERO_GRADIENT = 1 /* = transmissive */ } t7_bc;
/* T7_MIXED: state arrays in FP64; the reconstruction (frame, projection,
 * smoothness measures, selection, polynomials, face flux) runs in FP32 and the
 * flux difference and RK combination in FP64, so domain sums are conserved
 * to FP64 round-off.  Provided for the 1D and 2D systems (t7_euler_rhs,
 * t7_cfl_dt, t7_rk3_step, t7_run, t7_run_host); the reconstruction, batch,
 * adjoint and no-allocation entry points return T7_EINVAL. */
typedef enum { T7_F64 = 0, T7_F32 = 1, T7_MIXED = 2 } t7_prec;
typedef enum { T7_SCALAR_ADVECTION = 0, T7_EULER1D = 1, T7_EULER2D = 2, T7_BURGERS = 3 } t7_system;
/* T7_TENO7EXT: the paper's scheme.  T7_TENO5: the fifth-order TENO scheme
 * it is compared with (Sec. 2, Table co1: each face picks one of seven
 * five-point polynomials from its own three cutoff bits), provided for the
 * 1D systems through t7_euler_rhs, t7_cfl_dt, t7_rk3_step, t7_run and
 * t7_run_host; the other entry points reject a TENO5 context (T7_EINVAL). */
typedef enum { T7_TENO7EXT = 0, T7_TENO5 = 1 } t7_scheme;
/* Lax-Friedrichs splitting.  T7_ALPHA_GLOBAL: one alpha = max_i (|u_i| + c_i)
 * over the domain, the paper's global Lax-Friedrichs splitting (Sec. "One
 * dimensional Euler equations").  T7_ALPHA_PER_FIELD: one alpha per
 * characteristic field, alpha_k = max_i |lambda_k(U_i)| (1D Euler: u - c, u,
 * u + c), each field's split values formed from the projections of the flux
 * and the state in the face's frame, q+-_k = (L_k F +- alpha_k L_k U) / 2;
 * the CFL step is that of the global alpha (the largest alpha_k equals it).
 * Provided for 1D Euler in FP64 and FP32 with TENO7-ext through t7_euler_rhs,
 * t7_cfl_dt, t7_rk3_step and t7_run; any other combination is refused by
 * t7_create, and the other entry points refuse such a context (T7_EINVAL). */
typedef enum { T7_ALPHA_GLOBAL = 0, T7_ALPHA_PER_FIELD = 1 } t7_alpha_mode;

/* Grid and parameters of one problem.  Cell-centred uniform grid with cell
 * widths dx, dy; four ghost cells per side are built inside the kernels from
 * bc[] = {x_lo, x_hi, y_lo, y_hi} (y entries ignored in 1D).
 *   gamma     ratio of specific heats (Euler; the paper uses 1.4)
 *   adv_speed a in u_t + a u_x = 0 (scalar advection)
 *   CT        cutoff C_T of Eq. seclect (the paper uses 1e-5)
 *   eps_x/y   epsilon of Eq. TENO1; a negative value selects dx^3 (dy^3),
 *             the paper's choice (Sec. "The parameter epsilon"), or 1e-40
 *             for TENO5 (the value given with Eq. TENO1).
 *   scheme    t7_scheme (zero-initialised grids get TENO7-ext).  In FP32,
 *             TENO5's epsilon is raised to FLT_MIN (1e-40 is subnormal).
 *   alpha_mode t7_alpha_mode (zero-initialised grids get the global alpha). */
typedef struct {
    int sys;  /* t7_system */
    int prec; /* t7_prec   */
    int nx, ny; /* ny = 1 for 1D systems */
    double dx, dy;
    int bc[4];
    double gamma, adv_speed, CT, eps_x, eps_y;
    int scheme; /* t7_scheme */
    int alpha_mode; /* t7_alpha_mode */
} t7_grid;

typedef struct t7_ctx t7_ctx;

/* Context management (t7_create .. t7_sync) has no counterpart in the paper:
 * it holds the problem statement of Sec. 2 (the grid, the conservation law,
 * the boundary conditions) and the device workspace the other calls use.
 *
 * Create a context on the current CUDA device bound to `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Allocates the workspace
 * (3 state-sized buffers + a control block).  On success *out owns it. */
t7_status t7_create(const t7_grid *grid, void *stream, t7_ctx **out);
/* Free the context and its workspace (T7_EINVAL for NULL).  The caller makes
 * sure no work of the context is still queued.  (Context management: no
 * counterpart in the paper.) */
t7_status t7_destroy(t7_ctx *ctx);
/* Later calls run on `stream`.  Work already queued on the previous stream is
 * ordered before them (the new stream waits on an event recorded on the old
 * one), so the switch needs no synchronisation by the caller.  (Context
 * management: no counterpart in the paper.) */
t7_status t7_set_stream(t7_ctx *ctx, void *stream);
/* Last error message of this context (never NULL; no counterpart in the paper). */
const char *t7_last_error(const t7_ctx *ctx);
/* Block until the stream is idle; return and clear any latched device error
 * (no counterpart in the paper). */
t7_status t7_sync(t7_ctx *ctx);

/* Scalar TENO7-ext reconstruction of one sequence of point values
 * (Eqs. smooth_expl .. seclect, Eq. vec, Tables co2/co3).
 *   v_padded  device, n + 8 values at cells -4 .. n+3 (caller-padded)
 *   sign      +1: reconstruction upwind from the left; -1: its mirror image
 *   eps       epsilon of Eq. TENO1 (> 0)
 *   fhat      device, n + 1 face values at i+1/2, i = -1 .. n-1
 *   d3        device or NULL, n + 3 bytes: cutoff bits (d0 | d1<<1 | d2<<2)
 *             of faces -2 .. n
 *   D5        device or NULL, n + 1 bytes: Delta_i of faces -1 .. n-1 packed
 *             with its first component in bit 4 and its last in bit 0.
 * Uses the context's precision and CT; the system is irrelevant.  Async. */
t7_status t7_teno7_reconstruct(t7_ctx *ctx, const void *v_padded, int n, int sign, double eps, void *fhat,
                               uint8_t *d3, uint8_t *D5);

/* Right-hand side L(U) = -(F_{i+1/2} - F_{i-1/2})/dx (Eq. app) of the
 * context's 1D system, characteristic-wise with global Lax-Friedrichs
 * splitting, alpha = max_i (|u_i| + c_i) over the interior cells of U.
 *   U, dUdt   device, [m][nx]
 *   masks     device or NULL, [2][m][nx+1] bytes: Delta_i of the '+' (index 0)
 *             and '-' (index 1) splits per characteristic field and face
 *             i+1/2, i = -1 .. nx-1.  Async. */
t7_status t7_euler_rhs(t7_ctx *ctx, const void *U, void *dUdt, uint8_t *masks);

/* Time step from the CFL condition of the global Lax-Friedrichs scheme (Sec.
 * "One dimensional Euler equations": one alpha = max_i (|u_i| + c_i) over the
 * whole domain, the same alpha that splits the flux): dt = CFL dx / alpha(U)
 * in 1D, CFL / (alpha_x/dx + alpha_y/dy) in 2D.  U: device, the context's
 * layout.  Synchronises; *dt_out is a host double.  Non-physical or
 * non-finite cells return their status and leave *dt_out unset. */
t7_status t7_cfl_dt(t7_ctx *ctx, const void *U, double cfl, double *dt_out);

/* One step of the third-order SSP Runge-Kutta method (Sec. 2.1, Gottlieb-Shu;
 * the paper omits the formula, so the Shu-Osher form is used):
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 *   U  = 1/3 U + 2/3 (U2 + dt L(U2)),
 * each L the right-hand side of t7_euler_rhs with alpha recomputed from that
 * stage's state.  In place on device U (the context's layout), fixed dt > 0.
 * Async; non-physical or non-finite states met are latched and returned by
 * the next synchronising call. */
t7_status t7_rk3_step(t7_ctx *ctx, void *U, double dt);

/* March device U in place with t7_rk3_step's SSP-RK3 steps (Sec. 2.1) until
 * t_end (last step clipped to land on it) or max_steps steps, each step's dt
 * the CFL step of t7_cfl_dt (Sec. "One dimensional Euler equations"),
 * dt = CFL dx / alpha(U^n), computed on the device.  t_end may be +inf.
 * Synchronises; steps_out / t_out (host, nullable). */
t7_status t7_run(t7_ctx *ctx, void *U, double cfl, double t_end, int max_steps, int *steps_out, double *t_out);

/* As t7_run (SSP-RK3 steps of Sec. 2.1 at the CFL step) on a HOST array U_host ([m][nx],
 * context precision; pageable or page-locked): copies it to the context's
 * device state, runs, copies the result back.  With t_end = +inf (a known step count) on a 1D system the
 * result leaves in parts while the last stage computes.  Synchronises. */
t7_status t7_run_host(t7_ctx *ctx, void *U_host, double cfl, double t_end, int max_steps, int *steps_out,
                      double *t_out);

/* The paper has no adjoint; the adjoint calls differentiate its scheme (the
 * RHS of Eq. app with the TENO7-ext selection frozen, and the SSP-RK3 step of
 * Sec. 2.1) exactly.
 *
 * Discrete adjoint of t7_euler_rhs for 1D Euler: out = (dL/dU)^T v at the
 * state U, with the stencil selection (every Delta_i of both splits and all
 * fields) and the global Lax-Friedrichs alpha frozen at their values for U;
 * the Roe frame, the characteristic projection, the split fluxes and the flux
 * difference are differentiated exactly.  U, v, out: device [3][nx].  Async.
 * (FP32 contexts take the masks from a forward evaluation of U, so the
 * selection is the forward kernel's bit for bit.) */
t7_status t7_euler_rhs_adjoint(t7_ctx *ctx, const void *U, const void *v, void *out);

/* Adjoint of one SSP-RK3 step (Sec. 2.1) of size dt from the state U (the step's start,
 * unchanged): recomputes the stage states, then maps lambda (device [3][nx],
 * the adjoint of the step's result) in place to the adjoint of U:
 *   U1 = U + dt L(U); U2 = 3/4 U + 1/4 (U1 + dt L(U1)); U3 = 1/3 U + 2/3 (U2 + dt L(U2))
 * transposed, with L^T from t7_euler_rhs_adjoint at each stage.  Async. */
t7_status t7_rk3_step_adjoint(t7_ctx *ctx, const void *U, double dt, void *lambda);

/* Recorded steps, for reverse sweeps that replay a segment forward first
 * (checkpointing; no counterpart in the paper: the step is Sec. 2.1's).  A tape entry holds one step's stage states U1 and U2, the
 * forward Delta codes of its three stage states and their three alphas.
 * t7_tape_bytes: size of one entry for this context (a multiple of 256).
 * t7_rk3_step_record: one SSP-RK3 step of fixed dt from U_in to U_out (device
 *   [3][nx]; U_out may not alias U_in, which the adjoint needs later),
 *   writing the entry `tape` (device, 256-byte aligned, caller-owned).  Async.
 * t7_rk3_step_adjoint_recorded: the adjoint of that step -- the same map as
 *   t7_rk3_step_adjoint -- from U_in and its entry, without recomputing the
 *   stages: lambda (the adjoint of U_out) becomes the adjoint of U_in in
 *   place.  Async.  Both take a 1D Euler TENO7-ext FP64 or FP32 context. */
t7_status t7_tape_bytes(t7_ctx *ctx, size_t *bytes);
t7_status t7_rk3_step_record(t7_ctx *ctx, const void *U_in, void *U_out, double dt, void *tape);
t7_status t7_rk3_step_adjoint_recorded(t7_ctx *ctx, const void *U_in, const void *tape, double dt, void *lambda);

/* Ragged batch of independent 1D Euler problems (shock tubes) of uneven
 * length, each advanced by its own SSP-RK3 loop with its own CFL step
 * dt = CFL dx_t / alpha_t(U^n) to t_end (or max_steps), all in ONE persistent
 * launch: groups of `group_warps` warps take tubes from a device work queue,
 * costliest first (cells x estimated steps), so no host round trip happens
 * per step.  The
 * scheme inside each tube is exactly t7_run's (Eq. app, the TENO7-ext
 * reconstruction, Remark 3, SSP-RK3).
 *   ctx          created with sys = T7_EULER1D, nx = total cells, bc[0..1]
 *                applied at both ends of every tube
 *   U            device, [3][nx] (variable-major over the concatenation),
 *                advanced in place
 *   offsets      host, ntubes + 1 ascending, offsets[0] = 0, offsets[ntubes] = nx
 *   dx           host, per-tube cell width (epsilon = dx^3 per tube)
 *   group_warps  1, 2, 4 or 8: that many warps per tube, for every tube;
 *                -1, -2, -4 or -8: the same group size, but the costliest
 *                tubes -- those whose estimated cost (cells x estimated
 *                steps, the steps from the tube's initial wave speed) is above half
 *                of one group's share of the whole batch -- run first on
 *                whole 8-warp CTAs, so that no single tube sets the run time
 *                (with -8 there is nothing to split off);
 *                0: as -G with G chosen by t7_batch_autotune (8 if never
 *                tuned).  Any other value: T7_EINVAL.
 *                The results do not depend on this argument: every tube's
 *                arithmetic is the same for every group size.
 *   steps_out, t_out  host or NULL, per tube
 * Synchronises.  Returns non-physical / non-finite states met in any tube. */
t7_status t7_batch_run(t7_ctx *ctx, void *U, const int64_t *offsets, const double *dx, int ntubes, double t_end,
                       double cfl, int max_steps, int group_warps, int *steps_out, double *t_out);

/* Autotuner of the batch tile shape (no counterpart in the paper; the
 * scheme is t7_batch_run's): times trial_steps steps of every tube
 * for group_warps = 1, 2, 4, 8 on a device copy of U (U is not modified),
 * keeps the fastest in the context for later t7_batch_run calls, and returns
 * it in *group_out (nullable); ms_out (nullable, 4 floats) receives the trial
 * times.  Synchronises.  Trials of 10 or more steps are needed for the
 * ranking to hold over a whole run: smaller groups run more tubes at once,
 * whose joint working set (3 state copies per tube) can outgrow L2, and
 * that cost only shows once each tube has taken several steps -- over 2 or
 * 3 steps every group size streams its tubes in from DRAM alike. */
t7_status t7_batch_autotune(t7_ctx *ctx, const void *U, const int64_t *offsets, const double *dx, int ntubes,
                            double cfl, int trial_steps, int *group_out, float *ms_out);

/* Slabs of a decomposed 1D domain, or of a 2D domain cut along y (one per
 * rank, or per stream).  The scheme
 * is the conservative form Eq. app, whose stencils reach 4 cells per side
 * (the RHS at cell i depends on cells i-4 .. i+4: faces i-1/2 and i+1/2, their
 * 7-point polynomials and their neighbour faces' cutoff bits, Eq. vec), with
 * one global Lax-Friedrichs alpha over the whole domain (Sec. "One
 * dimensional Euler equations").  So a slab of nx cells takes every array
 * PADDED: [m][nx + 8], row stride nx + 8, cell 0 at offset 4; the 4 cells
 * before and after are halos the caller fills (from the neighbouring slabs,
 * or from the domain's boundary condition at its real ends) before a call
 * reads them.  alpha values are device doubles, so that a collective
 * (all-reduce max over the slabs) can feed them without a host round trip.
 * 2D Euler (sys = T7_EULER2D): the slab is ny rows of the domain's nx
 * columns and every array is [4][ny + 8][nx], row 0 at row offset 4; the 4
 * rows before and after are the halos (the y stencils reach 4 rows per side
 * by the same argument, dimension by dimension).  The x direction is whole,
 * so the context's bc[0..1] apply in x; bc[2..3] are not used.  alpha is two
 * device doubles (alpha_x = max(|u| + c), alpha_y = max(|v| + c)), and so is
 * alpha_out; dUdt is [4][ny][nx] and the masks as t7_euler_rhs's for the
 * slab's grid.
 * The context is created for the slab (nx = its cell count; 2D: nx columns,
 * ny = its row count); in 1D its bc[] is not used by these calls.  Async.
 * t7_slab_alpha: max_i (|u_i| + c_i) over the slab's own cells into the
 *   device double *alpha_out (reads only the interior of U).
 * t7_slab_rhs: L(U) = -(F_{i+1/2} - F_{i-1/2})/dx (Eq. app) of the slab's
 *   cells with the given global alpha (device double) into dUdt ([m][nx],
 *   unpadded); masks as t7_euler_rhs's (device or NULL).
 * t7_slab_stage: stage k (0, 1, 2) of the SSP-RK3 step (Sec. 2.1) of fixed
 *   dt, Shu-Osher form as t7_rk3_step:
 *     k = 0: out = Us + dt L(Us);  k = 1: out = 3/4 U0 + 1/4 (Us + dt L(Us));
 *     k = 2: out = 1/3 U0 + 2/3 (Us + dt L(Us)),
 *   with L from the global alpha of Us (device double *alpha).  Us, U0, out
 *   padded; only out's interior is written, and out may not alias Us (U0
 *   may alias out: the usual k = 2 call updates U^n in place).  alpha_out
 *   (device double or NULL) receives max(|u| + c) over the output's cells,
 *   the slab's part of the next stage's alpha.
 * Non-physical or non-finite states are latched as for t7_rk3_step. */
t7_status t7_slab_alpha(t7_ctx *ctx, const void *U, double *alpha_out);
t7_status t7_slab_rhs(t7_ctx *ctx, const void *U, const double *alpha, void *dUdt, uint8_t *masks);
t7_status t7_slab_stage(t7_ctx *ctx, int k, const void *Us, const void *U0, void *out, const double *alpha, double dt,
                        double *alpha_out);

/* The paper has no counterpart to this call (its step is t7_rk3_step's, Sec.
 * 2.1): it serves callers that cannot
 * allocate device memory -- plug-ins whose host application owns every device
 * allocation, real-time loops that forbid allocation after start-up, and
 * processes whose device memory is budgeted by an external allocator.
 *
 * One SSP-RK3 step of size dt of a 1D system (grid->sys advection, Burgers or
 * 1D Euler), in place on the caller's device array U ([m][nx], grid->prec),
 * on `stream` (a cudaStream_t; NULL = legacy default stream).  It creates no
 * context and allocates nothing: the two stage buffers and the control block
 * live in one file-scope device array of T7_STATIC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Sizes whose scratch does not fit (2 x m x nx x element size plus
 * 256 bytes, each buffer rounded up to 256 bytes) are rejected with T7_EINVAL
 * before any GPU work.  The first call on each device looks up that device's
 * address of the array (with the device current; concurrent first calls from
 * several host threads are safe).  Every call reuses the array and clears the
 * part that must start at zero; calls that overlap on the GPU (on different
 * streams, or from several host threads) race on it.  Results equal
 * t7_rk3_step's.  Every call copies its status word to the host and
 * synchronises the stream, so it must never be made on a stream that is being
 * captured into a CUDA graph (the capture would fail).  Returns any
 * non-physical or non-finite state met.  errbuf (nullable) receives a
 * message. */
#define T7_STATIC_SCRATCH_BYTES (16u << 20)
t7_status t7_rk3_step_static(const t7_grid *grid, void *U, double dt, void *stream, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* TENO7_H */
