/*
 * rhd.h -- C ABI of the GB300 library for one grey, M1-closure IMEX PD-ARS
 * radiation step (He, Wibking & Krumholz 2024, "An asymptotically-correct
 * implicit-explicit time integration scheme for finite volume
 * radiation-hydrodynamics").
 *
 * What one step computes (Sec. 3.2, eq. imex1 / imex2 with epsilon = 0):
 *   y(n+1/2) = y(n) + dt s(y(n)) + dt f(y(n+1/2))
 *   y(n+1)   = y(n) + dt [s(y(n)) + s(y(n+1/2))]/2
 *                   + dt [f(y(n+1/2)) + f(y(n+1))]/2
 * on a uniform Cartesian grid, with y = (rho v, Egas, E, F/(c chat)) and the
 * reduced-speed-of-light split of eq. (yrsla):
 *   s(y) = -div(0, 0, (chat/c) F, P)         explicit transport (Sec. 3.3:
 *          piecewise-linear faces, HLL fluxes, Sec. 4.3 wave speeds and the
 *          optional optical-depth factor on the energy flux),
 *   f(y) = (G, c G0, -chat G0, -G)           local implicit exchange (Sec. 3.3:
 *          eq. egupdate-fupdate, inner Newton on (Egas, R) of eq. FGFR/Rnew,
 *          energy closure, eq. numF1/numF2, momentum update, outer iteration).
 * Grey material: chi_P = chi_E = chi_F = chi = kappa rho.
 *
 * Units are the caller's: a_rad is the radiation constant (4 pi B / c =
 * a_rad T^4) and T = (Egas - |m|^2 / (2 rho)) / (rho kB_over_mu / (gamma - 1)).
 *
 * Conventions for every call:
 *  - Errors: every call returns an rhd_status; nothing is thrown across the
 *    ABI.  rhd_last_error() describes the most recent failure of a context.
 *  - Ownership: the library owns all device memory of a context (allocated in
 *    rhd_init, released in rhd_destroy).  Caller buffers passed to get/set are
 *    only read/written during the call (host buffers) or by work enqueued on
 *    the context's stream before the call returns (device buffers); the caller
 *    keeps ownership.
 *  - Layout of every field array: ncell = n[0]*n[1]*n[2] doubles, cell
 *    (i, j, k) at index i + n[0]*(j + n[1]*k) (x fastest).
 *  - Threads: a context must not be used by two host threads at once.
 */
#ifndef RHD_H
#define RHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rhd_ctx rhd_ctx; /* opaque; library-owned device state */

typedef enum {
  RHD_OK = 0,
  RHD_ERR_ARG = 1,          /* invalid argument or rejected input values */
  RHD_ERR_CUDA = 2,         /* a CUDA runtime call failed (see rhd_last_error) */
  RHD_ERR_NEWTON = 3,       /* inner Newton iteration did not converge (Sec. 3.3) */
  RHD_ERR_OUTER = 4,        /* outer iteration did not converge (Sec. 3.3) */
  RHD_ERR_NONPHYSICAL = 5,  /* T <= 0, E <= 0 or a non-finite value */
  RHD_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
  RHD_ERR_STATE = 7,        /* call out of order (e.g. step before all fields set) */
  RHD_ERR_BOUNDS = 8        /* a library built with -DRHD_BOUNDS_CHECK caught an index
                               outside its array in a stage kernel (fail_cell holds
                               the index); never returned by the default build */
} rhd_status;

/* Boundaries of the radiation transport.  PERIODIC: wrap; REFLECT: mirror
 * the cells, negating the normal flux; INFLOW: ghost cells hold the fixed
 * radiation state bc_state of that face (e.g. an isotropic source of
 * temperature T_s: E = a_rad T_s^4, F = 0).  HALO: the face is shared with
 * the neighbouring z-slab of a decomposed grid (3-D, z faces only, n[2] >= 3);
 * its ghost planes are the neighbour's boundary planes, copied in by
 * rhd_step_slabs before each stage. */
typedef enum {
  RHD_BC_PERIODIC = 0, RHD_BC_REFLECT = 1, RHD_BC_INFLOW = 2, RHD_BC_HALO = 3
} rhd_bc;
/* Time integration.  IMEX_PDARS: the paper's scheme (eq. imex1/imex2), the
 * local exchange solved in both stages.  RK2_SSP: the comparison scheme of
 * Sec. 4.2, transport alone in the first stage and the exchange solved once,
 * with the full step, after the second -- kept as a negative control for the
 * asymptotic diffusion limit, which it does not preserve. */
typedef enum { RHD_SCHEME_IMEX_PDARS = 0, RHD_SCHEME_RK2_SSP = 1 } rhd_scheme;
typedef enum { RHD_CLOSURE_M1 = 0, RHD_CLOSURE_EDDINGTON = 1 } rhd_closure;
/* Face states of E and F (Sec. 3.3).  PLM: linear with the monotonised-
 * central limiter (the default).  PPM: the paper's choice, the piecewise
 * parabolic edge values of Colella & Woodward (1984) -- fourth-order
 * interface values from limited slopes, then their monotonicity constraint
 * per cell -- without contact steepening or flattening.  PPM reads three
 * cells on each side of a face, so a reflecting or inflow axis needs n >= 3;
 * a forward-Euler transport stage keeps E > 0 for CFL <= 1/3 with PPM (1/2
 * with PLM).  rhd_adjoint takes PLM only; a batch holding a PPM problem runs
 * the default 2-D tile shape (rhd_batch_configure's tile2d is then ignored). */
/* PPM_CS: PPM with the limiter of Colella & Sekora (2008), which keeps
 * smooth extrema (fourth order there, where PPM's constraint flattens the
 * cell): interface values limited through second differences, and at an
 * extremum the parabola's curvature limited against C = 1.25 times the
 * neighbouring second differences.  It does not keep an edge within its
 * neighbours' range, so on rough data a face state can turn nonphysical
 * where PPM's would not.  Same stencil, n >= 3 rule and restrictions as PPM. */
typedef enum { RHD_RECON_PLM = 0, RHD_RECON_PPM = 1, RHD_RECON_PPM_CS = 2 } rhd_recon;
/* HLL energy-flux dissipation (Sec. 4.3): TAU scales it by
 * (1 - exp(-tau))/tau, tau = chi dx of the face; NONE is the paper's own
 * uncorrected IMEX choice. */
typedef enum { RHD_HLL_TAU = 0, RHD_HLL_NONE = 1 } rhd_hll_mode;
/* FP64: everything in double.  MIXED: reconstruction, closure and HLL fluxes
 * in single precision from double-precision differences; state, Newton solve,
 * exchange terms and all updates in double. */
typedef enum { RHD_PREC_FP64 = 0, RHD_PREC_MIXED = 1 } rhd_precision;

/* Fields of the state.  F is the physical lab-frame radiation flux; KAPPA is
 * the specific absorption opacity (chi = kappa rho).  RHO and KAPPA are
 * static; the other eight are evolved. */
typedef enum {
  RHD_F_RHO = 0, RHD_F_MX, RHD_F_MY, RHD_F_MZ, RHD_F_EGAS, RHD_F_ERAD,
  RHD_F_FX, RHD_F_FY, RHD_F_FZ, RHD_F_KAPPA, RHD_NFIELDS
} rhd_field;

typedef struct {
  int ndim;            /* 1, 2 or 3 */
  int64_t n[3];        /* cells per axis; axes >= ndim must be 1 */
  double dx[3];        /* cell widths (> 0 on the active axes) */
  int bc[3][2];        /* rhd_bc of the low/high face of each axis; a
                          reflecting axis needs n >= 2, a HALO face
                          (z only) n[2] >= 3 */
  double gamma;        /* adiabatic index (> 1) */
  double c;            /* speed of light (> 0) */
  double chat;         /* reduced speed of light, 0 < chat <= c (Sec. 3.2) */
  double a_rad;        /* radiation constant (> 0) */
  double kB_over_mu;   /* k_B/mu: c_v = kB_over_mu/(gamma-1) per unit mass */
  double cfl;          /* CFL number of the default step (> 0) */
  int closure;         /* rhd_closure */
  int vc_order;        /* 1: eq. numF1; 2: eq. numF2 and the (1+beta^2/2) terms */
  int hll_mode;        /* rhd_hll_mode */
  int precision;       /* rhd_precision */
  double newton_rtol;  /* inner convergence tolerance (Sec. 3.3: 1e-13) */
  double outer_rtol;   /* outer convergence tolerance (Sec. 3.3: 1e-13) */
  int newton_max_iter; /* bound on Newton updates per inner solve */
  int outer_max_iter;  /* bound on outer passes per local solve */
  /* -- added after the fields above; rhd_params_default sets them -- */
  int scheme;          /* rhd_scheme (default IMEX_PDARS) */
  /* temperature-dependent opacity chi = kappa rho (T/kappa_T_ref)^kappa_T_exp
   * in the local solve, evaluated at the current Newton iterate and held
   * fixed in the Jacobian (Sec. 3.3); the default 0 keeps chi = kappa rho.
   * A non-zero exponent needs hll_mode NONE (the optical-depth factor is
   * computed from the static kappa and rho). */
  double kappa_T_exp;
  double kappa_T_ref;  /* reference temperature (> 0, default 1) */
  double bc_state[3][2][4]; /* INFLOW faces: ghost E, Fx, Fy, Fz (E > 0) */
  /* non-grey material (eq. G0/G1): chi_0E = kappa rho (times the T factor
   * above), chi_0P = kappa_P_ratio chi_0E, chi_0F = kappa_F_ratio chi_0E;
   * both 1 (the default) is grey.  The TAU factor then uses chi_0F. */
  double kappa_P_ratio;
  double kappa_F_ratio;
  int reconstruction; /* rhd_recon */
  /* CFL number of the hydrodynamic step (rhd_hydro_step, rhd_step_split) */
  double cfl_hydro;
} rhd_params;

typedef struct {
  int status;          /* rhd_status of this call */
  int steps_done;      /* steps completed by this call */
  int64_t fail_cell;   /* smallest failing cell index, -1 if none */
  int fail_step;       /* step (within the call) that failed, -1 if none */
  int fail_stage;      /* 1 or 2, 0 if none */
  int max_newton;      /* most Newton updates of any local solve */
  int max_outer;       /* most outer passes of any local solve */
  int64_t sum_newton;  /* total Newton updates */
  int64_t n_solves;    /* local solves performed */
  double t;            /* simulated time of the context after the call */
  double dt;           /* step size used */
  int64_t sum_outer;   /* total outer passes */
} rhd_step_info;

/* Fill p with the library defaults: periodic, gamma 5/3, c = chat = 1,
 * a_rad = kB_over_mu = 1, CFL 0.4, M1, v/c order 2, HLL TAU, FP64,
 * tolerances 1e-13, 64 Newton updates, 32 outer passes, IMEX PD-ARS,
 * temperature-independent grey opacity (kappa_T_exp 0, kappa_T_ref 1,
 * kappa_P_ratio = kappa_F_ratio = 1), inflow states E = 1, F = 0, PLM faces,
 * hydrodynamic CFL 0.3.  The grid
 * fields are zeroed; the caller sets ndim, n and dx. */
void rhd_params_default(rhd_params* p);

/* Check p without touching the GPU.  Returns RHD_OK or RHD_ERR_ARG; on error
 * writes a message into msg (msglen bytes, may be NULL/0). */
rhd_status rhd_params_validate(const rhd_params* p, char* msg, int msglen);

/* Default step of Sec. 4.3's wave-speed bound: cfl / (chat * sum_d 1/dx_d),
 * or a negative value if p is invalid. */
double rhd_default_dt(const rhd_params* p);

/* Create a context on the current CUDA device: validates p, allocates the
 * device state (two ping-pong copies of the evolved fields, the stage buffer,
 * rho, kappa) and a private non-blocking stream.  *out is NULL on error. */
rhd_status rhd_init(const rhd_params* p, rhd_ctx** out);

/* Use an external CUDA stream (cudaStream_t passed as void*, e.g. torch's
 * current stream) for all later work of ctx.  The handle is taken literally:
 * NULL is CUDA's legacy default stream.  The caller keeps ownership of the
 * stream and must keep it alive; rhd_use_private_stream switches back. */
rhd_status rhd_set_stream(rhd_ctx* ctx, void* cuda_stream);

/* Switch ctx back to the private stream created by rhd_init. */
rhd_status rhd_use_private_stream(rhd_ctx* ctx);

/* Copy one field in (count must equal ncell).  src is a host pointer
 * (src_on_device = 0; pinned memory makes the copy asynchronous-capable) or a
 * device pointer on the context's device (src_on_device = 1).  Values are
 * validated on the device: rho > 0, Erad > 0 and kappa >= 0, all finite.  A
 * rejected field returns RHD_ERR_ARG and stays marked unset, so rhd_step
 * returns RHD_ERR_STATE until it is set again.  Synchronises the stream. */
rhd_status rhd_state_set(rhd_ctx* ctx, int field, const double* src,
                         int64_t count, int src_on_device);

/* All ten fields at once from one field-major array of RHD_NFIELDS*ncell
 * doubles (field f at src + f*ncell); same rules as rhd_state_set. */
rhd_status rhd_state_set_all(rhd_ctx* ctx, const double* src, int64_t count,
                             int src_on_device);

/* Copy one field out of the current state (count must equal ncell) to a host
 * or device buffer.  Synchronises the stream before returning. */
rhd_status rhd_state_get(rhd_ctx* ctx, int field, double* dst, int64_t count,
                         int dst_on_device);

/* One evolved field of the stage state y(n+1/2) of the last step the context
 * took (eq. imex1), e.g. for checkpointing the two stages; valid until the
 * next rhd_step/rhd_step_async.  RHO and KAPPA are rejected (RHD_ERR_ARG).
 * Synchronises the stream. */
rhd_status rhd_stage_get(rhd_ctx* ctx, int field, double* dst, int64_t count,
                         int dst_on_device);

/* All ten fields to one field-major array of RHD_NFIELDS*ncell doubles. */
rhd_status rhd_state_get_all(rhd_ctx* ctx, double* dst, int64_t count,
                             int dst_on_device);

/* Advance nsteps IMEX PD-ARS steps of size dt (dt <= 0: rhd_default_dt).
 * Enqueues 2 stage kernels per step, then waits once and reads the device
 * status.  On a failed step the context stays at the last completed step
 * (ping-pong buffers) and info (nullable) names the step, stage and smallest
 * failing cell. */
rhd_status rhd_step(rhd_ctx* ctx, int nsteps, double dt, rhd_step_info* info);

/* Enqueue nsteps without waiting (same semantics as rhd_step once the
 * matching rhd_sync returns).  At most one rhd_step_async batch may be
 * pending; kernels of later steps skip their work once a step has failed. */
rhd_status rhd_step_async(rhd_ctx* ctx, int nsteps, double dt);

/* Wait for the pending rhd_step_async batch and report it like rhd_step. */
rhd_status rhd_sync(rhd_ctx* ctx, rhd_step_info* info);

/* Step a state held in host memory: copy src in, advance nsteps >= 1 IMEX
 * PD-ARS steps of size dt (eq. imex1, imex2; dt <= 0: rhd_default_dt), and
 * copy the result to dst.  src and dst are host arrays of RHD_NFIELDS*ncell
 * doubles, field-major as in rhd_state_set_all, owned by the caller; dst
 * receives all ten fields (rho and kappa unchanged, and not copied back when
 * dst is src) and may be src itself, but must not otherwise overlap it.  The
 * copies run in up to 16 chunks of tile rows along the slowest grid axis (z
 * in 3-D) on the context's own two copy streams (even and odd fields) and
 * overlap the stage kernels, which run on its own compute streams of falling
 * priority, one per launch group: the
 * first step's stage 1 starts on the first chunks as soon as they and their
 * neighbours are in, and the last step's stage 2 ends on small groups of
 * chunks, each copied out as it finishes; the steps between run on the whole
 * grid.  With pinned (page-locked) buffers the
 * copies overlap the compute; pageable buffers give the same results without
 * the overlap.  Ordered after earlier work on the context's stream, which
 * waits for all of it; synchronises before returning; not for stream
 * capture.  The result equals rhd_state_set_all + rhd_step + rhd_state_get_all
 * bit for bit.  The input is validated as by rhd_state_set_all, after the
 * fact: a non-finite or out-of-range value returns RHD_ERR_ARG, leaves dst
 * unspecified and the context without a state (set it again).  On a failed
 * step info (nullable) reports it as rhd_step does, the context holds the
 * last completed step, and the evolved fields of dst are unspecified.  Any
 * other error (RHD_ERR_CUDA, RHD_ERR_STATE) also leaves the context without a
 * state.  Refused while a batch is pending, during a slab step and on a
 * context with a HALO face; a dst that overlaps src without being src
 * returns RHD_ERR_ARG. */
rhd_status rhd_step_host(rhd_ctx* ctx, const double* src, double* dst, int64_t count,
                         int nsteps, double dt, rhd_step_info* info);

/* Diagnostic, host only (no device work): the plan rhd_step_host follows
 * for the grid of p.  On return *nchunks = K, the chunks of tile rows along
 * the slowest axis: chunk k holds the tile rows rows[k] .. rows[k+1] - 1
 * and the cells cells[k] .. cells[k+1] - 1 (cell order of the state).
 * groups receives pairs (first chunk, end chunk): ngroups[0] stage-1 launch
 * groups, then ngroups[1] groups of the last step's stage 2, each copied
 * out as it finishes.  cells and rows hold cap >= K + 1 entries, groups
 * cap >= ngroups[0] + ngroups[1] pairs; a smaller cap, a NULL pointer or
 * invalid params return RHD_ERR_ARG (message: rhd_last_error(NULL)). */
rhd_status rhd_host_step_plan(const rhd_params* p, int* nchunks, int64_t* cells, int* rows,
                              int* groups, int ngroups[2], int cap);

/* Transport operator of the current state, s(y) of eq. (yrsla): the rates
 * dE/dt and dF/dt (physical flux) of the explicit stage (Sec. 3.3 face states
 * and HLL fluxes), without the local source terms.  rates: 4*ncell doubles,
 * field-major (E, Fx, Fy, Fz), on the host (dst_on_device = 0) or the device.
 * Returns RHD_ERR_NONPHYSICAL if a face state has E <= 0.  Uses the idle
 * ping-pong buffer as scratch for host destinations; synchronises. */
rhd_status rhd_transport(rhd_ctx* ctx, double* rates, int64_t count, int dst_on_device);

/* Conserved totals of the current state (Sec. 3.3): out[0] = sum over cells
 * of (Egas + (c/chat) E) V, out[1..3] = sum of (m + F/(c chat)) V, V the cell
 * volume.  Deterministic (fixed reduction order).  Synchronises. */
rhd_status rhd_totals(rhd_ctx* ctx, double out[4]);

/* Kernel timing with CUDA events on the context stream.  enable = 1 starts
 * recording (clears previous records), 0 stops.  rhd_profile_read returns, per
 * kernel kind k (0: stage 1, 1: stage 2, 2: totals), the number of launches
 * and the summed device time in milliseconds; synchronises. */
rhd_status rhd_profile(rhd_ctx* ctx, int enable);
rhd_status rhd_profile_read(rhd_ctx* ctx, int64_t launches[3], double ms[3]);

/* ---- Differentiation: reverse mode through whole steps ----
 * The paper has no adjoint; this derivative of the step it defines serves
 * gradient-based inversion (e.g. of initial temperatures or opacities).
 * A recorded state is 8 slots of ncell doubles (Egas, mx, my, mz, E, Fx, Fy,
 * Fz: the evolved fields in rhd_field order), one slot after another. */

/* Advance nsteps like rhd_step (dt <= 0: rhd_default_dt) and record the tape
 * the adjoint needs.  tape: device buffer owned by the caller, count =
 * (2*nsteps + 1) * 8 * ncell doubles, written as y(0), y(1/2), y(1), y(3/2),
 * ..., y(nsteps): every step's start state and its stage-1 state y(n+1/2) of
 * eq. (imex1).  The stage kernels write the tape directly; the context's
 * state becomes y(nsteps) on success and stays at y(0) on failure (info as
 * rhd_step's, nullable).  Synchronises. */
rhd_status rhd_step_record(rhd_ctx* ctx, int nsteps, double dt, double* tape,
                           int64_t count, rhd_step_info* info);

/* Reverse-mode derivative of nsteps recorded steps.  tape, count, nsteps and
 * dt as given to rhd_step_record (the same dt; <= 0: rhd_default_dt); the
 * context's rho and kappa must be those the steps ran with.  ybar: device
 * buffer of 8*ncell doubles (slots as in the tape) holding dL/dy(nsteps) on
 * entry and dL/dy(0) on return.  kappa_bar: device buffer of ncell doubles
 * to which dL/dkappa is added.  Both caller-owned.  The transport part is
 * the transpose of the PLM/HLL fluxes (Sec. 3.3, Sec. 4.3) on the active
 * branch of every limiter, maximum and clip; the implicit part applies the
 * implicit-function theorem to the converged local solve of eq.
 * (egupdate)-(fupdate).  The first call allocates 8*ncell + 18*(faces)
 * doubles of scratch that the context keeps.  Returns RHD_ERR_ARG for a
 * context with RK2-SSP, a temperature-dependent or non-grey opacity, an
 * inflow face or PPM faces, and RHD_ERR_NEWTON if the Jacobian of a
 * converged solve is singular.  Synchronises. */
rhd_status rhd_adjoint(rhd_ctx* ctx, const double* tape, int64_t count, int nsteps,
                       double dt, double* ybar, double* kappa_bar);

/* ---- Radiation hydrodynamics: the hydrodynamic subsystem and the
 * operator split of Sec. 3.1 ----
 * The gas state is rho (RHD_F_RHO, which these calls evolve), m and E_gas
 * (the total gas energy); ideal gas p = (gamma - 1)(E_gas - |m|^2/(2 rho)).
 * The paper leaves the hydrodynamic method to its host code; this library
 * advances the Euler equations by a method of lines with RK2-SSP (Shu &
 * Osher 1988), the primitives (rho, v, p) reconstructed with the context's
 * `reconstruction` and HLLC fluxes (Toro, Spruce & Speares 1994) with the
 * wave-speed bounds min/max(u -+ a) of both sides; ghost cells as for the
 * radiation (a reflecting wall negates the normal velocity).  FP64 in both
 * precisions.  Axes with an inflow face are refused (RHD_ERR_ARG).  The
 * first call allocates 10 * ncell + 5 * (faces of every axis) doubles of
 * scratch that the context keeps.  Failures (rho <= 0 or p <= 0 in a stage)
 * return RHD_ERR_NONPHYSICAL with the first failing step; that step is not
 * applied, earlier ones are.  info (nullable): steps_done, fail_cell,
 * fail_step, fail_stage (3 and 4: the hydrodynamic stages 1 and 2), dt (the
 * last step size) and t.  These calls synchronise. */

/* dt of the hydrodynamic step for the current state: cfl_hydro / max over
 * cells of sum_d (|v_d| + a)/dx_d, a = sqrt(gamma p / rho). */
rhd_status rhd_hydro_dt(rhd_ctx* ctx, double* dt);

/* nsteps RK2-SSP steps of the hydrodynamic subsystem alone, each of dt
 * (dt <= 0: rhd_hydro_dt of the state before each step); the radiation
 * fields are untouched.  Advances rhd_time. */
rhd_status rhd_hydro_step(rhd_ctx* ctx, int nsteps, double dt, rhd_step_info* info);

/* nsteps operator-split steps of the full system (Sec. 3.1): the
 * hydrodynamic step of dt_h (dt_h <= 0: rhd_hydro_dt of the state), then
 * the radiation update subcycled: nsub = ceil(dt_h / rhd_default_dt - 1e-12)
 * rhd_step steps of dt_h / nsub.  info: steps_done counts split steps; the
 * iteration statistics sum over the radiation steps; fail_stage 1-2 is a
 * radiation stage, 3-4 a hydrodynamic one. */
rhd_status rhd_step_split(rhd_ctx* ctx, int nsteps, double dt_h, rhd_step_info* info);

/* ---- Domain decomposition: z-slabs of one grid on one device ----
 * The radiation step needs no communication beyond ghost layers (Sec. 3.2:
 * the explicit stages read face neighbours, the implicit solve is local):
 * before each stage every slab receives the (E, F) planes of its neighbours
 * that its face states read (2 with PLM, 3 with PPM), and nothing else.
 * slabs[0..nslab-1] are contexts of consecutive z ranges of one 3-D grid,
 * bottom to top (slab s + 1 sits on slab s).  The contexts must be created
 * with identical params except n[2] (>= 3) and the z faces: every face
 * between two slabs is RHD_BC_HALO on both sides; the bottom face of slab 0
 * and the top face of the last slab are either both HALO (a periodic grid:
 * they face each other) or neither (their own reflecting or inflow faces).
 * All slabs share one stream and one device, and every field of every slab
 * must be set.  Advances nsteps steps of dt (dt <= 0: rhd_default_dt) with
 * the same arithmetic per cell as the undecomposed grid: the results are
 * bit-identical to it.  Each exchange is one cudaMemcpyAsync per field and
 * face, device to device (the calls a multi-GPU run would replace by
 * point-to-point sends); TAU-mode face factors at the slab faces are
 * computed from the neighbour's rho and kappa at the start of every call
 * (one TAU-factor kernel per slab).  Failure: all slabs stay at the last
 * step that every slab completed; info (nullable) reports as rhd_step with
 * fail_cell counted in the whole grid (cell index of slab s plus the cells
 * of the slabs below).
 * The first call allocates 27 * n[0] * n[1] doubles per slab.  A context
 * with a HALO face is refused (RHD_ERR_STATE) by every other stepping call
 * (rhd_step, rhd_step_async, rhd_transport, rhd_step_record, rhd_adjoint,
 * rhd_hydro_step, rhd_step_split).  Synchronises. */
rhd_status rhd_step_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                          rhd_step_info* info);

/* The hydrodynamic step (rhd_hydro_step) and the operator split
 * (rhd_step_split) of z-slabs, with the same slab rules and the same
 * results as on the undecomposed grid, bit for bit.  Before each of the two
 * RK2-SSP stages every slab receives the neighbours' boundary planes of the
 * primitives (rho, v, p), 2 with PLM and 3 with PPM; dt <= 0 (dt_h <= 0)
 * takes the CFL step of the whole grid (the largest bound of any slab); the
 * stage-2 result is committed to every slab only if no cell of any slab
 * failed.  Inflow faces are refused (RHD_ERR_ARG) as for one grid.  The
 * first call allocates the hydrodynamic scratch of rhd_hydro_step per slab
 * and 30 * n[0] * n[1] doubles of halo.  Synchronise. */
rhd_status rhd_hydro_step_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                                rhd_step_info* info);
rhd_status rhd_step_split_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt_h,
                                rhd_step_info* info);

/* ---- Domain decomposition across processes: one z-slab per process ----
 * The stage-by-stage form of rhd_step_slabs for slabs that live in different
 * processes or on different GPUs (Sec. 3.2: a stage of the scheme needs the
 * face neighbours' ghost planes and nothing else).  Each process holds one
 * slab context (params as rhd_step_slabs wants them: HALO faces between
 * slabs, the same grid otherwise) and the caller carries the planes between
 * neighbours, by NCCL send/receive or any other route.  One step:
 *   rhd_slab_planes_get(BOUNDARY_LOW and _HIGH, stage 1) -> send to the
 *     slabs below and above; rhd_slab_planes_set(GHOSTS_HIGH and _LOW) with
 *     what they sent; rhd_slab_stage(1, dt);
 *   the same with stage 2 planes; rhd_slab_stage(2, dt);
 *   rhd_slab_status; combine the statuses of all slabs; rhd_slab_commit(1)
 *     only if every slab succeeded (else 0: every slab keeps y(n)).
 * With HLL mode TAU, whenever rho or kappa of any slab changes: send
 * MATERIAL_LOW down and set it as MATERIAL_ABOVE, then send EPS_HIGH up and
 * set it as EPS_BELOW.  The slabs then evolve bit for bit like the whole grid
 * and like rhd_step_slabs.  Failed cells are numbered within the slab. */
enum {
  RHD_SLAB_BOUNDARY_LOW = 0,   /* get: E, Fx, Fy, Fz of the lowest `depth` planes of the
                                  stage's input state (stage 1 y(n), stage 2 y(n+1/2)) */
  RHD_SLAB_BOUNDARY_HIGH = 1,  /* get: the same of the highest `depth` planes */
  RHD_SLAB_GHOSTS_LOW = 2,     /* set: the ghost planes below (the BOUNDARY_HIGH of the
                                  slab below) */
  RHD_SLAB_GHOSTS_HIGH = 3,    /* set: the ghost planes above (the BOUNDARY_LOW of the
                                  slab above) */
  RHD_SLAB_MATERIAL_LOW = 4,   /* get: kappa, then rho, of plane 0 */
  RHD_SLAB_MATERIAL_ABOVE = 5, /* set: the MATERIAL_LOW of the slab above */
  RHD_SLAB_EPS_HIGH = 6,       /* get: TAU factors of the top face (needs MATERIAL_ABOVE) */
  RHD_SLAB_EPS_BELOW = 7,      /* set: the EPS_HIGH of the slab below */
  RHD_SLAB_PRIM_BOUNDARY_LOW = 8,   /* get: rho, vx, vy, vz, p of the lowest `depth` planes
                                       of the hydrodynamic stage (after phase 0 or 2) */
  RHD_SLAB_PRIM_BOUNDARY_HIGH = 9,  /* get: the same of the highest `depth` planes */
  RHD_SLAB_PRIM_GHOSTS_LOW = 10,    /* set: the primitive ghost planes below */
  RHD_SLAB_PRIM_GHOSTS_HIGH = 11    /* set: the primitive ghost planes above */
};

/* Doubles that a plane kind holds for this slab: 4 depth n0 n1 for the
 * boundary and ghost planes (depth 2 with PLM faces, 3 with PPM), laid out
 * [field E, Fx, Fy, Fz][plane, in z order][n0 n1]; 5 depth n0 n1 for the
 * primitive planes ([rho, vx, vy, vz, p][plane][n0 n1]); 2 n0 n1 for the
 * material planes; n0 n1 for the TAU factors.  -1 for a bad kind or a grid
 * that is not 3-D. */
int64_t rhd_slab_plane_doubles(const rhd_ctx* ctx, int what);

/* Copy planes of kind `what` (a get kind) into dst (count doubles, host or
 * device, caller-owned); `stage` (1 or 2) selects the input state of the
 * boundary planes and is ignored otherwise.  Host copies synchronise the
 * stream.  RHD_ERR_ARG for a context without a HALO face, a bad kind or
 * count; RHD_ERR_STATE for stage-2 planes before stage 1. */
rhd_status rhd_slab_planes_get(rhd_ctx* ctx, int what, int stage, double* dst, int64_t count,
                               int dst_on_device);

/* Store planes of kind `what` (a set kind) from src (count doubles, host or
 * device) in the slab's halo buffer; the face they belong to must be HALO. */
rhd_status rhd_slab_planes_set(rhd_ctx* ctx, int what, const double* src, int64_t count,
                               int src_on_device);

/* Run stage 1 (eq. imex1) or stage 2 (eq. imex2) of one step on the slab's
 * stream with the ghost planes set last (does not synchronise).  Stage 1
 * takes dt (<= 0: rhd_default_dt) and starts the step; stage 2 uses the same
 * dt.  RHD_ERR_STATE out of order, or with TAU factors whose neighbour planes
 * are not set for the current rho and kappa. */
rhd_status rhd_slab_stage(rhd_ctx* ctx, int stage, double dt);

/* After stage 2: wait for the slab's stream and return the slab's status
 * (info, nullable, as by rhd_step with fail_cell within the slab).  The step
 * is not applied until rhd_slab_commit. */
rhd_status rhd_slab_status(rhd_ctx* ctx, rhd_step_info* info);

/* After rhd_slab_status: commit != 0 makes y(n+1) the state and advances the
 * time by dt; 0 keeps y(n) (another slab failed).  After a hydrodynamic step
 * commit != 0 copies its staged result into the state (one more launch). */
rhd_status rhd_slab_commit(rhd_ctx* ctx, int commit);

/* The hydrodynamic step of a slab (RK2-SSP with HLLC faces, as
 * rhd_hydro_step_slabs), phase by phase:
 *   rhd_slab_hydro_speed on every slab, the largest smax of all slabs gives
 *     dt = cfl_hydro / smax (the whole grid's CFL step);
 *   rhd_slab_hydro_phase(0, dt): primitives of the state; exchange the
 *     PRIM_BOUNDARY planes into the neighbours' PRIM_GHOSTS;
 *     rhd_slab_hydro_phase(1): face fluxes and stage 1;
 *   rhd_slab_hydro_phase(2): primitives of stage 1; exchange again;
 *     rhd_slab_hydro_phase(3): face fluxes and stage 2, staged;
 *   rhd_slab_status, combine, rhd_slab_commit.
 * Periodic and reflecting x and y axes only (no inflow faces). */

/* *smax: the slab's largest sum_d (|v_d| + a)/dx_d (+inf if a cell has
 * rho <= 0 or p <= 0).  Synchronises the stream. */
rhd_status rhd_slab_hydro_speed(rhd_ctx* ctx, double* smax);

/* Run hydrodynamic phase 0 .. 3 (phase 0 takes dt > 0 and starts the step;
 * later phases use it) on the slab's stream, reading the primitive ghost
 * planes set last.  RHD_ERR_STATE out of order. */
rhd_status rhd_slab_hydro_phase(rhd_ctx* ctx, int phase, double dt);

/* Number of kernels this context has launched since rhd_init. */
int64_t rhd_launch_count(const rhd_ctx* ctx);

/* Simulated time of the context (sum of completed step sizes). */
double rhd_time(const rhd_ctx* ctx);

/* Message of the most recent failure of ctx (never NULL). */
const char* rhd_last_error(const rhd_ctx* ctx);

/* Release all device memory and the private stream.  NULL is ignored. */
void rhd_destroy(rhd_ctx* ctx);

/* ---------------------------------------------------------------------
 * Batched form: many independent 1-D and 2-D grids advanced together.
 *
 * Every problem has its own grid, physics and default time step
 * (rhd_default_dt of its params); all share one precision.  The fields of all
 * problems live in pooled device arrays.  One step is two launches of a
 * persistent kernel (stage 1 and stage 2 of eq. imex1/imex2) whose blocks
 * take (problem, tile) work items from an atomic counter; the launches of an
 * rhd_batch_step call are captured once into a CUDA graph and replayed on
 * later calls with the same step count.
 * ------------------------------------------------------------------- */
typedef struct rhd_batch rhd_batch;

/* Validate and allocate nprob problems (probs[p].ndim must be 1 or 2, one
 * precision for all).  *out is NULL on error (message: rhd_last_error(NULL)). */
rhd_status rhd_batch_init(const rhd_params* probs, int nprob, rhd_batch** out);

/* Run on this CUDA stream (drops the captured graphs).  The legacy default
 * stream (NULL) cannot hold a graph capture: with NULL the batch waits for
 * the legacy stream's earlier work and runs on its private stream. */
rhd_status rhd_batch_set_stream(rhd_batch* b, void* cuda_stream);

/* Launch configuration: tile2d selects the 2-D tile (0: 32 x 8, 1: 64 x 4,
 * 2: 16 x 16 cells), blocks_per_sm the persistent grid (1 or 2 blocks per SM).
 * Results do not depend on it (the autotuner in paper_2404_08247_gb300/autotune.py
 * picks it from timings). */
rhd_status rhd_batch_configure(rhd_batch* b, int tile2d, int blocks_per_sm);

/* enable = 0: rhd_batch_step enqueues its launches directly instead of
 * replaying a captured CUDA graph (results are identical; for tools that do
 * not see the nodes of a graph, such as some profiler configurations).
 * enable != 0 (the default): graphs. */
rhd_status rhd_batch_use_graphs(rhd_batch* b, int enable);

/* Cells of problem prob, or of the whole batch for prob < 0 (-1 on error). */
int64_t rhd_batch_cells(const rhd_batch* b, int prob);

/* State of one problem: RHD_NFIELDS * ncell doubles, field-major as in
 * rhd_state_set_all, host or device; same validation as rhd_state_set. */
rhd_status rhd_batch_state_set(rhd_batch* b, int prob, const double* src, int64_t count,
                               int src_on_device);
rhd_status rhd_batch_state_get(rhd_batch* b, int prob, double* dst, int64_t count,
                               int dst_on_device);

/* Advance every problem nsteps steps of its own dt.  On failure every problem
 * stays at the last completed step and info->fail_cell is a pooled cell index
 * (see rhd_batch_locate); info->t counts steps.  Synchronises. */
rhd_status rhd_batch_step(rhd_batch* b, int nsteps, rhd_step_info* info);

/* Map a pooled cell index to (problem, cell). */
rhd_status rhd_batch_locate(const rhd_batch* b, int64_t pooled_cell, int* prob,
                            int64_t* cell);

const char* rhd_batch_last_error(const rhd_batch* b);
void rhd_batch_destroy(rhd_batch* b);

/* Diagnostic: the reciprocal and reciprocal square root that the FP64
 * kernels use in place of IEEE division and square root (Newton-Raphson
 * steps from a single-precision seed), for n positive values.  x, rcp and
 * rsqrt are device buffers of n doubles owned by the caller; results go to
 * rcp[i] = 1/x[i] and rsqrt[i] = 1/sqrt(x[i]).  Lets tests bound their error
 * against IEEE results.  Runs on the legacy default stream and synchronises
 * the device.  Messages: rhd_last_error(NULL). */
rhd_status rhd_eval_recip(const double* x, int64_t n, double* rcp, double* rsqrt);

/* Diagnostic, with no counterpart in the paper: a throughput probe of the
 * fused multiply-add pipe of the FP64 arithmetic (precision RHD_PREC_FP64)
 * or of the single-precision arithmetic (RHD_PREC_MIXED), used to measure
 * the roofline denominators of the stage kernels on the GPU in use.
 * Launches nblocks blocks of 256 threads on `stream` (a cudaStream_t; NULL:
 * the legacy default stream), each thread running 8 independent chains of
 * iters multiply-adds, and returns without synchronising; *flops receives
 * the floating-point operations of the launch (2 per multiply-add), so that
 * a CUDA-event time around the call gives FLOP/s.  RHD_ERR_ARG for another
 * precision, nblocks or iters <= 0 or flops NULL.  Messages:
 * rhd_last_error(NULL). */
rhd_status rhd_fma_probe(int precision, int nblocks, int iters, void* stream, double* flops);

/* Largest grid, in cells, that rhd_step_noalloc accepts. */
#define RHD_NOALLOC_MAX_CELLS 262144

/* One IMEX step that allocates no device memory.  The paper has no
 * counterpart to this call: it serves callers that cannot allocate, such as
 * code whose device memory is wholly owned by another allocator (a
 * framework's caching pool) or code that must not call cudaMalloc/cudaFree
 * because those calls can synchronise the whole device.
 *
 * state_in, state_out: device pointers on the current device, each holding
 * RHD_NFIELDS*ncell doubles, field-major as in rhd_state_set_all; they must
 * not overlap.  state_out receives y(n+1) (rho and kappa are copied).  Input
 * values are not checked.  dt <= 0 selects rhd_default_dt(p); a dt that is
 * not finite returns RHD_ERR_ARG.  stream is a cudaStream_t (NULL: the
 * legacy default stream).  The caller owns both buffers.  When the step
 * fails (a status other than RHD_OK from a stage), state_in is unchanged and
 * the evolved fields of state_out are unspecified.
 *
 * The stage buffer y(n+1/2) and the status block live in file-scope device
 * arrays sized for RHD_NOALLOC_MAX_CELLS cells (16 MiB), which every GPU that
 * loads the library holds until the process exits; a larger grid returns
 * RHD_ERR_ARG with a message.  The first call on a device resolves the
 * arrays' device addresses (cudaGetSymbolAddress), a set-up to be done
 * before any stream capture begins; the addresses are kept for the life of
 * the process, so do not call this entry point again on a device after a
 * cudaDeviceReset of it.  All calls share the arrays: each call clears the
 * status block and rewrites the stage buffer, and calls that overlap on the
 * GPU (other streams or host threads) race.  Every call copies the status
 * block to the host and synchronises its stream before returning; info
 * (nullable) is filled as by rhd_step, with t = dt.  Messages:
 * rhd_last_error(NULL). */
rhd_status rhd_step_noalloc(const rhd_params* p, const double* state_in,
                            double* state_out, double dt, void* stream,
                            rhd_step_info* info);

#ifdef __cplusplus
}
#endif
#endif /* RHD_H */
