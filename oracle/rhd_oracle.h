/*
 * rhd_oracle.h -- serial FP64 CPU oracle of one grey IMEX PD-ARS radiation step
 * (He, Wibking & Krumholz 2024, "An asymptotically-correct implicit-explicit
 * time integration scheme for finite volume radiation-hydrodynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path.  Only
 * the tests, the package smoke check and the benchmark's CPU-baseline leg may
 * load or call it; the library never does, and it shares no code, header or
 * constant with the CUDA path.
 *
 * Everything is plain, slow, double precision, in the order the paper states
 * it:
 *   Sec. 3.2  eq. (yrsla), PD-ARS tableau, eq. (imex1), eq. (imex2)
 *   Sec. 3.3  Godunov transport (PLM faces + HLL; Sec. 4.3 wave speeds and the
 *             optional optical-depth correction of the HLL energy flux),
 *             eq. (egupdate)-(fupdate), eq. (FGFR), eq. (Rnew), the Newton
 *             Jacobian eq. (linear), the convergence test, the energy closure,
 *             eq. (numF1)/(numF2), the momentum update and the outer iteration.
 *
 * State layout: one array of ORC_NFIELD * ncell doubles, field-major, cell
 * index i + nx*(j + ny*k) (x fastest).  F is the physical lab-frame flux.
 */
#ifndef RHD_ORACLE_H
#define RHD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* field order inside the state array */
enum { ORC_RHO = 0, ORC_MX, ORC_MY, ORC_MZ, ORC_EGAS, ORC_ERAD, ORC_FX, ORC_FY,
       ORC_FZ, ORC_KAPPA, ORC_NFIELD };

enum { ORC_BC_PERIODIC = 0, ORC_BC_REFLECT = 1, ORC_BC_INFLOW = 2 };
enum { ORC_SCHEME_IMEX = 0, ORC_SCHEME_RK2_SSP = 1 };
enum { ORC_RECON_PLM = 0, ORC_RECON_PPM = 1, ORC_RECON_PPM_CS = 2 };
enum { ORC_CLOSURE_M1 = 0, ORC_CLOSURE_EDDINGTON = 1 };
enum { ORC_HLL_TAU = 0, ORC_HLL_NONE = 1 };

/* status codes */
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NEWTON = 3, ORC_ERR_OUTER = 4,
       ORC_ERR_NONPHYSICAL = 5 };

typedef struct {
  int ndim;               /* 1, 2 or 3 */
  long long n[3];         /* cells per axis (unused axes = 1) */
  double dx[3];           /* cell widths */
  int bc[3][2];           /* [axis][lo/hi] boundary kind */
  double gamma;           /* adiabatic index */
  double c, chat;         /* speed of light and reduced speed of light */
  double a_rad;           /* radiation constant a_r (4 pi B / c = a_r T^4) */
  double kB_over_mu;      /* k_B / (mu m_H): c_v = kB_over_mu / (gamma - 1) */
  double cfl;             /* CFL number for the default time step */
  int closure;            /* ORC_CLOSURE_* */
  int vc_order;           /* 1: eq. (numF1); 2: eq. (numF2) and (1+beta^2/2) */
  int hll_mode;           /* ORC_HLL_* */
  double newton_rtol;     /* epsilon of the inner convergence test */
  double outer_rtol;      /* tolerance of the outer iteration */
  int newton_max_iter;
  int outer_max_iter;
  int scheme;             /* ORC_SCHEME_*: eq. imex1/imex2, or RK2-SSP (Sec. 4.2) */
  double kappa_T_exp;     /* chi = kappa rho (T / kappa_T_ref)^kappa_T_exp */
  double kappa_T_ref;
  double bc_state[3][2][4]; /* ghost E, Fx, Fy, Fz of ORC_BC_INFLOW faces */
  double kappa_P_ratio;   /* chi_0P / chi_0E (1: grey) */
  double kappa_F_ratio;   /* chi_0F / chi_0E (1: grey) */
  int reconstruction;     /* ORC_RECON_*: face states of the transport */
  double cfl_hydro;       /* CFL number of the hydrodynamic step */
} orc_params;

typedef struct {
  int status;             /* ORC_* code of the first failure, 0 if none */
  long long fail_cell;    /* cell index of the first failure, -1 if none */
  int max_newton;         /* most Newton updates taken by one local solve */
  int max_outer;          /* most outer passes taken by one local solve */
  long long sum_newton;   /* total Newton updates */
  long long n_solves;     /* number of local solves */
} orc_info;

/* Default time step: CFL / (chat * sum_d 1/dx_d). */
double orc_dt(const orc_params* p);

/* Eddington tensor D (P = D E) of one radiation state; F physical. */
void orc_eddington_tensor(const orc_params* p, double E, const double F[3],
                          double D[3][3]);

/* Transport operator s(y) of eq. (yrsla): rates dE/dt and dF/dt (physical F)
 * for every cell.  rate has 4*ncell doubles: E, Fx, Fy, Fz (field-major).
 * Returns ORC_OK or ORC_ERR_NONPHYSICAL (a face state with E <= 0). */
int orc_transport(const orc_params* p, const double* U, double* rate,
                  long long* fail_cell);

/* Implicit local solve of one cell, eq. (egupdate)-(fupdate), with the
 * stage weight theta.  y = {Egas, mx, my, mz, E, Fx, Fy, Fz} holds the state
 * after the explicit terms on input and the solution on output.  chi is
 * kappa rho; with kappa_T_exp != 0 the opacity is chi (T/kappa_T_ref)^exp at
 * the current gas temperature. */
int orc_local_solve(const orc_params* p, double theta, double dt, double rho,
                    double chi, double y[8], int* n_newton, int* n_outer);

/* One full IMEX PD-ARS step of size dt (dt <= 0: orc_dt). */
int orc_step(const orc_params* p, double* U, double dt, orc_info* info);

/* Conserved totals: [0] = sum (Egas + (c/chat) E) V,
 * [1..3] = sum (m + F/(c chat)) V. */
void orc_totals(const orc_params* p, const double* U, double out[4]);

/* ---- adjoint (rhd_oracle_adj.c) ----
 * Tapes and adjoint states are slot-major: 8 slots (Egas, mx, my, mz, E, Fx,
 * Fy, Fz) of ncell doubles each. */

/* One step as orc_step that also writes the tape: y(n), y(n+1/2), y(n+1),
 * 3 x 8 x ncell doubles. */
/* ---- the hydrodynamic subsystem and the operator split (Sec. 3.1),
 * rhd_oracle_hydro.c ---- */

/* dt of the hydrodynamic step: cfl_hydro / max over cells of
 * sum_d (|v_d| + a)/dx_d, a the adiabatic sound speed; <= 0 if a cell is
 * nonphysical. */
double orc_hydro_dt(const orc_params* p, const double* U);

/* Rates d(rho, m_x, m_y, m_z, E_gas)/dt of the Euler equations (Sec. 3.1),
 * rate[5][N]. */
int orc_hydro_rate(const orc_params* p, const double* U, double* rate,
                   long long* fail_cell);

/* One RK2-SSP step of the hydrodynamic subsystem; the radiation fields are
 * untouched.  On failure U is left unchanged. */
int orc_hydro_step(const orc_params* p, double* U, double dt, long long* fail_cell);

/* One operator-split step: the hydrodynamic step of dt_h (dt_h <= 0:
 * orc_hydro_dt), then nsub = ceil(dt_h / orc_dt - 1e-12) radiation steps of
 * dt_h / nsub.  *nsub_out (nullable) receives nsub. */
int orc_split_step(const orc_params* p, double* U, double dt_h, orc_info* info,
                   int* nsub_out);

/* the transport's reconstruction, shared with the hydrodynamic subsystem */
double orc_recon_mc_slope(double um, double u0, double up);
void orc_recon_ppm_edges(const double u[5], double* aL, double* aR);
void orc_recon_ppm_cs_edges(const double u[5], double* aL, double* aR);

int orc_step_tape(const orc_params* p, double* U, double dt, double* tape);

/* Adjoint of one taped step: ybar0 = dL/dy(n) from ybar1 = dL/dy(n+1);
 * kbar (ncell) += dL/dkappa.  rho, kappa: the static fields. */
int orc_step_adjoint(const orc_params* p, const double* rho, const double* kappa,
                     const double* tape, double dt, const double* ybar1,
                     double* ybar0, double* kbar);

/* Adjoint of one converged local solve (implicit-function theorem). */
int orc_local_solve_adjoint(const orc_params* p, double theta, double dt, double rho,
                            double chi, const double yout[8], const double ybar_out[8],
                            double ybar_in[8], double* chibar);

#ifdef __cplusplus
}
#endif
#endif
