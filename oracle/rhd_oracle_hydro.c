/*
 * rhd_oracle_hydro.c -- serial FP64 CPU oracle of the hydrodynamic
 * subsystem of Sec. 3.1 (the Euler equations advanced explicitly by a
 * method of lines with RK2-SSP) and of the operator split that subcycles the
 * radiation step (rhd_oracle.c) inside each hydrodynamic step.
 *
 * TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU baseline are
 * its only users.  Plain loops over cells and faces.
 *
 * The paper delegates the hydrodynamic method to its host code; the
 * readings below are textbook choices:
 *   - state (rho, m, E_gas), E_gas the total gas energy, ideal gas
 *     p = (gamma - 1)(E_gas - |m|^2 / (2 rho));
 *   - face states: the primitives (rho, v, p) reconstructed with the
 *     transport's option (PLM with the MC limiter, PPM, or PPM with the
 *     Colella-Sekora limiter), per component;
 *   - fluxes: the HLLC Riemann solver (Toro, Spruce & Speares 1994) with
 *     the wave-speed bounds S_L = min(u_L - a_L, u_R - a_R),
 *     S_R = max(u_L + a_L, u_R + a_R) (Davis 1988);
 *   - time: RK2-SSP (Shu & Osher 1988), U1 = U + dt L(U),
 *     U(n+1) = (U + U1 + dt L(U1)) / 2;
 *   - ghost cells: periodic wrap, or a reflecting wall that mirrors the cell
 *     and negates the normal velocity.  An inflow axis (a radiation boundary)
 *     is refused.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "rhd_oracle.h"

static long long ncell(const orc_params* p) { return p->n[0] * p->n[1] * p->n[2]; }

static const int HYD_FIELD[5] = {ORC_RHO, ORC_MX, ORC_MY, ORC_MZ, ORC_EGAS};

typedef struct {
  double rho, v[3], p;
} prim;

static prim to_prim(const orc_params* p, const double* U, long long idx) {
  const long long N = ncell(p);
  prim w;
  w.rho = U[ORC_RHO * N + idx];
  double ke = 0.0;
  for (int j = 0; j < 3; ++j) {
    w.v[j] = U[(ORC_MX + j) * N + idx] / w.rho;
    ke += 0.5 * w.rho * w.v[j] * w.v[j];
  }
  w.p = (p->gamma - 1.0) * (U[ORC_EGAS * N + idx] - ke);
  return w;
}

/* primitive state of the cell at ic shifted by off along axis d */
static prim hfetch(const orc_params* p, const double* U, const long long ic[3], int d,
                   int off) {
  long long q[3] = {ic[0], ic[1], ic[2]};
  const long long nd = p->n[d];
  long long x = q[d] + off;
  int flip = 0;
  if (x < 0) {
    if (p->bc[d][0] == ORC_BC_PERIODIC) {
      x = ((x % nd) + nd) % nd;
    } else {
      x = -1 - x;
      flip = 1;
    }
  } else if (x >= nd) {
    if (p->bc[d][1] == ORC_BC_PERIODIC) {
      x = x % nd;
    } else {
      x = 2 * nd - 1 - x;
      flip = 1;
    }
  }
  if (x < 0) x = 0;       /* a mirror deeper than the axis: cells the */
  if (x >= nd) x = nd - 1; /* reconstruction in use does not read      */
  q[d] = x;
  prim w = to_prim(p, U, q[0] + p->n[0] * (q[1] + p->n[1] * q[2]));
  if (flip) w.v[d] = -w.v[d];
  return w;
}

static double comp(const prim* w, int k) { return k == 0 ? w->rho : (k == 4 ? w->p : w->v[k - 1]); }

static void set_comp(prim* w, int k, double x) {
  if (k == 0)
    w->rho = x;
  else if (k == 4)
    w->p = x;
  else
    w->v[k - 1] = x;
}

/* face states between s[2] and s[3] of the six cells s[0..5] */
static void hface_states(const orc_params* p, const prim s[6], prim* L, prim* R) {
  for (int k = 0; k < 5; ++k) {
    double u[6];
    for (int o = 0; o < 6; ++o) u[o] = comp(&s[o], k);
    double l, r;
    if (p->reconstruction == ORC_RECON_PPM || p->reconstruction == ORC_RECON_PPM_CS) {
      void (*edges)(const double*, double*, double*) =
          p->reconstruction == ORC_RECON_PPM ? orc_recon_ppm_edges : orc_recon_ppm_cs_edges;
      double al, ar, bl, br;
      edges(u, &al, &ar);     /* cell s[2] */
      edges(u + 1, &bl, &br); /* cell s[3] */
      l = ar;
      r = bl;
    } else {
      l = u[2] + 0.5 * orc_recon_mc_slope(u[1], u[2], u[3]);
      r = u[3] - 0.5 * orc_recon_mc_slope(u[2], u[3], u[4]);
    }
    set_comp(L, k, l);
    set_comp(R, k, r);
  }
}

/* physical flux of the Euler equations along d: (rho u, rho u v + p e_d,
 * (E + p) u); also the conserved state */
static void euler_flux(const orc_params* p, int d, const prim* w, double U[5], double F[5]) {
  const double u = w->v[d];
  double ke = 0.5 * w->rho * (w->v[0] * w->v[0] + w->v[1] * w->v[1] + w->v[2] * w->v[2]);
  double E = w->p / (p->gamma - 1.0) + ke;
  U[0] = w->rho;
  F[0] = w->rho * u;
  for (int j = 0; j < 3; ++j) {
    U[1 + j] = w->rho * w->v[j];
    F[1 + j] = w->rho * u * w->v[j] + (j == d ? w->p : 0.0);
  }
  U[4] = E;
  F[4] = (E + w->p) * u;
}

/* HLLC flux through a face along d (Toro, Riemann Solvers and Numerical
 * Methods for Fluid Dynamics, 3rd ed., Sec. 10.4: the contact speed S* and
 * the star states U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S* in the normal
 * and v_K in the transverse momentum, E_K/rho_K + (S* - u_K)(S* +
 * p_K/(rho_K (S_K - u_K))))) */
static int hllc(const orc_params* p, int d, const prim* L, const prim* R, double F[5]) {
  if (!(L->rho > 0.0) || !(L->p > 0.0) || !(R->rho > 0.0) || !(R->p > 0.0))
    return ORC_ERR_NONPHYSICAL;
  const double g = p->gamma;
  const double aL = sqrt(g * L->p / L->rho), aR = sqrt(g * R->p / R->rho);
  const double uL = L->v[d], uR = R->v[d];
  const double SL = fmin(uL - aL, uR - aR);
  const double SR = fmax(uL + aL, uR + aR);
  double UL[5], FL[5], UR[5], FR[5];
  euler_flux(p, d, L, UL, FL);
  euler_flux(p, d, R, UR, FR);
  if (SL >= 0.0) {
    memcpy(F, FL, sizeof(FL));
    return ORC_OK;
  }
  if (SR <= 0.0) {
    memcpy(F, FR, sizeof(FR));
    return ORC_OK;
  }
  const double Ss = (R->p - L->p + L->rho * uL * (SL - uL) - R->rho * uR * (SR - uR)) /
                    (L->rho * (SL - uL) - R->rho * (SR - uR));
  const prim* K = Ss >= 0.0 ? L : R;
  const double SK = Ss >= 0.0 ? SL : SR;
  const double* UK = Ss >= 0.0 ? UL : UR;
  const double* FK = Ss >= 0.0 ? FL : FR;
  const double uK = K->v[d];
  const double fac = K->rho * (SK - uK) / (SK - Ss);
  double Us[5];
  Us[0] = fac;
  for (int j = 0; j < 3; ++j) Us[1 + j] = fac * (j == d ? Ss : K->v[j]);
  Us[4] = fac * (UK[4] / K->rho + (Ss - uK) * (Ss + K->p / (K->rho * (SK - uK))));
  for (int q = 0; q < 5; ++q) F[q] = FK[q] + SK * (Us[q] - UK[q]);
  return ORC_OK;
}

static int axis_ok(const orc_params* p) {
  for (int d = 0; d < p->ndim; ++d)
    if (p->bc[d][0] == ORC_BC_INFLOW || p->bc[d][1] == ORC_BC_INFLOW) return 0;
  return 1;
}

double orc_hydro_dt(const orc_params* p, const double* U) {
  const long long N = ncell(p);
  double smax = 0.0;
  for (long long i = 0; i < N; ++i) {
    prim w = to_prim(p, U, i);
    if (!(w.rho > 0.0) || !(w.p > 0.0)) return -1.0;
    const double a = sqrt(p->gamma * w.p / w.rho);
    double s = 0.0;
    for (int d = 0; d < p->ndim; ++d) s += (fabs(w.v[d]) + a) / p->dx[d];
    if (s > smax) smax = s;
  }
  return p->cfl_hydro / smax;
}

int orc_hydro_rate(const orc_params* p, const double* U, double* rate, long long* fail_cell) {
  const long long N = ncell(p);
  memset(rate, 0, sizeof(double) * 5 * (size_t)N);
  if (fail_cell) *fail_cell = -1;
  if (!axis_ok(p)) return ORC_ERR_ARG;
  for (int d = 0; d < p->ndim; ++d)
    for (long long i2 = 0; i2 < p->n[2]; ++i2)
      for (long long i1 = 0; i1 < p->n[1]; ++i1)
        for (long long i0 = 0; i0 < p->n[0]; ++i0) {
          const long long ic[3] = {i0, i1, i2};
          const long long idx = i0 + p->n[0] * (i1 + p->n[1] * i2);
          prim s[7];
          for (int o = -3; o <= 3; ++o) s[o + 3] = hfetch(p, U, ic, d, o);
          double lo[5], hi[5];
          prim L, R;
          /* face i-1/2: cells i-3 .. i+2; face i+1/2: cells i-2 .. i+3 */
          hface_states(p, &s[0], &L, &R);
          int st = hllc(p, d, &L, &R, lo);
          if (st == ORC_OK) {
            hface_states(p, &s[1], &L, &R);
            st = hllc(p, d, &L, &R, hi);
          }
          if (st != ORC_OK) {
            if (fail_cell) *fail_cell = idx;
            return st;
          }
          for (int q = 0; q < 5; ++q) rate[q * N + idx] -= (hi[q] - lo[q]) / p->dx[d];
        }
  return ORC_OK;
}

static int physical(const orc_params* p, const double* U, long long* fail_cell) {
  const long long N = ncell(p);
  for (long long i = 0; i < N; ++i) {
    prim w = to_prim(p, U, i);
    if (!(w.rho > 0.0) || !(w.p > 0.0) || !isfinite(w.p)) {
      if (fail_cell) *fail_cell = i;
      return ORC_ERR_NONPHYSICAL;
    }
  }
  return ORC_OK;
}

int orc_hydro_step(const orc_params* p, double* U, double dt, long long* fail_cell) {
  const long long N = ncell(p);
  const size_t bytes = sizeof(double) * ORC_NFIELD * (size_t)N;
  long long fc = -1;
  if (fail_cell) *fail_cell = -1;
  double* U1 = (double*)malloc(bytes);
  double* L = (double*)malloc(sizeof(double) * 5 * (size_t)N);
  if (!U1 || !L) {
    free(U1);
    free(L);
    return ORC_ERR_ARG;
  }
  int st = orc_hydro_rate(p, U, L, &fc);
  if (st == ORC_OK) {
    memcpy(U1, U, bytes);
    for (int q = 0; q < 5; ++q)
      for (long long i = 0; i < N; ++i) U1[HYD_FIELD[q] * N + i] += dt * L[q * N + i];
    st = physical(p, U1, &fc);
  }
  if (st == ORC_OK) st = orc_hydro_rate(p, U1, L, &fc);
  if (st == ORC_OK) {
    for (int q = 0; q < 5; ++q)
      for (long long i = 0; i < N; ++i) {
        const long long k = HYD_FIELD[q] * N + i;
        U1[k] = 0.5 * (U[k] + (U1[k] + dt * L[q * N + i]));
      }
    st = physical(p, U1, &fc);
  }
  if (st == ORC_OK) memcpy(U, U1, bytes);
  if (fail_cell) *fail_cell = fc;
  free(U1);
  free(L);
  return st;
}

int orc_split_step(const orc_params* p, double* U, double dt_h, orc_info* info,
                   int* nsub_out) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->fail_cell = -1;
  }
  if (nsub_out) *nsub_out = 0;
  if (!(dt_h > 0.0)) dt_h = orc_hydro_dt(p, U);
  if (!(dt_h > 0.0)) {
    if (info) info->status = ORC_ERR_NONPHYSICAL;
    return ORC_ERR_NONPHYSICAL;
  }
  long long fc = -1;
  int st = orc_hydro_step(p, U, dt_h, &fc);
  if (st != ORC_OK) {
    if (info) {
      info->status = st;
      info->fail_cell = fc;
    }
    return st;
  }
  const double dt_rad = orc_dt(p);
  int nsub = (int)ceil(dt_h / dt_rad - 1e-12);
  if (nsub < 1) nsub = 1;
  if (nsub_out) *nsub_out = nsub;
  for (int k = 0; k < nsub; ++k) {
    orc_info one;
    st = orc_step(p, U, dt_h / nsub, &one);
    if (info) {
      if (one.max_newton > info->max_newton) info->max_newton = one.max_newton;
      if (one.max_outer > info->max_outer) info->max_outer = one.max_outer;
      info->sum_newton += one.sum_newton;
      info->n_solves += one.n_solves;
    }
    if (st != ORC_OK) {
      if (info) {
        info->status = st;
        info->fail_cell = one.fail_cell;
      }
      return st;
    }
  }
  return ORC_OK;
}
