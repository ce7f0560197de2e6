/*
 * rhd_oracle.c -- serial FP64 CPU oracle of one grey IMEX PD-ARS radiation
 * step (He, Wibking & Krumholz 2024).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU baseline are its only users.  It is deliberately plain: no blocking, no
 * fusion, loops over cells and faces in the order the paper describes them.
 *
 * Readings of passages the paper leaves open are marked "reading:" below.
 */
#include "rhd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static long long ncell_of(const orc_params* p) {
  return p->n[0] * p->n[1] * p->n[2];
}

/* ---------------------------------------------------------------- time step */

/* Sec. 4.3: the radiation wave speed never exceeds the (reduced) speed of
 * light, so the explicit CFL step is fixed by chat and the cell widths.
 * reading: multi-dimensional CFL = CFL / (chat * sum_d 1/dx_d). */
double orc_dt(const orc_params* p) {
  double s = 0.0;
  for (int d = 0; d < p->ndim; ++d) s += 1.0 / p->dx[d];
  return p->cfl / (p->chat * s);
}

/* ------------------------------------------------------------- the closure */

/* The paper leaves the closure free (Sec. 2.1).  reading: Levermore's M1
 * closure, P = D E with D = (1-xi)/2 I + (3 xi - 1)/2 n n, reduced flux
 * f = |F| / (c E) clipped to [0, 1], xi = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)).
 * Zero flux gives the isotropic D = I/3.  The Eddington option is D = I/3. */
void orc_eddington_tensor(const orc_params* p, double E, const double F[3],
                          double D[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = (i == j) ? 1.0 / 3.0 : 0.0;
  if (p->closure == ORC_CLOSURE_EDDINGTON) return;
  double Fmag = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  if (Fmag == 0.0) return;
  double f = Fmag / (p->c * E);
  if (f > 1.0) f = 1.0;
  if (f < 0.0) f = 0.0;
  double xi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
  double nhat[3] = {F[0] / Fmag, F[1] / Fmag, F[2] / Fmag};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      D[i][j] = 0.5 * (1.0 - xi) * (i == j ? 1.0 : 0.0) +
                0.5 * (3.0 * xi - 1.0) * nhat[i] * nhat[j];
}

/* ---------------------------------------------------------- reconstruction */

/* reading: PLM with the monotonised-central limiter,
 * slope = minmod(2 d-, (d- + d+)/2, 2 d+), minmod of mixed signs = 0. */
static double minmod3(double a, double b, double c) {
  if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
  if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
  return 0.0;
}

static double mc_slope(double um, double u0, double up) {
  double dm = u0 - um;
  double dp = up - u0;
  return minmod3(2.0 * dm, 0.5 * (dm + dp), 2.0 * dp);
}

/* One cell's radiation variables as the transport sees them. */
typedef struct {
  double E;
  double F[3];
  double chi;
} rad_cell;

/* Fetch the cell at coordinate (i0,i1,i2) shifted by off along axis d, with
 * ghost cells made by the boundary condition.  reading: periodic wrap, or a
 * reflecting wall that mirrors the cell and negates the normal flux. */
static rad_cell fetch(const orc_params* p, const double* U, const long long ic[3],
                      int d, int off) {
  long long q[3] = {ic[0], ic[1], ic[2]};
  long long nd = p->n[d];
  long long x = q[d] + off;
  int flip = 0, inflow = -1; /* inflow: side (0 low, 1 high) of an inflow ghost */
  if (x < 0) {
    if (p->bc[d][0] == ORC_BC_PERIODIC) {
      x = ((x % nd) + nd) % nd;
    } else {
      if (p->bc[d][0] == ORC_BC_INFLOW) inflow = 0;
      x = -1 - x;
      flip = 1;
    }
  } else if (x >= nd) {
    if (p->bc[d][1] == ORC_BC_PERIODIC) {
      x = x % nd;
    } else {
      if (p->bc[d][1] == ORC_BC_INFLOW) inflow = 1;
      x = 2 * nd - 1 - x;
      flip = 1;
    }
  }
  /* a mirror deeper than the axis (only for stencil cells that the
   * reconstruction in use does not read, e.g. PLM's outermost pair) */
  if (x < 0) x = 0;
  if (x >= nd) x = nd - 1;
  q[d] = x;
  long long N = ncell_of(p);
  long long idx = q[0] + p->n[0] * (q[1] + p->n[1] * q[2]);
  rad_cell r;
  r.E = U[ORC_ERAD * N + idx];
  r.F[0] = U[ORC_FX * N + idx];
  r.F[1] = U[ORC_FY * N + idx];
  r.F[2] = U[ORC_FZ * N + idx];
  if (flip) r.F[d] = -r.F[d];
  r.chi = U[ORC_KAPPA * N + idx] * U[ORC_RHO * N + idx];
  if (inflow >= 0) {
    /* reading: an inflow ghost holds the face's fixed radiation state; its
     * opacity (used only by the TAU factor) is that of the mirrored cell */
    r.E = p->bc_state[d][inflow][0];
    for (int j = 0; j < 3; ++j) r.F[j] = p->bc_state[d][inflow][1 + j];
  }
  return r;
}

/* PPM interface value between cells j and j+1 (Colella & Woodward 1984,
 * uniform zones): (u_j + u_{j+1})/2 - (dm_{j+1} - dm_j)/6 with dm the
 * MC-limited slopes; from u_{j-1} .. u_{j+2}. */
static double ppm_interface(double um, double u0, double up, double upp) {
  return 0.5 * (u0 + up) - (mc_slope(u0, up, upp) - mc_slope(um, u0, up)) / 6.0;
}

/* PPM edge values (aL, aR) of cell j from u_{j-2} .. u_{j+2}, made monotone
 * (Colella & Woodward 1984): a cell at an extremum is flat, and an edge value
 * that would put an extremum of the parabola inside the cell is moved. */
static void ppm_edges(const double u[5], double* aL, double* aR) {
  double l = ppm_interface(u[0], u[1], u[2], u[3]);
  double r = ppm_interface(u[1], u[2], u[3], u[4]);
  double u0 = u[2];
  if ((r - u0) * (u0 - l) <= 0.0) {
    l = r = u0;
  } else {
    double dd = r - l, m6 = 6.0 * (u0 - 0.5 * (l + r));
    if (dd * m6 > dd * dd)
      l = 3.0 * u0 - 2.0 * r;
    else if (-dd * dd > dd * m6)
      r = 3.0 * u0 - 2.0 * l;
  }
  *aL = l;
  *aR = r;
}

/* The PPM limiter of Colella & Sekora (2008), which keeps smooth extrema
 * (the option ORC_RECON_PPM_CS; C = 1.25).  Interface value between cells j
 * and j+1 from u_{j-1} .. u_{j+2}: the fourth-order value
 * 7/12 (u_j + u_{j+1}) - 1/12 (u_{j-1} + u_{j+2}); if it does not lie
 * between u_j and u_{j+1}, its second difference 3 (u_j - 2a + u_{j+1}) is
 * limited against the second differences of the cells on either side (the
 * smallest magnitude if all three share a sign, else zero) and
 * a = (u_j + u_{j+1})/2 - D2_lim/6. */
static const double CS_C = 1.25;

static int same_sign3(double a, double b, double c) {
  return (a > 0.0 && b > 0.0 && c > 0.0) || (a < 0.0 && b < 0.0 && c < 0.0);
}

static double cs_interface(double um, double u0, double up, double upp) {
  double a = 7.0 / 12.0 * (u0 + up) - 1.0 / 12.0 * (um + upp);
  if ((a - u0) * (up - a) < 0.0) {
    double d2 = 3.0 * (u0 - 2.0 * a + up);
    double d2l = um - 2.0 * u0 + up;
    double d2r = u0 - 2.0 * up + upp;
    double lim = 0.0;
    if (same_sign3(d2, d2l, d2r)) {
      double m = fmin(CS_C * fabs(d2), fmin(fabs(d2l), fabs(d2r)));
      lim = d2 > 0.0 ? m : -m;
    }
    a = 0.5 * (u0 + up) - lim / 6.0;
  }
  return a;
}

/* Edge values (aL, aR) of cell j from u_{j-2} .. u_{j+2} with the
 * Colella-Sekora constraint: at a local extremum (of the edge values or of
 * the cell averages) the parabola's curvature -12 u_j + 6 (aL + aR) is
 * limited against C times the second differences of cells j-1, j and j+1
 * (smallest magnitude if all share its sign, else zero) and both edges are
 * scaled towards u_j by the ratio; elsewhere an edge more than twice as far
 * from u_j as the other is moved to twice that distance (as in the
 * Colella-Woodward constraint), so the parabola stays monotone. */
static void ppm_cs_edges(const double u[5], double* aL, double* aR) {
  double l = cs_interface(u[0], u[1], u[2], u[3]);
  double r = cs_interface(u[1], u[2], u[3], u[4]);
  const double u0 = u[2];
  if ((r - u0) * (u0 - l) <= 0.0 || (u[1] - u0) * (u0 - u[3]) <= 0.0) {
    double d2 = -12.0 * u0 + 6.0 * (l + r);
    double d2c = u[1] - 2.0 * u0 + u[3];
    double d2l = u[0] - 2.0 * u[1] + u0;
    double d2r = u0 - 2.0 * u[3] + u[4];
    double lim = 0.0;
    if (same_sign3(d2, d2c, d2l) && same_sign3(d2, d2c, d2r)) {
      double m = fmin(fabs(d2), CS_C * fmin(fabs(d2c), fmin(fabs(d2l), fabs(d2r))));
      lim = d2 > 0.0 ? m : -m;
    }
    if (d2 != 0.0) {
      double fac = lim / d2;
      l = u0 + (l - u0) * fac;
      r = u0 + (r - u0) * fac;
    } else {
      l = r = u0;
    }
  } else {
    double dl = u0 - l, dr = r - u0;
    if (fabs(dr) >= 2.0 * fabs(dl))
      r = u0 + 2.0 * dl;
    else if (fabs(dl) >= 2.0 * fabs(dr))
      l = u0 - 2.0 * dr;
  }
  *aL = l;
  *aR = r;
}

/* Face states of the face between s[2] and s[3] along axis d from the
 * stencil s[0..5] (cells i-2 .. i+3): E and F.
 *   PLM (reading: Sec. 3.3 uses PPM; PLM with the monotonised-central
 *   limiter is the default): cell a + half its slope | cell b - half its
 *   slope, from s[1..4];
 *   PPM: the right edge value of s[2] | the left edge value of s[3]. */
static void face_states(const orc_params* p, const rad_cell* s, double* EL, double FL[3],
                        double* ER, double FR[3]) {
  if (p->reconstruction == ORC_RECON_PPM || p->reconstruction == ORC_RECON_PPM_CS) {
    void (*edges)(const double*, double*, double*) =
        p->reconstruction == ORC_RECON_PPM ? ppm_edges : ppm_cs_edges;
    double u[6], l, r;
    for (int q = 0; q < 4; ++q) {
      for (int k = 0; k < 6; ++k) u[k] = q == 0 ? s[k].E : s[k].F[q - 1];
      edges(u, &l, &r);       /* cell s[2] */
      double left = r;
      edges(u + 1, &l, &r);   /* cell s[3] */
      if (q == 0) {
        *EL = left;
        *ER = l;
      } else {
        FL[q - 1] = left;
        FR[q - 1] = l;
      }
    }
    return;
  }
  const rad_cell *am = &s[1], *a = &s[2], *b = &s[3], *bp = &s[4];
  *EL = a->E + 0.5 * mc_slope(am->E, a->E, b->E);
  *ER = b->E - 0.5 * mc_slope(a->E, b->E, bp->E);
  for (int j = 0; j < 3; ++j) {
    FL[j] = a->F[j] + 0.5 * mc_slope(am->F[j], a->F[j], b->F[j]);
    FR[j] = b->F[j] - 0.5 * mc_slope(a->F[j], b->F[j], bp->F[j]);
  }
}

/* HLL flux through the face between cells s[2] and s[3] along axis d, for
 * the RSLA transport system of eq. (yrsla): conserved (E, F/(c chat)) with
 * fluxes ((chat/c) F_d, P_d.).  out[0] = energy flux, out[1..3] = flux of
 * F/(c chat). */
static int hll_face(const orc_params* p, int d, const rad_cell* s, double out[4]) {
  const double c = p->c, chat = p->chat;
  const rad_cell *a = &s[2], *b = &s[3];
  double EL = 0.0, ER = 0.0, FL[3], FR[3];
  face_states(p, s, &EL, FL, &ER, FR);
  if (!(EL > 0.0) || !(ER > 0.0)) return ORC_ERR_NONPHYSICAL;
  /* reading: a reconstructed face flux above the free-streaming limit
   * |F| <= c E is scaled back onto that limit. */
  double nL = sqrt(FL[0] * FL[0] + FL[1] * FL[1] + FL[2] * FL[2]);
  double nR = sqrt(FR[0] * FR[0] + FR[1] * FR[1] + FR[2] * FR[2]);
  if (nL > c * EL)
    for (int j = 0; j < 3; ++j) FL[j] *= c * EL / nL;
  if (nR > c * ER)
    for (int j = 0; j < 3; ++j) FR[j] *= c * ER / nR;

  double DL[3][3], DR[3][3];
  orc_eddington_tensor(p, EL, FL, DL);
  orc_eddington_tensor(p, ER, FR, DR);

  /* Sec. 4.3: S = +-sqrt(f) c with f the Eddington-tensor component along the
   * face normal; under the RSLA the speed is chat.  reading: the larger of the
   * two sides, never below the diffusion-limit value 1/sqrt(3). */
  double sf = fmax(sqrt(DL[d][d]), sqrt(DR[d][d]));
  sf = fmax(sf, 1.0 / sqrt(3.0));
  double SR = chat * sf;
  double SL = -SR;

  /* Sec. 4.3 HLL energy flux with the factor epsilon on the diffusive term.
   * NONE (the paper's IMEX method): epsilon = 1.  TAU: reading,
   * epsilon = (1 - exp(-tau)) / tau with tau the optical depth of one cell
   * width at the face, which is 1 when thin and 1/tau when thick. */
  double eps = 1.0;
  if (p->hll_mode == ORC_HLL_TAU) {
    /* reading: the optical depth of the face is that of the flux-mean
     * opacity chi_0F (= chi for grey material) */
    double tau = 0.5 * (a->chi + b->chi) * p->dx[d] * p->kappa_F_ratio;
    if (tau > 0.0) eps = -expm1(-tau) / tau;
  }
  double phiL = (chat / c) * FL[d];
  double phiR = (chat / c) * FR[d];
  out[0] = (SR * phiL - SL * phiR + eps * SR * SL * (ER - EL)) / (SR - SL);
  for (int j = 0; j < 3; ++j) {
    double PL = DL[d][j] * EL;
    double PR = DR[d][j] * ER;
    double uL = FL[j] / (c * chat);
    double uR = FR[j] / (c * chat);
    out[1 + j] = (SR * PL - SL * PR + SR * SL * (uR - uL)) / (SR - SL);
  }
  return ORC_OK;
}

/* s(y) of eq. (yrsla): dE/dt = -div((chat/c) F), d(F/(c chat))/dt = -div P.
 * The rate of the physical flux F is c chat times the latter. */
int orc_transport(const orc_params* p, const double* U, double* rate,
                  long long* fail_cell) {
  const long long N = ncell_of(p);
  memset(rate, 0, sizeof(double) * 4 * (size_t)N);
  if (fail_cell) *fail_cell = -1;
  for (int d = 0; d < p->ndim; ++d) {
    for (long long i2 = 0; i2 < p->n[2]; ++i2)
      for (long long i1 = 0; i1 < p->n[1]; ++i1)
        for (long long i0 = 0; i0 < p->n[0]; ++i0) {
          long long ic[3] = {i0, i1, i2};
          long long idx = i0 + p->n[0] * (i1 + p->n[1] * i2);
          rad_cell s[7];
          for (int o = -3; o <= 3; ++o) s[o + 3] = fetch(p, U, ic, d, o);
          double lo[4], hi[4];
          /* face i-1/2: stencil cells i-3 .. i+2; face i+1/2: i-2 .. i+3 */
          if (hll_face(p, d, &s[0], lo) != ORC_OK || hll_face(p, d, &s[1], hi) != ORC_OK) {
            if (fail_cell) *fail_cell = idx;
            return ORC_ERR_NONPHYSICAL;
          }
          rate[0 * N + idx] -= (hi[0] - lo[0]) / p->dx[d];
          for (int j = 0; j < 3; ++j)
            rate[(1 + j) * N + idx] -=
                p->c * p->chat * (hi[1 + j] - lo[1 + j]) / p->dx[d];
        }
  }
  return ORC_OK;
}

/* -------------------------------------------------------- the local solve */

/* Implicit stage of one cell, Sec. 3.3, grey material: chi_0P = chi_0E =
 * chi_0F = chi, so every (chi_0F - chi_0E) term of eq. (G0), (G1), (Rnew) and
 * (numF1) vanishes and (2 chi_0E - chi_0F) = chi.
 *
 * Inner stage: Newton-Raphson on x = (Egas, R) for eq. (FGFR),
 *   F_G = Egas - Egas^(t) + (c/chat) R,   F_R = E - E^(t) - R,
 * where E(Egas, R) follows from eq. (Rnew) with v and F frozen:
 *   R = theta dt [chat chi (aT^4 - E)(1 + beta^2/2) + chi (chat/c) v.F/c],
 * with the paper's Jacobian (beta^2 terms dropped).  Outer stage: eq. (numF1)
 * or (numF2) for F, the momentum update, then a repeat of the inner stage with
 * the new v and F until the v- and F-terms of R settle. */
/* Opacity at gas temperature T: chi0 = kappa rho, times (T/T_ref)^exp when the
 * opacity depends on temperature (the paper's chi carry the superscript
 * (t+1) of the iterate, Sec. 3.3). */
static double chi_at(const orc_params* p, double chi0, double T) {
  if (p->kappa_T_exp == 0.0) return chi0;
  return chi0 * pow(T / p->kappa_T_ref, p->kappa_T_exp);
}

int orc_local_solve(const orc_params* p, double theta, double dt, double rho,
                    double chi0, double y[8], int* n_newton, int* n_outer) {
  const double c = p->c, chat = p->chat, a = p->a_rad;
  const double Cv = rho * p->kB_over_mu / (p->gamma - 1.0); /* C_v = rho c_v */
  const double Eg0 = y[0];
  const double m0[3] = {y[1], y[2], y[3]};
  const double E0 = y[4];
  const double F0[3] = {y[5], y[6], y[7]};
  const int order2 = p->vc_order == 2;
  const double rP = p->kappa_P_ratio, rF = p->kappa_F_ratio;
  *n_newton = 0;
  *n_outer = 0;

  /* With chi = 0 every exchange term of eq. (egupdate)-(fupdate) vanishes. */
  if (chi0 == 0.0) return ORC_OK;

  /* reading: E_tot = Egas^(t) + (c/chat) E^(t), the energy the source terms
   * conserve (the printed chat/c factor is read as a typo; both agree when
   * chat = c). */
  const double Etot = Eg0 + (c / chat) * E0;
  const double eps = p->newton_rtol;
  const double tdt = theta * dt;

  double Eg = Eg0, R = 0.0; /* reading: Newton starts from (Egas^(t), 0) */
  double m[3] = {m0[0], m0[1], m0[2]};
  double F[3] = {F0[0], F0[1], F0[2]};
  double E = E0;
  /* reading: the closure tensor D = P/E of the (v.v.P) term of eq. (Rnew) is
   * frozen with v and F in the inner stage: that of the explicit state in
   * the first pass, then the one of the previous pass's flux update */
  double D[3][3];
  orc_eddington_tensor(p, E0, F0, D);

  for (int outer = 0; outer < p->outer_max_iter; ++outer) {
    *n_outer = outer + 1;
    /* v, F and D frozen for the inner stage */
    double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
    double beta2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / (c * c);
    double g = order2 ? 1.0 + 0.5 * beta2 : 1.0;
    double vF = v[0] * F[0] + v[1] * F[1] + v[2] * F[2];
    double Ekin = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
    double vDv = 0.0; /* v_i D_ij v_j / c^2 */
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) vDv += v[i] * D[i][j] * v[j];
    vDv /= c * c;

    /* ---- inner Newton-Raphson on (Egas, R) ---- */
    int converged = 0;
    for (int it = 0;; ++it) {
      double T = (Eg - Ekin) / Cv;
      if (!(T > 0.0) || !isfinite(T) || !isfinite(R)) return ORC_ERR_NONPHYSICAL;
      double aT4 = a * T * T * T * T; /* 4 pi B / c */
      /* eq. (G0): chi_0E = chi, chi_0P = rP chi, chi_0F = rF chi, all at the
       * current temperature (their ratios are constant) */
      double chiE = chi_at(p, chi0, T), chiP = rP * chiE, chiF = rF * chiE;
      /* E as a function of (Egas, R): eq. (Rnew) solved for E, with
       * P = D E; order 1 keeps the O(v/c) terms only */
      double num = chiP * aT4 * g + (2.0 * chiE - chiF) * vF / (c * c) - R / (chat * tdt);
      double den = chiE * g - (order2 ? (chiF - chiE) * (beta2 + vDv) : 0.0);
      double Ex = num / den;
      double FG = Eg - Eg0 + (c / chat) * R;
      double FR = Ex - E0 - R;
      if (fabs(FG / Etot) < eps && fabs((c / chat) * FR / Etot) < eps) {
        converged = 1;
        break;
      }
      if (it >= p->newton_max_iter) break;
      /* Jacobian of eq. (linear), the paper's simplified form (v^2/c^2 terms
       * dropped, chiP/chiE constant) */
      double J00 = 1.0;
      double J01 = c / chat;
      double J10 = (chiP / chiE) * 4.0 * a * T * T * T / Cv; /* (1/C_v) d(chiP/chiE aT^4)/dT */
      /* reading: with chi = chi0 (T/T_ref)^p the -R/(chat theta dt den) term
       * of E(Egas, R) above depends on T through den (proportional to
       * chi_0E), which adds p R/(T chat theta dt den) to dE/dT.  The printed
       * J10 is dE/dEgas at constant chi; Sec. 3.3 notes that the Jacobian
       * sets only the rate of convergence, not the converged solution, and
       * with the exact term the iteration converges quadratically instead of
       * linearly. */
      if (p->kappa_T_exp != 0.0)
        J10 += p->kappa_T_exp * R / (T * chat * tdt * den) / Cv;
      double J11 = -1.0 / (chat * chiE * tdt) - 1.0;
      double det = J00 * J11 - J01 * J10;
      double dEg = (-FG * J11 + FR * J01) / det;
      double dR = (-FR * J00 + FG * J10) / det;
      Eg += dEg;
      R += dR;
      *n_newton += 1;
    }
    if (!converged) return ORC_ERR_NEWTON;

    /* Energy closure: F_G = F_R = 0 give E - E^(t) = R = -(chat/c)(Egas -
     * Egas^(t)).  reading: the printed c/chat factor is read as chat/c, the
     * form consistent with eq. (FGFR) (they agree when chat = c). */
    E = E0 - (chat / c) * (Eg - Eg0);

    /* ---- outer stage: flux and momentum ---- */
    double T = (Eg - Ekin) / Cv;
    double aT4 = a * T * T * T * T;
    double chiE = chi_at(p, chi0, T), chiP = rP * chiE, chiF = rF * chiE;
    orc_eddington_tensor(p, E, F, D); /* reading: P from the new E and the
                                         flux of the previous outer pass */
    double rhs[3];
    for (int i = 0; i < 3; ++i) {
      double vP = 0.0;
      for (int j = 0; j < 3; ++j) vP += v[j] * D[j][i] * E; /* v_j P_ji */
      rhs[i] = F0[i] + chat * tdt * (chiP * aT4 * v[i] + chiF * vP + (chiF - chiE) * E * v[i]);
    }
    double Fn[3], mn[3];
    if (order2) {
      /* eq. (fupdate) with eq. (G1) to O(v^2/c^2):
       *   [(1 + chat theta dt chiF g) I + b v v^T] F = rhs,
       *   b = 2 chat theta dt (chiF - chiE)/c^2 (zero for grey material,
       *   eq. numF2), solved by the Sherman-Morrison formula */
      double aa = 1.0 + chat * chiF * g * tdt;
      double b = 2.0 * chat * tdt * (chiF - chiE) / (c * c);
      double vr = v[0] * rhs[0] + v[1] * rhs[1] + v[2] * rhs[2];
      double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      double corr = b * vr / (aa + b * v2);
      for (int i = 0; i < 3; ++i) Fn[i] = (rhs[i] - corr * v[i]) / aa;
    } else {
      for (int i = 0; i < 3; ++i) Fn[i] = rhs[i] / (1.0 + chat * chiF * tdt); /* (numF1) */
    }
    for (int i = 0; i < 3; ++i) mn[i] = m0[i] - (Fn[i] - F0[i]) / (c * chat); /* momentum */

    /* reading: the "terms proportional to v and F in R" of eq. (Rnew) are
     *   Q = theta dt chat [(chiP aT^4 - chiE E)(g - 1) + (2 chiE - chiF) v.F/c^2
     *                      + (chiF - chiE)(beta^2 + v.D.v/c^2) E]
     * (order 1: the v.F term alone); compare the Q the inner stage used with
     * the Q of the updated v and F (and the closure the next pass freezes).
     * The change is also measured against the magnitude of the terms, Qs,
     * so that a Q which is a cancelling sum cannot cycle at its rounding
     * level. */
    double vn[3] = {mn[0] / rho, mn[1] / rho, mn[2] / rho};
    double beta2n = (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]) / (c * c);
    double gn = order2 ? 1.0 + 0.5 * beta2n : 1.0;
    double vFn = vn[0] * Fn[0] + vn[1] * Fn[1] + vn[2] * Fn[2];
    double vDvn = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) vDvn += vn[i] * D[i][j] * vn[j];
    vDvn /= c * c;
    double k = chat * tdt;
    double Q_old = k * ((chiP * aT4 - chiE * E) * (g - 1.0) + (2.0 * chiE - chiF) * vF / (c * c) +
                        (order2 ? (chiF - chiE) * (beta2 + vDv) * E : 0.0));
    double Q_new = k * ((chiP * aT4 - chiE * E) * (gn - 1.0) + (2.0 * chiE - chiF) * vFn / (c * c) +
                        (order2 ? (chiF - chiE) * (beta2n + vDvn) * E : 0.0));
    double Q_scale =
        k * (fabs((chiP * aT4 - chiE * E) * (gn - 1.0)) +
             fabs(2.0 * chiE - chiF) *
                 (fabs(vn[0] * Fn[0]) + fabs(vn[1] * Fn[1]) + fabs(vn[2] * Fn[2])) / (c * c) +
             (order2 ? fabs(chiF - chiE) * (beta2n + fabs(vDvn)) * E : 0.0));

    for (int i = 0; i < 3; ++i) {
      F[i] = Fn[i];
      m[i] = mn[i];
    }
    double dQ = fabs(Q_new - Q_old);
    if (dQ <= p->outer_rtol * fabs(Q_old) || dQ <= p->outer_rtol * fabs(R) ||
        dQ <= p->outer_rtol * Q_scale) {
      y[0] = Eg;
      y[1] = m[0];
      y[2] = m[1];
      y[3] = m[2];
      y[4] = E;
      y[5] = F[0];
      y[6] = F[1];
      y[7] = F[2];
      if (!(E > 0.0) || !isfinite(E) || !isfinite(F[0]) || !isfinite(F[1]) ||
          !isfinite(F[2]))
        return ORC_ERR_NONPHYSICAL;
      return ORC_OK;
    }
  }
  return ORC_ERR_OUTER;
}

/* ---------------------------------------------------------- the IMEX step */

static void record(orc_info* info, int st, long long cell) {
  if (info && st != ORC_OK && info->status == ORC_OK) {
    info->status = st;
    info->fail_cell = cell;
  }
}

/* Implicit part of one stage over all cells: U holds the explicit state on
 * input and the solution on output. */
static int implicit_all(const orc_params* p, double* U, double theta, double dt,
                        orc_info* info) {
  const long long N = ncell_of(p);
  for (long long i = 0; i < N; ++i) {
    double rho = U[ORC_RHO * N + i];
    double chi = U[ORC_KAPPA * N + i] * rho;
    /* y order: Egas, m, E, F */
    double yy[8] = {U[ORC_EGAS * N + i], U[ORC_MX * N + i], U[ORC_MY * N + i],
                    U[ORC_MZ * N + i],   U[ORC_ERAD * N + i], U[ORC_FX * N + i],
                    U[ORC_FY * N + i],   U[ORC_FZ * N + i]};
    int nn = 0, no = 0;
    int st = orc_local_solve(p, theta, dt, rho, chi, yy, &nn, &no);
    if (info) {
      if (nn > info->max_newton) info->max_newton = nn;
      if (no > info->max_outer) info->max_outer = no;
      info->sum_newton += nn;
      info->n_solves += 1;
    }
    if (st != ORC_OK) {
      record(info, st, i);
      return st;
    }
    U[ORC_EGAS * N + i] = yy[0];
    U[ORC_MX * N + i] = yy[1];
    U[ORC_MY * N + i] = yy[2];
    U[ORC_MZ * N + i] = yy[3];
    U[ORC_ERAD * N + i] = yy[4];
    U[ORC_FX * N + i] = yy[5];
    U[ORC_FY * N + i] = yy[6];
    U[ORC_FZ * N + i] = yy[7];
  }
  return ORC_OK;
}

static const int RAD_FIELD[4] = {ORC_ERAD, ORC_FX, ORC_FY, ORC_FZ};

/* eq. (imex1) and (imex2) with epsilon = 0 in the PD-ARS tableau:
 *   y(n+1/2) = y(n) + dt s(y(n)) + dt f(y(n+1/2))
 *   y(n+1)   = y(n) + dt [s(y(n)) + s(y(n+1/2))]/2
 *                   + dt [f(y(n+1/2)) + f(y(n+1))]/2
 * The stage-1 relation fixes dt f(y(n+1/2)) = y(n+1/2) - y*, y* the explicit
 * state of stage 1; stage 2 uses it as such.  On failure U is left at y(n).
 * RK2-SSP (Sec. 4.2, the comparison scheme):
 *   y(n+1/2) = y(n) + dt s(y(n))
 *   y(n+1)   = y(n) + dt [s(y(n)) + s(y(n+1/2))]/2 + dt f(y(n+1)),
 * the same code with the first implicit stage skipped (y(n+1/2) = y*, so the
 * (y(n+1/2) - y*)/2 term vanishes) and theta = 1 in the second. */
int orc_step(const orc_params* p, double* U, double dt, orc_info* info) {
  const long long N = ncell_of(p);
  const size_t bytes = sizeof(double) * ORC_NFIELD * (size_t)N;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->fail_cell = -1;
  }
  if (dt <= 0.0) dt = orc_dt(p);

  double* Un = (double*)malloc(bytes);     /* y(n) */
  double* Uh = (double*)malloc(bytes);     /* y*, then y(n+1/2) */
  double* Ystar = (double*)malloc(bytes);  /* copy of y* */
  double* s0 = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  double* s1 = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  int st = ORC_OK;
  long long fc = -1;
  if (!Un || !Uh || !Ystar || !s0 || !s1) {
    st = ORC_ERR_ARG;
    goto done;
  }
  memcpy(Un, U, bytes);

  /* ---- stage 1: explicit s(y(n)), then implicit with theta = 1 ---- */
  st = orc_transport(p, Un, s0, &fc);
  if (st != ORC_OK) {
    record(info, st, fc);
    goto done;
  }
  memcpy(Uh, Un, bytes);
  for (int r = 0; r < 4; ++r)
    for (long long i = 0; i < N; ++i)
      Uh[RAD_FIELD[r] * N + i] = Un[RAD_FIELD[r] * N + i] + dt * s0[r * N + i];
  memcpy(Ystar, Uh, bytes);
  /* RK2-SSP (Sec. 4.2): no exchange in the first stage, y(n+1/2) = y* */
  if (p->scheme != ORC_SCHEME_RK2_SSP) {
    st = implicit_all(p, Uh, 1.0, dt, info);
    if (st != ORC_OK) goto done;
  }

  /* ---- stage 2: explicit part of eq. (imex2), then implicit, theta = 1/2 ---- */
  st = orc_transport(p, Uh, s1, &fc);
  if (st != ORC_OK) {
    record(info, st, fc);
    goto done;
  }
  {
    double* U2 = Ystar; /* reuse: becomes the stage-2 explicit state */
    /* evolved fields: y(n) + dt/2 [s(y(n)) + s(y(n+1/2))] + (1/2) dt f(y(n+1/2)) */
    static const int EVOLVED[8] = {ORC_EGAS, ORC_MX, ORC_MY, ORC_MZ,
                                   ORC_ERAD, ORC_FX, ORC_FY, ORC_FZ};
    for (int e = 0; e < 8; ++e) {
      int f = EVOLVED[e];
      int r = -1;
      for (int q = 0; q < 4; ++q)
        if (RAD_FIELD[q] == f) r = q;
      for (long long i = 0; i < N; ++i) {
        double yn = Un[f * N + i];
        double sn = (r >= 0) ? s0[r * N + i] : 0.0;
        double sh = (r >= 0) ? s1[r * N + i] : 0.0;
        double dtf_half = Uh[f * N + i] - U2[f * N + i]; /* y(n+1/2) - y* */
        U2[f * N + i] = yn + dt * (0.5 * sn + 0.5 * sh) + 0.5 * dtf_half;
      }
    }
    /* static fields stay those of y(n) */
    for (long long i = 0; i < N; ++i) {
      U2[ORC_RHO * N + i] = Un[ORC_RHO * N + i];
      U2[ORC_KAPPA * N + i] = Un[ORC_KAPPA * N + i];
    }
    /* IMEX: (dt/2) f(y(n+1)) in eq. (imex2); RK2-SSP: dt f(y(n+1)) */
    st = implicit_all(p, U2, p->scheme == ORC_SCHEME_RK2_SSP ? 1.0 : 0.5, dt, info);
    if (st != ORC_OK) goto done;
    memcpy(U, U2, bytes);
  }

done:
  free(Un);
  free(Uh);
  free(Ystar);
  free(s0);
  free(s1);
  return st;
}

/* ---------------------------------------------------------- the totals */

/* Sec. 3.3: with the energy closure the scheme conserves Egas + (c/chat) E,
 * and with the momentum update m + F/(c chat), cell by cell up to rounding. */
void orc_totals(const orc_params* p, const double* U, double out[4]) {
  const long long N = ncell_of(p);
  double V = 1.0;
  for (int d = 0; d < p->ndim; ++d) V *= p->dx[d];
  for (int q = 0; q < 4; ++q) out[q] = 0.0;
  for (long long i = 0; i < N; ++i) {
    out[0] += (U[ORC_EGAS * N + i] + (p->c / p->chat) * U[ORC_ERAD * N + i]) * V;
    out[1] += (U[ORC_MX * N + i] + U[ORC_FX * N + i] / (p->c * p->chat)) * V;
    out[2] += (U[ORC_MY * N + i] + U[ORC_FY * N + i] / (p->c * p->chat)) * V;
    out[3] += (U[ORC_MZ * N + i] + U[ORC_FZ * N + i] / (p->c * p->chat)) * V;
  }
}

/* the reconstruction as the hydrodynamic subsystem (rhd_oracle_hydro.c)
 * uses it */
double orc_recon_mc_slope(double um, double u0, double up) { return mc_slope(um, u0, up); }

void orc_recon_ppm_edges(const double u[5], double* aL, double* aR) { ppm_edges(u, aL, aR); }

void orc_recon_ppm_cs_edges(const double u[5], double* aL, double* aR) {
  ppm_cs_edges(u, aL, aR);
}
