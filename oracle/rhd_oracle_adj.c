/*
 * rhd_oracle_adj.c -- serial FP64 CPU oracle of the adjoint (reverse-mode
 * derivative) of one IMEX PD-ARS step.
 *
 * TEST INFRASTRUCTURE ONLY, like rhd_oracle.c: the tests and the benchmark
 * are its only users.
 *
 * One step (Sec. 3.2, eq. imex1 / imex2) is
 *   y*  = y(n) + dt s(y(n))                       explicit stage 1
 *   yh  = LS_1(y*)                                implicit stage 1, theta = 1
 *   y** = y(n) + dt/2 [s(y(n)) + s(yh)] + (yh - y*)/2     explicit stage 2
 *   y1  = LS_1/2(y**)                             implicit stage 2, theta = 1/2
 * Given dL/dy1 the adjoint returns dL/dy(n) and adds dL/dkappa.
 *
 * Transport s: the derivative of each HLL face flux with respect to its
 * 4-cell stencil, taken on the active branch of every limiter, max and clip
 * (Sec. 3.3 Godunov step, Sec. 4.3 wave speeds and optical-depth factor).
 *
 * Local solve LS: the implicit-function theorem on the converged state.  At
 * the solution of eq. (egupdate)-(fupdate) (grey, F from eq. numF2/numF1 with
 * P from the final E and F) the 8 unknowns satisfy, with m eliminated by the
 * momentum update m = p - F/(c chat), p = m(t) + F(t)/(c chat):
 *   r_G = Egas - Egas(t) + (c/chat) R
 *   r_E = E - E(t) - R
 *   r_F = F (1 + k g) - F(t) - k (a T^4 v + v.P)
 *   R   = k [(a T^4 - E) g + v.F/c^2],  k = chat chi theta dt,
 *   v = m/rho, g = 1 + beta^2/2 (order 2) or 1, T = (Egas - |m|^2/2rho)/C_v,
 * so dL/dinputs = -(dr/dinputs)^T lambda with (dr/dx)^T lambda = dL/dx,
 * x = (Egas, E, F).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "rhd_oracle.h"

static long long ncell_of(const orc_params* p) { return p->n[0] * p->n[1] * p->n[2]; }

/* ----------------------------------------------------- transport, forward */

/* half of the MC-limited slope and its derivatives (dum, du0, dup) */
static double half_slope_d(double um, double u0, double up, double g[3]) {
  double dm = u0 - um, dp = up - u0;
  g[0] = g[1] = g[2] = 0.0;
  int s = (dm > 0.0 && dp > 0.0) ? 1 : ((dm < 0.0 && dp < 0.0) ? -1 : 0);
  if (!s) return 0.0;
  double m = fmin(fmin(fabs(dm), fabs(dp)), 0.25 * fabs(dm + dp));
  if (m == fabs(dm)) {
    g[0] = -1.0; g[1] = 1.0;
  } else if (m == fabs(dp)) {
    g[1] = -1.0; g[2] = 1.0;
  } else {
    g[0] = -0.25; g[2] = 0.25;
  }
  return s * m;
}

/* M1 coefficients P = ha I + hb F F^T (F = flux / c, |F| clipped to E) and
 * their partial derivatives with respect to E and F2 = |F|^2. */
static void m1_coeffs_d(const orc_params* p, double E, const double F[3], double* ha,
                        double* hb, double d[4]) {
  if (p->closure == ORC_CLOSURE_EDDINGTON) {
    *ha = E / 3.0;
    *hb = 0.0;
    d[0] = 1.0 / 3.0; d[1] = 0.0; d[2] = 0.0; d[3] = 0.0;
    return;
  }
  double F2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
  double E2 = E * E;
  if (F2 > E2) {
    *ha = 0.0;
    *hb = E / F2;
    d[0] = 0.0; d[1] = 0.0; d[2] = 1.0 / F2; d[3] = -E / (F2 * F2);
    return;
  }
  double s = sqrt(4.0 * E2 - 3.0 * F2);
  *ha = (s - E) / 3.0;
  *hb = 3.0 / (2.0 * E + s);
  double dsE = 4.0 * E / s, dsF = -1.5 / s;
  d[0] = (dsE - 1.0) / 3.0;
  d[1] = dsF / 3.0;
  d[2] = -(*hb) * (*hb) / 3.0 * (2.0 + dsE);
  d[3] = -(*hb) * (*hb) / 3.0 * dsF;
}

typedef struct {
  double E, F[3], Fin[3];
  int resc;
  double ha, hb, dh[4], P[3];
} face_state;

static void state_prepare(const orc_params* p, int d, double E, const double Fin[3],
                          face_state* st) {
  st->E = E;
  for (int j = 0; j < 3; ++j) st->Fin[j] = st->F[j] = Fin[j];
  double n2 = Fin[0] * Fin[0] + Fin[1] * Fin[1] + Fin[2] * Fin[2];
  st->resc = n2 > E * E;
  if (st->resc) {
    double n = sqrt(n2);
    for (int j = 0; j < 3; ++j) st->F[j] = Fin[j] * E / n;
  }
  m1_coeffs_d(p, E, st->F, &st->ha, &st->hb, st->dh);
  for (int j = 0; j < 3; ++j) st->P[j] = st->hb * st->F[d] * st->F[j];
  st->P[d] += st->ha;
}

/* Face flux (E, F/c units) through the face between a and b along d and, if
 * obar != NULL, its reverse sweep: g[k][q] += d(obar . flux)/d cell_k[q] for
 * the stencil (am, a, b, bp) and *geps += d/d eps.  Cells hold (E, F/c). */
static int face_vjp(const orc_params* p, int d, const double* cell[4], double eps,
                    double out[4], const double* obar, double g[4][4], double* geps) {
  const double chat = p->chat;
  double L[4], R[4], gl[4][3], gr[4][3];
  for (int q = 0; q < 4; ++q) {
    L[q] = cell[1][q] + half_slope_d(cell[0][q], cell[1][q], cell[2][q], gl[q]);
    R[q] = cell[2][q] - half_slope_d(cell[1][q], cell[2][q], cell[3][q], gr[q]);
  }
  if (!(L[0] > 0.0) || !(R[0] > 0.0)) return ORC_ERR_NONPHYSICAL;
  face_state sl, sr;
  state_prepare(p, d, L[0], &L[1], &sl);
  state_prepare(p, d, R[0], &R[1], &sr);
  double num = sl.P[d], den = sl.E;
  int side = 0;
  if (sr.P[d] * sl.E > sl.P[d] * sr.E) {
    num = sr.P[d]; den = sr.E; side = 1;
  }
  if (3.0 * num < den) {
    num = 1.0; den = 3.0; side = -1;
  }
  double S = chat * sqrt(num / den);
  double hc = 0.5 * chat, hS = 0.5 * S;
  out[0] = hc * (sl.F[d] + sr.F[d]) - eps * hS * (sr.E - sl.E);
  for (int j = 0; j < 3; ++j) out[1 + j] = hc * (sl.P[j] + sr.P[j]) - hS * (sr.F[j] - sl.F[j]);
  if (!obar) return ORC_OK;

  /* ---- reverse sweep ---- */
  double gEL = eps * hS * obar[0], gER = -eps * hS * obar[0];
  double gFL[3] = {0, 0, 0}, gFR[3] = {0, 0, 0}, gPL[3] = {0, 0, 0}, gPR[3] = {0, 0, 0};
  gFL[d] += hc * obar[0];
  gFR[d] += hc * obar[0];
  *geps += -hS * (sr.E - sl.E) * obar[0];
  double ghS = -eps * (sr.E - sl.E) * obar[0];
  for (int j = 0; j < 3; ++j) {
    gPL[j] += hc * obar[1 + j];
    gPR[j] += hc * obar[1 + j];
    gFR[j] += -hS * obar[1 + j];
    gFL[j] += hS * obar[1 + j];
    ghS += -(sr.F[j] - sl.F[j]) * obar[1 + j];
  }
  double gS = 0.5 * ghS;
  if (side >= 0) {
    double x = num / den, gx = gS * chat * 0.5 / sqrt(x);
    double gnum = gx / den, gden = -gx * num / (den * den);
    if (side == 0) {
      gPL[d] += gnum; gEL += gden;
    } else {
      gPR[d] += gnum; gER += gden;
    }
  }
  face_state* sts[2] = {&sl, &sr};
  double* gPs[2] = {gPL, gPR};
  double* gEs[2] = {&gEL, &gER};
  double* gFs[2] = {gFL, gFR};
  for (int side2 = 0; side2 < 2; ++side2) {
    face_state* st = sts[side2];
    double* gP = gPs[side2];
    double* gF = gFs[side2];
    double gPF = gP[0] * st->F[0] + gP[1] * st->F[1] + gP[2] * st->F[2];
    double gha = gP[d];
    double ghb = st->F[d] * gPF;
    for (int j = 0; j < 3; ++j) gF[j] += st->hb * st->F[d] * gP[j];
    gF[d] += st->hb * gPF;
    *gEs[side2] += gha * st->dh[0] + ghb * st->dh[2];
    double gF2 = gha * st->dh[1] + ghb * st->dh[3];
    for (int j = 0; j < 3; ++j) gF[j] += 2.0 * gF2 * st->F[j];
    if (st->resc) {
      double n2 = st->Fin[0] * st->Fin[0] + st->Fin[1] * st->Fin[1] + st->Fin[2] * st->Fin[2];
      double n = sqrt(n2);
      double fg = st->Fin[0] * gF[0] + st->Fin[1] * gF[1] + st->Fin[2] * gF[2];
      *gEs[side2] += fg / n;
      for (int j = 0; j < 3; ++j) gF[j] = (st->E / n) * (gF[j] - st->Fin[j] * fg / n2);
    }
  }
  double gLq[4] = {gEL, gFL[0], gFL[1], gFL[2]};
  double gRq[4] = {gER, gFR[0], gFR[1], gFR[2]};
  for (int q = 0; q < 4; ++q) {
    g[1][q] += gLq[q];
    g[0][q] += gLq[q] * gl[q][0];
    g[1][q] += gLq[q] * gl[q][1];
    g[2][q] += gLq[q] * gl[q][2];
    g[2][q] += gRq[q];
    g[1][q] -= gRq[q] * gr[q][0];
    g[2][q] -= gRq[q] * gr[q][1];
    g[3][q] -= gRq[q] * gr[q][2];
  }
  return ORC_OK;
}

/* d/dtau of the optical-depth factor (1 - exp(-tau))/tau,
 * (tau exp(-tau) - (1 - exp(-tau)))/tau^2.  For small tau the two terms of
 * the numerator cancel; there the Taylor series of the derivative,
 * sum over k >= 1 of (-1)^k k tau^(k-1) / (k+1)!, is summed to k = 8. */
static double tau_factor_d(double tau) {
  if (tau < 0.05) {
    double s = 0.0, term_fact = 2.0; /* (k+1)! */
    double tpow = 1.0;               /* tau^(k-1) */
    for (int k = 1; k <= 8; ++k) {
      s += ((k & 1) ? -1.0 : 1.0) * k * tpow / term_fact;
      tpow *= tau;
      term_fact *= (double)(k + 2);
    }
    return s;
  }
  double e = exp(-tau);
  return (tau * e + expm1(-tau)) / (tau * tau);
}

/* stencil cell at offset o from (i0,i1,i2) along d with the boundary fold */
static long long fold_cell(const orc_params* p, const long long ic[3], int d, int o,
                           int* flip) {
  long long q[3] = {ic[0], ic[1], ic[2]};
  long long nd = p->n[d], x = q[d] + o;
  *flip = 0;
  if (x < 0) {
    if (p->bc[d][0] == ORC_BC_PERIODIC) x = ((x % nd) + nd) % nd;
    else { x = -1 - x; *flip = 1; }
  } else if (x >= nd) {
    if (p->bc[d][1] == ORC_BC_PERIODIC) x = x % nd;
    else { x = 2 * nd - 1 - x; *flip = 1; }
  }
  q[d] = x;
  return q[0] + p->n[0] * (q[1] + p->n[1] * q[2]);
}

/* Adjoint of rate = s(y) accumulated through y_target += alpha * rate:
 * given ybar_target (slot order Egas, m, E, F), add d/d y_state to ybar_state
 * (E and F slots) and dL/dkappa to kbar.  Y: slot-major state (8 x N) whose
 * transport is taken; rho, kappa: static fields. */
static int transport_adjoint(const orc_params* p, const double* Y, const double* rho,
                             const double* kappa, double alpha, const double* ybar_target,
                             double* ybar_state, double* kbar) {
  const long long N = ncell_of(p);
  const double c = p->c;
  for (int d = 0; d < p->ndim; ++d) {
    for (long long i2 = 0; i2 < p->n[2]; ++i2)
      for (long long i1 = 0; i1 < p->n[1]; ++i1)
        for (long long i0 = 0; i0 < p->n[0]; ++i0) {
          long long ic[3] = {i0, i1, i2};
          long long b = i0 + p->n[0] * (i1 + p->n[1] * i2);
          /* the face on the low side of cell b: between b-1 and b */
          long long idx[4];
          int flip[4];
          for (int o = -2; o <= 1; ++o) idx[o + 2] = fold_cell(p, ic, d, o, &flip[o + 2]);
          int wall = (ic[d] == 0 && p->bc[d][0] != ORC_BC_PERIODIC);
          double cells[4][4];
          const double* cp[4];
          for (int k = 0; k < 4; ++k) {
            cells[k][0] = Y[4 * N + idx[k]];
            for (int j = 0; j < 3; ++j) cells[k][1 + j] = Y[(5 + j) * N + idx[k]] / c;
            if (flip[k]) cells[k][1 + d] = -cells[k][1 + d];
            cp[k] = cells[k];
          }
          double eps = 1.0, tau = 0.0;
          if (p->hll_mode == ORC_HLL_TAU) {
            tau = 0.5 * (kappa[idx[1]] * rho[idx[1]] + kappa[idx[2]] * rho[idx[2]]) * p->dx[d];
            if (tau > 0.0) eps = -expm1(-tau) / tau;
          }
          /* flux adjoint: rate_a -= Phi/dx, rate_b += Phi/dx; rate of F/c */
          double obar[4];
          for (int q = 0; q < 4; ++q) {
            int slot = q == 0 ? 4 : 4 + q;
            double sc = alpha * (q == 0 ? 1.0 : c) / p->dx[d];
            double ub = ybar_target[slot * N + b] * sc;
            double ua = wall ? 0.0 : ybar_target[slot * N + idx[1]] * sc;
            obar[q] = ub - ua;
          }
          double out[4], g[4][4] = {{0}}, geps = 0.0;
          if (face_vjp(p, d, cp, eps, out, obar, g, &geps) != ORC_OK) return ORC_ERR_NONPHYSICAL;
          for (int k = 0; k < 4; ++k) {
            ybar_state[4 * N + idx[k]] += g[k][0];
            for (int j = 0; j < 3; ++j) {
              double gj = g[k][1 + j] / c;
              if (flip[k] && j == d) gj = -gj;
              ybar_state[(5 + j) * N + idx[k]] += gj;
            }
          }
          if (p->hll_mode == ORC_HLL_TAU && kbar) {
            double dtau = geps * tau_factor_d(tau) * 0.5 * p->dx[d];
            kbar[idx[1]] += dtau * rho[idx[1]];
            kbar[idx[2]] += dtau * rho[idx[2]];
          }
          /* the top wall face (cell b = n-1, between b and ghost n) */
          if (ic[d] == p->n[d] - 1 && p->bc[d][1] != ORC_BC_PERIODIC) {
            long long jdx[4];
            int jflip[4];
            for (int o = -1; o <= 2; ++o) jdx[o + 1] = fold_cell(p, ic, d, o, &jflip[o + 1]);
            double cj[4][4];
            const double* cjp[4];
            for (int k = 0; k < 4; ++k) {
              cj[k][0] = Y[4 * N + jdx[k]];
              for (int j = 0; j < 3; ++j) cj[k][1 + j] = Y[(5 + j) * N + jdx[k]] / c;
              if (jflip[k]) cj[k][1 + d] = -cj[k][1 + d];
              cjp[k] = cj[k];
            }
            double eps2 = 1.0, tau2 = 0.0;
            if (p->hll_mode == ORC_HLL_TAU) {
              tau2 = 0.5 * (kappa[jdx[1]] * rho[jdx[1]] + kappa[jdx[2]] * rho[jdx[2]]) * p->dx[d];
              if (tau2 > 0.0) eps2 = -expm1(-tau2) / tau2;
            }
            double ob2[4];
            for (int q = 0; q < 4; ++q) {
              int slot = q == 0 ? 4 : 4 + q;
              double sc = alpha * (q == 0 ? 1.0 : c) / p->dx[d];
              ob2[q] = -ybar_target[slot * N + b] * sc; /* only cell b's rate */
            }
            double o2[4], g2[4][4] = {{0}}, geps2 = 0.0;
            if (face_vjp(p, d, cjp, eps2, o2, ob2, g2, &geps2) != ORC_OK)
              return ORC_ERR_NONPHYSICAL;
            for (int k = 0; k < 4; ++k) {
              ybar_state[4 * N + jdx[k]] += g2[k][0];
              for (int j = 0; j < 3; ++j) {
                double gj = g2[k][1 + j] / c;
                if (jflip[k] && j == d) gj = -gj;
                ybar_state[(5 + j) * N + jdx[k]] += gj;
              }
            }
            if (p->hll_mode == ORC_HLL_TAU && kbar) {
              double dtau = geps2 * tau_factor_d(tau2) * 0.5 * p->dx[d];
              kbar[jdx[1]] += dtau * rho[jdx[1]];
              kbar[jdx[2]] += dtau * rho[jdx[2]];
            }
          }
        }
  }
  return ORC_OK;
}

/* --------------------------------------------------- local solve adjoint */

/* 5 x 9 Jacobian of (r_G, r_E, r_F) with respect to
 * (Egas, E, F1, F2, F3, p1, p2, p3, chi) at the converged state y. */
static void ls_jacobian(const orc_params* p, double tdt, double rho, double chi,
                        const double y[8], double J[5][9]) {
  const double c = p->c, chat = p->chat, a = p->a_rad, cc = c * chat, cr = c / chat;
  const double Cv = rho * p->kB_over_mu / (p->gamma - 1.0);
  const int order2 = p->vc_order == 2;
  double Eg = y[0], E = y[4];
  double m[3] = {y[1], y[2], y[3]}, F[3] = {y[5], y[6], y[7]};
  double v[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
  double Ek = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
  double T = (Eg - Ek) / Cv, B = a * T * T * T * T, dB = 4.0 * a * T * T * T;
  double b2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / (c * c);
  double g = order2 ? 1.0 + 0.5 * b2 : 1.0;
  double w = (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]) / (c * c);
  double k = chat * chi * tdt, dk = chat * tdt;
  double Ft[3] = {F[0] / c, F[1] / c, F[2] / c};
  double ha, hb, dh[4];
  m1_coeffs_d(p, E, Ft, &ha, &hb, dh);
  double vFt = v[0] * Ft[0] + v[1] * Ft[1] + v[2] * Ft[2];
  double vP[3];
  for (int i = 0; i < 3; ++i) vP[i] = ha * v[i] + hb * vFt * Ft[i];
  for (int col = 0; col < 9; ++col) {
    double dEg = col == 0, dE = col == 1, dchi = col == 8;
    double dF[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
    if (col >= 2 && col <= 4) {
      dF[col - 2] = 1.0;
      dm[col - 2] = -1.0 / cc;
    }
    if (col >= 5 && col <= 7) dm[col - 5] = 1.0;
    double dv[3] = {dm[0] / rho, dm[1] / rho, dm[2] / rho};
    double dEk = (m[0] * dm[0] + m[1] * dm[1] + m[2] * dm[2]) / rho;
    double dT = (dEg - dEk) / Cv, dBv = dB * dT;
    double dg = order2 ? (v[0] * dv[0] + v[1] * dv[1] + v[2] * dv[2]) / (c * c) : 0.0;
    double dw = (dv[0] * F[0] + dv[1] * F[1] + dv[2] * F[2] + v[0] * dF[0] + v[1] * dF[1] +
                 v[2] * dF[2]) / (c * c);
    double dkk = dk * dchi;
    double dR = dkk * ((B - E) * g + w) + k * ((dBv - dE) * g + (B - E) * dg + dw);
    J[0][col] = dEg + cr * dR;
    J[1][col] = dE - dR;
    double dFt[3] = {dF[0] / c, dF[1] / c, dF[2] / c};
    double dF2 = 2.0 * (Ft[0] * dFt[0] + Ft[1] * dFt[1] + Ft[2] * dFt[2]);
    double dha = dh[0] * dE + dh[1] * dF2, dhb = dh[2] * dE + dh[3] * dF2;
    double dvFt = dv[0] * Ft[0] + dv[1] * Ft[1] + dv[2] * Ft[2] + v[0] * dFt[0] +
                  v[1] * dFt[1] + v[2] * dFt[2];
    for (int i = 0; i < 3; ++i) {
      double dvP = dha * v[i] + ha * dv[i] + dhb * vFt * Ft[i] + hb * dvFt * Ft[i] +
                   hb * vFt * dFt[i];
      J[2 + i][col] = dF[i] * (1.0 + k * g) + F[i] * (dkk * g + k * dg) -
                      dkk * (B * v[i] + vP[i]) - k * (dBv * v[i] + B * dv[i] + dvP);
    }
  }
}

/* solve A^T x = b for a 5 x 5 A (Gaussian elimination, partial pivoting) */
static int solve5_transposed(double A[5][9], const double b[5], double x[5]) {
  double M[5][6];
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j < 5; ++j) M[i][j] = A[j][i];
    M[i][5] = b[i];
  }
  for (int col = 0; col < 5; ++col) {
    int piv = col;
    for (int r = col + 1; r < 5; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return 1;
    if (piv != col)
      for (int j = 0; j < 6; ++j) {
        double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t;
      }
    for (int r = col + 1; r < 5; ++r) {
      double f = M[r][col] / M[col][col];
      for (int j = col; j < 6; ++j) M[r][j] -= f * M[col][j];
    }
  }
  for (int i = 4; i >= 0; --i) {
    double s = M[i][5];
    for (int j = i + 1; j < 5; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  return 0;
}

/* Adjoint of one local solve: yin -> yout (both Egas, m, E, F).  Given
 * ybar_out, writes ybar_in and returns dL/dchi. */
int orc_local_solve_adjoint(const orc_params* p, double theta, double dt, double rho,
                            double chi, const double yout[8], const double ybar_out[8],
                            double ybar_in[8], double* chibar) {
  const double cc = p->c * p->chat;
  double J[5][9];
  ls_jacobian(p, theta * dt, rho, chi, yout, J);
  double xbar[5] = {ybar_out[0], ybar_out[4], ybar_out[5] - ybar_out[1] / cc,
                    ybar_out[6] - ybar_out[2] / cc, ybar_out[7] - ybar_out[3] / cc};
  double lam[5];
  if (solve5_transposed(J, xbar, lam)) return ORC_ERR_NEWTON;
  double pbar[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int r = 0; r < 5; ++r) s += J[r][5 + i] * lam[r];
    pbar[i] = ybar_out[1 + i] - s;
  }
  ybar_in[0] = lam[0];
  ybar_in[4] = lam[1];
  for (int i = 0; i < 3; ++i) {
    ybar_in[5 + i] = lam[2 + i] + pbar[i] / cc;
    ybar_in[1 + i] = pbar[i];
  }
  double s = 0.0;
  for (int r = 0; r < 5; ++r) s += J[r][8] * lam[r];
  *chibar = -s;
  return ORC_OK;
}

/* ----------------------------------------------------------- step tape */

static const int SLOT_FIELD[8] = {ORC_EGAS, ORC_MX, ORC_MY, ORC_MZ,
                                  ORC_ERAD, ORC_FX, ORC_FY, ORC_FZ};

/* One step, as orc_step, that also records the tape the adjoint needs: three
 * states of 8 x N doubles (slot-major, slots Egas, mx, my, mz, E, Fx, Fy, Fz):
 * y(n), yh = y(n+1/2) and y1 = y(n+1).  U is advanced in place. */
int orc_step_tape(const orc_params* p, double* U, double dt, double* tape) {
  const long long N = ncell_of(p);
  for (int s = 0; s < 8; ++s)
    memcpy(tape + (size_t)s * N, U + SLOT_FIELD[s] * N, sizeof(double) * N);
  /* y(n+1/2) is the stage-1 result: one step with the stage-2 work skipped
   * would need another entry point, so run stage 1 here by hand. */
  double* rate = (double*)malloc(sizeof(double) * 4 * (size_t)N);
  if (!rate) return ORC_ERR_ARG;
  if (dt <= 0.0) dt = orc_dt(p);
  long long fc;
  int st = orc_transport(p, U, rate, &fc);
  for (long long i = 0; i < N && st == ORC_OK; ++i) {
    double rho = U[ORC_RHO * N + i], chi = U[ORC_KAPPA * N + i] * rho, y[8];
    for (int s = 0; s < 8; ++s) y[s] = U[SLOT_FIELD[s] * N + i];
    y[4] += dt * rate[i];
    for (int j = 0; j < 3; ++j) y[5 + j] += dt * rate[(1 + j) * N + i];
    int nn, no;
    st = orc_local_solve(p, 1.0, dt, rho, chi, y, &nn, &no);
    for (int s = 0; s < 8; ++s) tape[((size_t)8 + s) * N + i] = y[s];
  }
  free(rate);
  if (st != ORC_OK) return st;
  orc_info info;
  st = orc_step(p, U, dt, &info);
  if (st != ORC_OK) return st;
  for (int s = 0; s < 8; ++s)
    memcpy(tape + ((size_t)16 + s) * N, U + SLOT_FIELD[s] * N, sizeof(double) * N);
  return ORC_OK;
}

/* Adjoint of one step from its tape.  ybar1 = dL/dy(n+1) (8 x N, slots as the
 * tape) gives ybar0 = dL/dy(n); dL/dkappa is added to kbar (N).  rho, kappa:
 * the static fields.  With y2 = (y(n) + yh)/2 + (dt/2) s(yh) the explicit
 * state of stage 2 written without y* (the two are equal algebraically):
 *   ybar2   = LS_(1/2)^T ybar1
 *   ybar_h  = ybar2 / 2 + (dt/2) s'(yh)^T ybar2
 *   ybar_s  = LS_1^T ybar_h                       (ybar_s = dL/dy*)
 *   ybar(n) = ybar2 / 2 + ybar_s + dt s'(y(n))^T ybar_s
 */
int orc_step_adjoint(const orc_params* p, const double* rho, const double* kappa,
                     const double* tape, double dt, const double* ybar1, double* ybar0,
                     double* kbar) {
  const long long N = ncell_of(p);
  if (dt <= 0.0) dt = orc_dt(p);
  double* q = (double*)calloc(8 * (size_t)N, sizeof(double));
  double* gh = (double*)calloc(8 * (size_t)N, sizeof(double));
  if (!q || !gh) {
    free(q);
    free(gh);
    return ORC_ERR_ARG;
  }
  const double* Yn = tape;
  const double* Yh = tape + (size_t)8 * N;
  const double* Y1 = tape + (size_t)16 * N;
  int st = ORC_OK;
  /* implicit stage 2 */
  for (long long i = 0; i < N && st == ORC_OK; ++i) {
    double y[8], b[8], bin[8], cb;
    for (int s = 0; s < 8; ++s) {
      y[s] = Y1[s * N + i];
      b[s] = ybar1[s * N + i];
    }
    st = orc_local_solve_adjoint(p, 0.5, dt, rho[i], kappa[i] * rho[i], y, b, bin, &cb);
    for (int s = 0; s < 8; ++s) q[s * N + i] = bin[s];
    kbar[i] += cb * rho[i];
  }
  for (long long j = 0; j < 8 * N; ++j) {
    gh[j] = 0.5 * q[j];
    ybar0[j] = 0.5 * q[j];
  }
  if (st == ORC_OK) st = transport_adjoint(p, Yh, rho, kappa, 0.5 * dt, q, gh, kbar);
  /* implicit stage 1 */
  for (long long i = 0; i < N && st == ORC_OK; ++i) {
    double y[8], b[8], bin[8], cb;
    for (int s = 0; s < 8; ++s) {
      y[s] = Yh[s * N + i];
      b[s] = gh[s * N + i];
    }
    st = orc_local_solve_adjoint(p, 1.0, dt, rho[i], kappa[i] * rho[i], y, b, bin, &cb);
    for (int s = 0; s < 8; ++s) q[s * N + i] = bin[s];
    kbar[i] += cb * rho[i];
  }
  for (long long j = 0; j < 8 * N; ++j) ybar0[j] += q[j];
  if (st == ORC_OK) st = transport_adjoint(p, Yn, rho, kappa, dt, q, ybar0, kbar);
  free(q);
  free(gh);
  return st;
}
