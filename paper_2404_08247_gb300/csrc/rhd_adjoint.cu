// rhd_adjoint.cu -- reverse-mode derivative of the IMEX PD-ARS step.
//
// One step (Sec. 3.2, eq. imex1/imex2, epsilon = 0) written with the stage-2
// explicit state y2 = (y(n) + yh)/2 + (dt/2) s(yh), which equals eq. (imex2)'s
// explicit part because dt f(yh) = yh - y*:
//   y*  = y(n) + dt s(y(n)),  yh = LS_1(y*),  y2 = ...,  y1 = LS_(1/2)(y2).
// Given ybar1 = dL/dy1 the adjoint is
//   q    = LS_(1/2)^T ybar1                                  (kernel A)
//   gh   = q/2 + (dt/2) s'(yh)^T q                           (faces B, cell C)
//   q'   = LS_1^T gh,   ybar(n) = q/2 + q' + dt s'(y(n))^T q'  (cell C, faces D, gather)
// LS^T is the implicit-function theorem on the converged local solve
// (Sec. 3.3, eq. egupdate-fupdate): with x = (Egas, E, F) and the momentum
// eliminated by m = p - F/(c chat), p = m(t) + F(t)/(c chat), the solution
// satisfies r(x; Egas(t), E(t), F(t), p, chi) = 0 with
//   r_G = Egas - Egas(t) + (c/chat) R,  r_E = E - E(t) - R,
//   r_F = F (1 + k g) - F(t) - k (a T^4 v + v.P),  R = k [(a T^4 - E) g + v.F/c^2],
// k = chat chi theta dt, so (dr/dx)^T lambda = xbar gives every input cotangent.
// s'^T is the transpose of the PLM/HLL transport (Sec. 3.3 Godunov step, Sec.
// 4.3 speeds and optical-depth factor) on the active branch of every limiter,
// max and clip.  It is done per face: kernel B/D differentiates each face flux
// once and writes its 16 stencil partials (and the two opacity partials of its
// optical-depth factor) to scratch; the next per-cell kernel gathers the four
// faces per axis that touch its cell.  No atomics: every sum has a fixed order.
#include "rhd_adjoint.cuh"

namespace rhd {

// ------------------------------------------------------------ face partials

// Face grid of axis d: n[d] faces per line (periodic; face n == face 0) or
// n[d] + 1 (reflecting; faces 0..n, face 0 and face n on the walls).  Face f
// lies between cells f-1 and f of its line.
__host__ __device__ inline int faces_along(const Geometry& g, int d) {
  return g.n[d] + (g.bc[d][0] != RHD_BC_PERIODIC ? 1 : 0);
}

__host__ __device__ inline long long face_count(const Geometry& g, int d) {
  return (long long)g.ncell / g.n[d] * faces_along(g, d);
}

__device__ __forceinline__ long long face_index(const Geometry& g, int d, int x, int y, int z) {
  int n0 = d == 0 ? faces_along(g, 0) : g.n[0];
  int n1 = d == 1 ? faces_along(g, 1) : g.n[1];
  return x + (long long)n0 * (y + (long long)n1 * z);
}

// Half PLM slope (monotonised-central limiter) and its gradient with respect to
// (u_-, u_0, u_+) on the active branch; zero at an extremum.  Signs and the
// minimum are taken on the integer pipe, as in the forward half_slope.
__device__ __forceinline__ double half_slope_vjp(double um, double u0, double up, double& gm,
                                                 double& g0, double& gp) {
  double dm = u0 - um, dp = up - u0;
  double q = 0.25 * (dm + dp);
  long long bm = dbits(dm), bp = dbits(dp);
  long long am = bm & kMag, ap = bp & kMag, aq = abs_bits(q);
  gm = g0 = gp = 0.0;
  if (!(((bm ^ bp) >= 0) & (am != 0) & (ap != 0))) return 0.0;
  long long m = min(min(am, ap), aq);
  // the selected candidate, as a signed linear form in (um, u0, up)
  if (m == am) {
    gm = -1.0; g0 = 1.0;
  } else if (m == ap) {
    g0 = -1.0; gp = 1.0;
  } else {
    gm = -0.25; gp = 0.25;
  }
  return __longlong_as_double(m | (bm & ~kMag));
}

// One face state after the free-streaming rescale, with the closure
// coefficients P = ha I + hb Ft Ft^T and their partials in (E, |Ft|^2).
struct FaceState {
  double E, F[3];
  double Fin[3], n2;  // the reconstructed flux before the rescale
  bool resc;
  double ha, hb, ha_E, ha_F2, hb_E, hb_F2;
  double P[3];  // row d of P
};

__device__ __forceinline__ void face_state(int d, int closure, double E, const double Fin[3],
                                           FaceState& s) {
  s.E = E;
  s.n2 = Fin[0] * Fin[0] + Fin[1] * Fin[1] + Fin[2] * Fin[2];
  s.resc = lt_nn(E * E, s.n2);
  double sc = s.resc ? E * rsqrt_pos(s.n2) : 1.0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    s.Fin[j] = Fin[j];
    s.F[j] = Fin[j] * sc;
  }
  if (closure == RHD_CLOSURE_EDDINGTON) {
    s.ha = E * (1.0 / 3.0);
    s.hb = 0.0;
    s.ha_E = 1.0 / 3.0;
    s.ha_F2 = s.hb_E = s.hb_F2 = 0.0;
  } else {
    double F2 = s.F[0] * s.F[0] + s.F[1] * s.F[1] + s.F[2] * s.F[2];
    if (lt_nn(E * E, F2)) {  // only through rounding of the rescale
      double iF2 = rcp_pos(F2);
      s.ha = 0.0;
      s.hb = E * iF2;
      s.ha_E = s.ha_F2 = 0.0;
      s.hb_E = iF2;
      s.hb_F2 = -E * iF2 * iF2;
    } else {
      // s = sqrt(4E^2 - 3F2), ha = (s - E)/3, hb = 3/(2E + s)
      double x = 4.0 * E * E - 3.0 * F2;
      double ir = rsqrt_pos(x);
      double r = x * ir;
      s.ha = (r - E) * (1.0 / 3.0);
      s.hb = 3.0 * rcp_pos(2.0 * E + r);
      double r_E = 4.0 * E * ir, r_F2 = -1.5 * ir;
      s.ha_E = (r_E - 1.0) * (1.0 / 3.0);
      s.ha_F2 = r_F2 * (1.0 / 3.0);
      double hb2 = s.hb * s.hb * (1.0 / 3.0);
      s.hb_E = -hb2 * (2.0 + r_E);
      s.hb_F2 = -hb2 * r_F2;
    }
  }
  double t = s.hb * s.F[d];
#pragma unroll
  for (int j = 0; j < 3; ++j) s.P[j] = t * s.F[j];
  s.P[d] += s.ha;
}

// Reverse of face_state: (gE, gF) hold the cotangents of E and of the rescaled
// Ft on entry (gP that of row d of P); on exit (gE, gF) are those of E and of
// the reconstructed Ft.
__device__ __forceinline__ void face_state_vjp(int d, const FaceState& s, const double gP[3],
                                               double& gE, double gF[3]) {
  double gPF = gP[0] * s.F[0] + gP[1] * s.F[1] + gP[2] * s.F[2];
  double gha = gP[d];
  double ghb = s.F[d] * gPF;
#pragma unroll
  for (int j = 0; j < 3; ++j) gF[j] += s.hb * s.F[d] * gP[j];
  gF[d] += s.hb * gPF;
  gE += gha * s.ha_E + ghb * s.hb_E;
  double gF2 = 2.0 * (gha * s.ha_F2 + ghb * s.hb_F2);
#pragma unroll
  for (int j = 0; j < 3; ++j) gF[j] += gF2 * s.F[j];
  if (s.resc) {
    // F = Fin E / |Fin|
    double in = rsqrt_pos(s.n2);
    double fg = s.Fin[0] * gF[0] + s.Fin[1] * gF[1] + s.Fin[2] * gF[2];
    gE += fg * in;
    double a = s.E * in, b = fg * in * in;
#pragma unroll
    for (int j = 0; j < 3; ++j) gF[j] = a * (gF[j] - s.Fin[j] * b);
  }
}

// d/dtau of the optical-depth factor (1 - exp(-tau))/tau.  Below tau = 0.05 the
// closed form cancels; there its Taylor series sum_k (-1)^k k tau^(k-1)/(k+1)!
// is used through tau^5 (truncation < 1e-14 relative).
__device__ __forceinline__ double tau_factor_deriv(double tau) {
  if (tau < 0.05) {
    return -0.5 + tau * (1.0 / 3.0 + tau * (-0.125 + tau * (1.0 / 30.0 +
           tau * (-1.0 / 144.0 + tau * (1.0 / 840.0 - tau * (1.0 / 5760.0))))));
  }
  double e = exp(-tau);
  return (e * (1.0 + tau) - 1.0) / (tau * tau);
}

struct FaceArgs {
  Geometry g;
  Physics ph;
  const double* rho;
  const double* kappa;
  const double* y[4];    // state whose transport is differentiated: E, Fx, Fy, Fz
  const double* cot[4];  // cotangent of the stage target: E, Fx, Fy, Fz
  double alpha;          // the stage weight of s (dt or dt/2)
  double* fp;            // face partials, FP_SLOTS per face, slot-major per axis
  long long off[3];      // start of axis d in fp
  long long nface[3];
  long long total;
};

// The face along axis D (a template parameter, so that every index into the
// per-axis arrays below is a compile-time constant and stays in registers).
template <int D>
__device__ __forceinline__ void face_vjp(const FaceArgs& A, long long fidx) {
  constexpr int d = D;
  const Geometry& g = A.g;
  int nf = faces_along(g, d);
  int fc[3];
  {
    int n0 = d == 0 ? nf : g.n[0];
    int n1 = d == 1 ? nf : g.n[1];
    fc[0] = (int)(fidx % n0);
    long long r = fidx / n0;
    fc[1] = (int)(r % n1);
    fc[2] = (int)(r / n1);
  }
  const int f = fc[d];
  const double inv_c = A.ph.inv_c;
  // stencil cells f-2, f-1 | f, f+1 along d (folded), as (E, Ft)
  double u[4][4];
  int idx[4];
  bool ghost[4];
  const int base = fc[0] * g.stride[0] + fc[1] * g.stride[1] + fc[2] * g.stride[2] -
                   f * g.stride[d];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    bool flip;
    int x = fold(f + p - 2, g.n[d], g.bc[d][0], g.bc[d][1], flip);
    idx[p] = base + x * g.stride[d];
    ghost[p] = (f + p - 2 < 0 || f + p - 2 >= g.n[d]) && flip;
    u[p][0] = __ldg(A.y[0] + idx[p]);
#pragma unroll
    for (int j = 0; j < 3; ++j) u[p][1 + j] = __ldg(A.y[1 + j] + idx[p]) * inv_c;
    if (flip) u[p][1 + d] = -u[p][1 + d];
  }
  // face cotangent: the face flux enters rate(b) with +1/dx and rate(a) with
  // -1/dx; rates of F are c times those of Ft; ghost cells carry no rate
  double ob[4];
  {
    double s = A.alpha * g.inv_dx[d];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double ub = ghost[2] ? 0.0 : __ldg(A.cot[q] + idx[2]);
      double ua = ghost[1] ? 0.0 : __ldg(A.cot[q] + idx[1]);
      ob[q] = (ub - ua) * s * (q == 0 ? 1.0 : A.ph.c);
    }
  }
  // ---- forward: reconstruction, closure, speeds ----
  double L[4], R[4], gl[4][3], gr[4][3];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    L[q] = u[1][q] + half_slope_vjp(u[0][q], u[1][q], u[2][q], gl[q][0], gl[q][1], gl[q][2]);
    R[q] = u[2][q] - half_slope_vjp(u[1][q], u[2][q], u[3][q], gr[q][0], gr[q][1], gr[q][2]);
  }
  FaceState sl, sr;
  face_state(d, A.ph.closure, L[0], &L[1], sl);
  face_state(d, A.ph.closure, R[0], &R[1], sr);
  double num = sl.P[d], den = sl.E;
  int side = 0;
  if (lt_nn(sl.P[d] * sr.E, sr.P[d] * sl.E)) {
    num = sr.P[d];
    den = sr.E;
    side = 1;
  }
  if (lt_nn(3.0 * num, den)) side = -1;
  const double chat = A.ph.chat;
  // S = chat sqrt(num/den) = chat num / sqrt(num den)
  double rq = side < 0 ? 0.0 : rsqrt_pos(num * den);
  double S = side < 0 ? chat * sqrt(1.0 / 3.0) : chat * num * rq;
  double eps = 1.0, tau = 0.0;
  bool tau_mode = A.ph.hll_mode == RHD_HLL_TAU;
  if (tau_mode) {
    tau = 0.5 * (__ldg(A.kappa + idx[1]) * __ldg(A.rho + idx[1]) +
                 __ldg(A.kappa + idx[2]) * __ldg(A.rho + idx[2])) * g.dx[d];
    eps = tau_factor(tau);
  }
  // ---- reverse: HLL ----
  const double hc = 0.5 * chat, hS = 0.5 * S;
  double dE = sr.E - sl.E;
  double gEL = eps * hS * ob[0], gER = -gEL;
  double gFL[3] = {0.0, 0.0, 0.0}, gFR[3] = {0.0, 0.0, 0.0};
  double gPL[3], gPR[3];
  gFL[d] = hc * ob[0];
  gFR[d] = hc * ob[0];
  double geps = -hS * dE * ob[0];
  double ghS = -eps * dE * ob[0];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gPL[j] = hc * ob[1 + j];
    gPR[j] = hc * ob[1 + j];
    gFR[j] -= hS * ob[1 + j];
    gFL[j] += hS * ob[1 + j];
    ghS -= (sr.F[j] - sl.F[j]) * ob[1 + j];
  }
  if (side >= 0) {
    // S = chat sqrt(num/den): dS/d(num/den) = chat^2 / (2 S), 1/S = den rq / chat
    double gx = 0.25 * ghS * chat * den * rq;
    double iden = rcp_pos(den);
    double gnum = gx * iden, gden = -gx * num * iden * iden;
    if (side == 0) {
      gPL[d] += gnum;
      gEL += gden;
    } else {
      gPR[d] += gnum;
      gER += gden;
    }
  }
  face_state_vjp(d, sl, gPL, gEL, gFL);
  face_state_vjp(d, sr, gPR, gER, gFR);
  // ---- reverse: reconstruction ----
  double gq[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) gq[p][q] = 0.0;
  {
    double gLq[4] = {gEL, gFL[0], gFL[1], gFL[2]};
    double gRq[4] = {gER, gFR[0], gFR[1], gFR[2]};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      gq[0][q] += gLq[q] * gl[q][0];
      gq[1][q] += gLq[q] * (1.0 + gl[q][1]) - gRq[q] * gr[q][0];
      gq[2][q] += gLq[q] * gl[q][2] + gRq[q] * (1.0 - gr[q][1]);
      gq[3][q] -= gRq[q] * gr[q][2];
    }
  }
  // store: d/dE and d/dF (physical F: Ft = F/c), not yet mirrored
  double* out = A.fp + A.off[d] + fidx;
  const long long NF = A.nface[d];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    out[(4 * p) * NF] = gq[p][0];
#pragma unroll
    for (int j = 0; j < 3; ++j) out[(4 * p + 1 + j) * NF] = gq[p][1 + j] * inv_c;
  }
  double ka = 0.0, kb = 0.0;
  if (tau_mode) {
    // tau = (chi_a + chi_b) dx/2, chi = kappa rho
    double gt = geps * tau_factor_deriv(tau) * 0.5 * g.dx[d];
    ka = gt * __ldg(A.rho + idx[1]);
    kb = gt * __ldg(A.rho + idx[2]);
  }
  out[16 * NF] = ka;
  out[17 * NF] = kb;
}

__global__ void __launch_bounds__(256) face_vjp_kernel(const FaceArgs A) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.total) return;
  int d = 0;
  while (d + 1 < A.g.ndim && t >= A.off[d + 1] / FP_SLOTS) ++d;
  long long fidx = t - A.off[d] / FP_SLOTS;
  if (d == 0) face_vjp<0>(A, fidx);
  else if (d == 1) face_vjp<1>(A, fidx);
  else face_vjp<2>(A, fidx);
}

// Sum of the face partials of axis d that belong to cell (c), with the mirror
// images of reflecting walls folded back: acc (E, Fx, Fy, Fz) and kacc.
__device__ __forceinline__ void gather_axis(const Geometry& g, const double* fp,
                                            const long long off[3], const long long nface[3],
                                            int d, const int c[3], double acc[4],
                                            double& kacc) {
  const int n = g.n[d];
  const bool refl = g.bc[d][0] != RHD_BC_PERIODIC;
  const double* F = fp + off[d];
  const long long NF = nface[d];
  int cc[3] = {c[0], c[1], c[2]};
  const int j = c[d];
  auto add = [&](int f, int p, bool flip) {
    cc[d] = f;
    long long fi = face_index(g, d, cc[0], cc[1], cc[2]);
    acc[0] += F[(4 * p) * NF + fi];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double v = F[(4 * p + 1 + q) * NF + fi];
      acc[1 + q] += (flip && q == d) ? -v : v;
    }
  };
  auto addk = [&](int f, int slot) {
    cc[d] = f;
    kacc += F[slot * NF + face_index(g, d, cc[0], cc[1], cc[2])];
  };
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int f = j + 2 - p;  // the face whose stencil position p is this cell
    if (!refl) {
      add((f + n) % n, p, false);
    } else {
      if (f >= 0 && f <= n) add(f, p, false);
      if (j <= 1 && 1 - j - p >= 0) add(1 - j - p, p, true);            // ghost -1-j
      if (j >= n - 2 && 2 * n + 1 - j - p <= n) add(2 * n + 1 - j - p, p, true);  // ghost 2n-1-j
    }
  }
  if (!refl) {
    addk(j, 17);
    addk((j + 1) % n, 16);
  } else {
    addk(j, 17);
    addk(j + 1, 16);
    if (j == 0) addk(0, 16);
    if (j == n - 1) addk(n, 17);
  }
}

// ---------------------------------------------------------- local solve

// Solve M x = b for a 5 x 5 M (row-major, destroyed) by Gaussian elimination
// with partial pivoting; rows are swapped with compile-time indices only.
__device__ __forceinline__ bool solve5(double M[5][5], double b[5]) {
  double ipiv[5];
#pragma unroll
  for (int col = 0; col < 5; ++col) {
    // pivot: the largest |M[r][col]|, r >= col, moved into row col
#pragma unroll
    for (int r = col + 1; r < 5; ++r) {
      if (abs_bits(M[col][col]) < abs_bits(M[r][col])) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          double t = M[col][k];
          M[col][k] = M[r][k];
          M[r][k] = t;
        }
        double t = b[col];
        b[col] = b[r];
        b[r] = t;
      }
    }
    const long long pb = dbits(M[col][col]);
    if ((pb & kMag) == 0 || (pb & kMag) >= kInfBits) return false;
    // 1/pivot with the pivot's sign
    const double inv = __longlong_as_double(
        dbits(rcp_pos(__longlong_as_double(pb & kMag))) | (pb & ~kMag));
    ipiv[col] = inv;
#pragma unroll
    for (int r = col + 1; r < 5; ++r) {
      double f = M[r][col] * inv;
#pragma unroll
      for (int k = col + 1; k < 5; ++k) M[r][k] -= f * M[col][k];
      b[r] -= f * b[col];
    }
  }
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    double s = b[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k) s -= M[i][k] * b[k];
    b[i] = s * ipiv[i];
  }
  return true;
}

// Adjoint of one converged local solve with output y (Egas, m, E, F) and
// stage weight theta (tdt = theta dt).  ybar: cotangent of the output; on exit
// yin: cotangent of the input state; chibar: dL/dchi.  Returns false if the
// Jacobian of the converged system is singular.
__device__ bool ls_adjoint(const Physics& ph, double tdt, double rho, double chi,
                           const double y[8], const double ybar[8], double yin[8],
                           double& chibar) {
  const double cr = ph.c_over_chat, icc = ph.inv_cchat, ic2 = ph.inv_c2;
  const double irho = rcp_pos(rho);
  const double Cv = rho * ph.cv_spec, iCv = rcp_pos(Cv);
  const bool o2 = ph.vc_order == 2;
  const double Eg = y[0], E = y[4];
  const double m[3] = {y[1], y[2], y[3]}, F[3] = {y[5], y[6], y[7]};
  double v[3], Ft[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = m[i] * irho;
    Ft[i] = F[i] * ph.inv_c;
  }
  const double Ek = 0.5 * (m[0] * v[0] + m[1] * v[1] + m[2] * v[2]);
  const double T = (Eg - Ek) * iCv;
  const double T3 = T * T * T;
  const double B = ph.a_rad * T3 * T, Bp = 4.0 * ph.a_rad * T3;
  const double b2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * ic2;
  const double g = o2 ? 1.0 + 0.5 * b2 : 1.0;
  const double w = (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]) * ic2;
  const double dk = ph.chat * tdt;  // dk/dchi
  const double k = dk * chi;
  // closure coefficients of P = ha I + hb Ft Ft^T and their partials
  double ha, hb, ha_E = 0.0, ha_F2 = 0.0, hb_E = 0.0, hb_F2 = 0.0;
  if (ph.closure == RHD_CLOSURE_EDDINGTON) {
    ha = E * (1.0 / 3.0);
    hb = 0.0;
    ha_E = 1.0 / 3.0;
  } else {
    double F2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2];
    if (lt_nn(E * E, F2)) {
      double iF2 = rcp_pos(F2);
      ha = 0.0;
      hb = E * iF2;
      hb_E = iF2;
      hb_F2 = -E * iF2 * iF2;
    } else {
      double x = 4.0 * E * E - 3.0 * F2;
      double ir = rsqrt_pos(x), r = x * ir;
      ha = (r - E) * (1.0 / 3.0);
      hb = 3.0 * rcp_pos(2.0 * E + r);
      double r_E = 4.0 * E * ir, r_F2 = -1.5 * ir;
      ha_E = (r_E - 1.0) * (1.0 / 3.0);
      ha_F2 = r_F2 * (1.0 / 3.0);
      double hb2 = hb * hb * (1.0 / 3.0);
      hb_E = -hb2 * (2.0 + r_E);
      hb_F2 = -hb2 * r_F2;
    }
  }
  const double vFt = v[0] * Ft[0] + v[1] * Ft[1] + v[2] * Ft[2];

  // R = k[(B - E) g + w] and its partials; m-partials are per unit of m
  const double R_Eg = k * g * Bp * iCv;
  const double R_E = -k * g;
  double R_F[3], R_m[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R_F[i] = k * v[i] * ic2;
    R_m[i] = k * irho * (-g * Bp * v[i] * rho * iCv + (o2 ? (B - E) * v[i] * ic2 : 0.0) +
                         F[i] * ic2);
  }
  const double R_chi = dk * ((B - E) * g + w);

  // Jacobian J[row][col]: rows (G, E, F1..3); cols (Egas, E, F1..3) with
  // m = p - F/(c chat) folded in, then (p1..3), then chi.
  double Jx[5][5], Jp[5][3], Jc[5];
  Jx[0][0] = 1.0 + cr * R_Eg;
  Jx[0][1] = cr * R_E;
  Jx[1][0] = -R_Eg;
  Jx[1][1] = 1.0 - R_E;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double RFt = R_F[j] - R_m[j] * icc;
    Jx[0][2 + j] = cr * RFt;
    Jx[1][2 + j] = -RFt;
    Jp[0][j] = cr * R_m[j];
    Jp[1][j] = -R_m[j];
  }
  Jc[0] = cr * R_chi;
  Jc[1] = -R_chi;
  // r_F,i = F_i (1 + k g) - F_i(t) - k S_i,  S_i = B v_i + ha v_i + hb (v.Ft) Ft_i
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double S_i = B * v[i] + ha * v[i] + hb * vFt * Ft[i];
    Jx[2 + i][0] = -k * Bp * iCv * v[i];
    Jx[2 + i][1] = -k * (ha_E * v[i] + hb_E * vFt * Ft[i]);
    Jc[2 + i] = dk * (F[i] * g - S_i);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double dij = i == j ? 1.0 : 0.0;
      // partial in F_j at fixed m
      double dS_F = ph.inv_c * (2.0 * Ft[j] * (ha_F2 * v[i] + hb_F2 * vFt * Ft[i]) +
                                hb * v[j] * Ft[i] + hb * vFt * dij);
      double pF = dij * (1.0 + k * g) - k * dS_F;
      // partial in m_j
      double dS_m = -Bp * iCv * v[i] * v[j] + (B * dij + ha * dij + hb * Ft[i] * Ft[j]) * irho;
      double pm = F[i] * k * (o2 ? v[j] * irho * ic2 : 0.0) - k * dS_m;
      Jx[2 + i][2 + j] = pF - pm * icc;
      Jp[2 + i][j] = pm;
    }
  }
  // (dr/dx)^T lambda = xbar,  xbar = (Egas, E, F - m/(c chat)) cotangents
  double M[5][5], lam[5];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int s = 0; s < 5; ++s) M[r][s] = Jx[s][r];
  lam[0] = ybar[0];
  lam[1] = ybar[4];
#pragma unroll
  for (int j = 0; j < 3; ++j) lam[2 + j] = ybar[5 + j] - ybar[1 + j] * icc;
  if (!solve5(M, lam)) return false;
  yin[0] = lam[0];
  yin[4] = lam[1];
  double cs = 0.0;
#pragma unroll
  for (int r = 0; r < 5; ++r) cs += Jc[r] * lam[r];
  chibar = -cs;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < 5; ++r) s += Jp[r][j] * lam[r];
    double pbar = ybar[1 + j] - s;
    yin[1 + j] = pbar;
    yin[5 + j] = lam[2 + j] + pbar * icc;
  }
  return true;
}

// ------------------------------------------------------------ cell kernels

struct CellArgs {
  Geometry g;
  Physics ph;
  double tdt;              // theta dt of the local solve (mode A, C)
  const double* rho;
  const double* kappa;
  const double* ys[NY];    // converged local-solve output (mode A: y1, C: yh)
  double* ybar[NY];        // the running adjoint dL/dy
  double* q[NY];           // stage cotangent scratch
  const double* fp;        // face partials to gather (null: none)
  long long off[3], nface[3];
  double* kbar;            // dL/dkappa (accumulated)
  DevStatus* st;
  int step;
};

// mode A: ybar += gather(fp); q = LS_(1/2)^T ybar                 (stage 2)
// mode C: gh = q/2 + gather(fp); q' = LS_1^T gh; ybar = q/2 + q'; q = q'  (stage 1)
// mode E: ybar += gather(fp)                                        (last)
template <int MODE>
__global__ void __launch_bounds__(256, 1) cell_adj_kernel(const CellArgs A) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const Geometry& g = A.g;
  if (i >= g.ncell) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0}, kacc = 0.0;
  if (A.fp) {
    int c[3];
    c[0] = i % g.n[0];
    int r = i / g.n[0];
    c[1] = r % g.n[1];
    c[2] = r / g.n[1];
    for (int d = 0; d < g.ndim; ++d) gather_axis(g, A.fp, A.off, A.nface, d, c, acc, kacc);
  }
  double kb = kacc;
  if (MODE == 2) {
    A.ybar[Y_ERAD][i] += acc[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) A.ybar[Y_FX + j][i] += acc[1 + j];
    A.kbar[i] += kb;
    return;
  }
  double cot[8];
  if (MODE == 0) {
#pragma unroll
    for (int s = 0; s < 8; ++s) cot[s] = A.ybar[s][i];
  } else {
#pragma unroll
    for (int s = 0; s < 8; ++s) cot[s] = 0.5 * A.q[s][i];
  }
  cot[Y_ERAD] += acc[0];
#pragma unroll
  for (int j = 0; j < 3; ++j) cot[Y_FX + j] += acc[1 + j];
  double y[8], yin[8], chibar = 0.0;
#pragma unroll
  for (int s = 0; s < 8; ++s) y[s] = __ldg(A.ys[s] + i);
  const double rho = __ldg(A.rho + i);
  const double chi = __ldg(A.kappa + i) * rho;
  bool ok = ls_adjoint(A.ph, A.tdt, rho, chi, y, cot, yin, chibar);
  if (!ok) {
    unsigned long long key = ((unsigned long long)i << 8) | (unsigned long long)RHD_ERR_NEWTON;
    unsigned long long old = atomicMin(&A.st->fail_key, key);
    if (key < old) {
      A.st->fail_step = A.step;
      A.st->fail_stage = MODE == 0 ? 2 : 1;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) yin[s] = 0.0;
    chibar = 0.0;
  }
  // the face terms first, then the solve's: the same order whether or not a
  // checkpoint boundary split the face terms off into the finishing gather
  double kv = A.kbar[i] + kb;
  A.kbar[i] = kv + chibar * rho;
  if (MODE == 0) {
#pragma unroll
    for (int s = 0; s < 8; ++s) A.q[s][i] = yin[s];
  } else {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      A.ybar[s][i] = 0.5 * A.q[s][i] + yin[s];
      A.q[s][i] = yin[s];
    }
  }
}

// ------------------------------------------------------------ launchers

long long adjoint_scratch_doubles(const Geometry& g) {
  long long s = 0;
  for (int d = 0; d < g.ndim; ++d) s += FP_SLOTS * face_count(g, d);
  return s;
}

static void face_layout(const Geometry& g, long long off[3], long long nface[3]) {
  long long o = 0;
  for (int d = 0; d < 3; ++d) {
    off[d] = o;
    nface[d] = d < g.ndim ? face_count(g, d) : 0;
    o += FP_SLOTS * nface[d];
  }
}

// One adjoint step: ybar holds dL/dy1 (plus, if pending_fp, the face partials
// of the previous adjoint step still to be gathered into it) and is left as
// the partial dL/dy(n) whose transport part is in fp (gathered by the next
// call with pending_fp = true, or by launch_adjoint_finish).
cudaError_t launch_adjoint_step(const AdjointStep& S, cudaStream_t s) {
  const Geometry& g = S.g;
  const int N = g.ncell;
  const int nb = (N + 255) / 256;
  CellArgs C;
  C.g = g;
  C.ph = S.ph;
  C.rho = S.rho;
  C.kappa = S.kappa;
  for (int q = 0; q < NY; ++q) {
    C.ybar[q] = S.ybar + (size_t)q * N;
    C.q[q] = S.q + (size_t)q * N;
  }
  face_layout(g, C.off, C.nface);
  C.kbar = S.kbar;
  C.st = S.st;
  C.step = S.step;

  FaceArgs F;
  F.g = g;
  F.ph = S.ph;
  F.rho = S.rho;
  F.kappa = S.kappa;
  F.fp = S.fp;
  face_layout(g, F.off, F.nface);
  F.total = 0;
  for (int d = 0; d < g.ndim; ++d) F.total += F.nface[d];
  const int fb = (int)((F.total + 255) / 256);

  // A: stage-2 local solve at y1
  C.tdt = 0.5 * S.dt;
  for (int q = 0; q < NY; ++q) C.ys[q] = S.y1 + (size_t)q * N;
  C.fp = S.pending_fp ? S.fp : nullptr;
  cell_adj_kernel<0><<<nb, 256, 0, s>>>(C);
  // B: transport at yh, weight dt/2, cotangent q
  for (int q = 0; q < 4; ++q) {
    F.y[q] = S.yh + (size_t)(Y_ERAD + q) * N;
    F.cot[q] = S.q + (size_t)(Y_ERAD + q) * N;
  }
  F.alpha = 0.5 * S.dt;
  face_vjp_kernel<<<fb, 256, 0, s>>>(F);
  // C: stage-1 local solve at yh
  C.tdt = S.dt;
  for (int q = 0; q < NY; ++q) C.ys[q] = S.yh + (size_t)q * N;
  C.fp = S.fp;
  cell_adj_kernel<1><<<nb, 256, 0, s>>>(C);
  // D: transport at y(n), weight dt, cotangent q'
  for (int q = 0; q < 4; ++q) F.y[q] = S.yn + (size_t)(Y_ERAD + q) * N;
  F.alpha = S.dt;
  face_vjp_kernel<<<fb, 256, 0, s>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(const AdjointStep& S, cudaStream_t s) {
  const Geometry& g = S.g;
  const int N = g.ncell;
  CellArgs C;
  C.g = g;
  C.ph = S.ph;
  C.tdt = 0.0;
  C.rho = S.rho;
  C.kappa = S.kappa;
  for (int q = 0; q < NY; ++q) {
    C.ys[q] = nullptr;
    C.ybar[q] = S.ybar + (size_t)q * N;
    C.q[q] = S.q + (size_t)q * N;
  }
  C.fp = S.fp;
  face_layout(g, C.off, C.nface);
  C.kbar = S.kbar;
  C.st = S.st;
  C.step = S.step;
  cell_adj_kernel<2><<<(N + 255) / 256, 256, 0, s>>>(C);
  return cudaGetLastError();
}

}  // namespace rhd
