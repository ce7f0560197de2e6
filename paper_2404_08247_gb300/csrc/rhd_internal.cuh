// rhd_internal.cuh -- device-side building blocks of the IMEX PD-ARS step.
//
// Internal to the library (csrc/*.cu).  Every routine cites the passage of
// He, Wibking & Krumholz (2024) it implements; readings of passages the paper
// leaves open are the library's documented choices (M1 closure, PLM with the
// monotonised-central limiter, symmetric HLL speeds floored at chat/sqrt(3),
// E_tot = Egas + (c/chat) E, energy closure E = E(t) - (chat/c) dEgas).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rhd.h"

namespace rhd {

// evolved-field slots of a state buffer (NY * ncell doubles, slot-major)
enum { Y_EGAS = 0, Y_MX, Y_MY, Y_MZ, Y_ERAD, Y_FX, Y_FY, Y_FZ, NY };

// Device status block: the first failing launch records its step, stage and
// the smallest failing cell; every later kernel of the batch sees the key and
// skips its work, so the last good ping-pong buffer is never overwritten.
struct DevStatus {
  unsigned long long fail_key;  // (cell << 8) | rhd_status, ~0ull if none
  int fail_step;
  int fail_stage;
  int max_newton;
  int max_outer;
  unsigned long long sum_newton;
  unsigned long long n_solves;
  unsigned long long sum_outer;
};

// Index checks of the bounds-checked build (-DRHD_BOUNDS_CHECK).  chk_index
// returns whether 0 <= i < n; an index outside records RHD_ERR_BOUNDS in the
// status block, with the index in place of the cell (its low 56 bits), and
// the caller skips the access (a load gives 0).  Nothing traps: the context
// stays usable and the step reports the status.  The default build compiles
// the plain accesses.
#ifdef RHD_BOUNDS_CHECK
__device__ __forceinline__ bool chk_index(DevStatus* st, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicMin(&st->fail_key, (((unsigned long long)i & 0x00ffffffffffffffull) << 8) | 8ull);
  return false;
}
#define RHD_LDG(st, p, i, n) (chk_index((st), (i), (n)) ? __ldg((p) + (i)) : 0.0)
#define RHD_LD(st, p, i, n) (chk_index((st), (i), (n)) ? (p)[i] : 0.0)
#define RHD_ST(st, p, i, n, v)                  \
  do {                                          \
    if (chk_index((st), (i), (n))) (p)[i] = (v); \
  } while (0)
#else
#define RHD_LDG(st, p, i, n) __ldg((p) + (i))
#define RHD_LD(st, p, i, n) ((p)[i])
#define RHD_ST(st, p, i, n, v) ((p)[i] = (v))
#endif

struct Geometry {
  int ndim;
  int n[3];
  int stride[3];
  int ncell;
  int bc[3][2];
  double dx[3];
  double inv_dx[3];
  double bc_state[3][2][4];  // ghost E, Fx, Fy, Fz of RHD_BC_INFLOW faces
};

struct Physics {
  double c, chat, a_rad;
  double cv_spec;       // kB_over_mu / (gamma - 1): C_v = rho cv_spec
  double inv_c;         // 1/c
  double c_over_chat;   // c/chat
  double chat_over_c;   // chat/c
  double inv_c2;        // 1/c^2
  double inv_cchat;     // 1/(c chat)
  int closure, vc_order, hll_mode;
  double newton_rtol, outer_rtol;
  int newton_max, outer_max;
  int scheme;              // rhd_scheme
  double kappa_T_exp;      // chi = kappa rho (T / T_ref)^kappa_T_exp
  double inv_kappa_T_ref;  // 1 / T_ref
  double kappa_P_ratio;    // chi_0P / chi_0E
  double kappa_F_ratio;    // chi_0F / chi_0E
  int reconstruction;      // rhd_recon
};

struct StageArgs {
  Geometry g;
  Physics ph;
  double dt;
  int step;            // step index within the batch (for the status block)
  const double* rho;
  const double* kappa;
  const double* yt[NY];  // state whose transport s(.) is taken, one pointer per slot
  const double* yn[NY];  // y(n) (stage 2 only)
  double* yo[NY];        // stage output
  const double* eps[3];  // TAU mode: per-face optical-depth factors, or null
                         // (then computed from kappa and rho on the fly)
  double* rate[4];       // transport-only launch: dE/dt, dFx/dt, dFy/dt, dFz/dt
  long long cell_base;   // added to cell indices in failure reports (batched pools)
  DevStatus* st;
  // RHD_BC_HALO z faces: the ghost planes the neighbouring slabs supplied,
  // per side [4 fields E, Fx, Fy, Fz][HALO_PLANES planes][n0 n1], planes in
  // z order (low side: z = -3..-1; high side: z = n2..n2+2); and the TAU
  // factors of the low slab face (n0 n1)
  const double* halo[2] = {nullptr, nullptr};
  const double* eps_zlo = nullptr;
  // tile rows skipped along the slowest axis (z in 3-D, y in 2-D, x in 1-D):
  // a launch over the rows [blk_off, blk_off + grid extent) of that axis
  int blk_off = 0;
  // stages 1 and 2: each cell's solve cost (outer passes and Newton updates,
  // packed in a byte) in this stage of the previous step, read to order the
  // local solves of a plane by cost and rewritten; null: solves in cell order
  unsigned char* cost = nullptr;
};

// ghost planes a HALO face holds (the widest face stencil: PPM's 3)
constexpr int HALO_PLANES = 3;

// slot pointers of a slot-major buffer of NY * n doubles
template <typename P>
inline void slots_of(P* out, P base, int n) {
  for (int q = 0; q < NY; ++q) out[q] = base + (size_t)q * n;
}

// ------------------------------------------------- FP64 off the FP64 pipe
// On this GPU the FP64 pipe, which limits the FP64 step, also executes double
// compares, minima and conversions (about one FMA slot each), and division
// and square root take about ten.  The helpers below give the same answers
// with the integer pipe doing what it can:
//  * non-negative, non-NaN doubles order like their IEEE bit patterns as
//    signed 64-bit integers, so their compares and minima are integer ops;
//  * rcp_pos / rsqrt_pos: 1/x and 1/sqrt(x) for x > 0 by Newton-Raphson
//    iteration (r <- r + r (1 - x r); y <- y + y (1/2 - x y^2 / 2), each step
//    doubling the correct bits; e.g. P. Markstein, IBM J. Res. Dev. 34 (1990))
//    from a single-precision seed whose exponent is rebiased with integer
//    arithmetic: two steps from a 2^-22 seed leave ~1 ulp (the IEEE operation
//    is used outside the single-precision exponent range).
constexpr long long kMag = 0x7fffffffffffffffll;
constexpr long long kInfBits = 0x7ff0000000000000ll;

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// x > 0 and finite (false for NaN)
__device__ __forceinline__ bool pos_finite(double x) {
  long long b = dbits(x);
  return b > 0 && b < kInfBits;
}
__device__ __forceinline__ bool finite_bits(double x) { return (dbits(x) & kMag) < kInfBits; }
// |x|, and a < b / a <= b / max(a, b) for a, b >= 0 (not NaN)
__device__ __forceinline__ long long abs_bits(double x) { return dbits(x) & kMag; }
__device__ __forceinline__ bool lt_nn(double a, double b) { return dbits(a) < dbits(b); }
__device__ __forceinline__ bool le_nn(double a, double b) { return dbits(a) <= dbits(b); }
__device__ __forceinline__ double max_nn(double a, double b) {
  return __longlong_as_double(max(dbits(a), dbits(b)));
}

__device__ __forceinline__ bool seed_range(double x) {
  int e = (int)(dbits(x) >> 52);  // biased exponent of x > 0
  return e > 1023 - 120 && e < 1023 + 120;
}
// x as a float with the mantissa truncated (x > 0 within seed_range)
__device__ __forceinline__ float seed_float(double x) {
  return __int_as_float((int)((dbits(x) >> 29) - (896ll << 23)));
}
// a positive normal float widened exactly
__device__ __forceinline__ double seed_double(float f) {
  return __longlong_as_double(((long long)__float_as_int(f) + (896ll << 23)) << 29);
}
__device__ __forceinline__ double rcp_pos(double x) {
  if (!seed_range(x)) return 1.0 / x;
  double r = seed_double(__fdividef(1.0f, seed_float(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double rsqrt_pos(double x) {
  if (!seed_range(x)) return 1.0 / sqrt(x);
  double y = seed_double(rsqrtf(seed_float(x)));
  double h = 0.5 * x;
  double e = fma(-h * y, y, 0.5);
  y = fma(y, e, y);
  e = fma(-h * y, y, 0.5);
  return fma(y, e, y);
}

// ---------------------------------------------------------------- limiter
// Half of the PLM slope with the monotonised-central limiter:
// (1/2) minmod(2 d-, (d- + d+)/2, 2 d+) = sgn * min(|d-|, |d+|, |d- + d+|/4),
// zero unless d- and d+ share a sign.  Face states are u -+ half_slope.
template <typename R>
__device__ __forceinline__ R half_slope(R um, R u0, R up) {
  R dm = u0 - um;
  R dp = up - u0;
  R m = fmin(fmin(fabs(dm), fabs(dp)), R(0.25) * fabs(dm + dp));
  return (dm > R(0) && dp > R(0)) ? m : ((dm < R(0) && dp < R(0)) ? -m : R(0));
}

// double: the same value with the sign tests and the minimum on the integer
// pipe (0.25 |d- + d+| = |0.25 (d- + d+)| exactly)
template <>
__device__ __forceinline__ double half_slope<double>(double um, double u0, double up) {
  double dm = u0 - um;
  double dp = up - u0;
  double q = 0.25 * (dm + dp);
  long long bm = dbits(dm), bp = dbits(dp);
  long long am = bm & kMag, ap = bp & kMag;
  long long m = min(min(am, ap), abs_bits(q));
  bool take = ((bm ^ bp) >= 0) & (am != 0) & (ap != 0);  // same sign, both nonzero
  return __longlong_as_double(take ? (m | (bm & ~kMag)) : 0ll);
}

// ---------------------------------------------------------------- PPM
// Piecewise parabolic face states (Colella & Woodward 1984, the paper's
// reconstruction in Sec. 3.3) written with half slopes h = dm/2 of the
// limiter above.  Interface value between cells u0 and up (their eq. 1.6 with
// the limited slopes of eq. 1.8): (u0 + up)/2 - (dm(up) - dm(u0))/6
// = (u0 + up)/2 - (h1 - h0)/3; it lies between u0 and up.
template <typename R>
__device__ __forceinline__ R ppm_interface(R u0, R up, R h0, R h1) {
  return R(0.5) * (u0 + up) - (h1 - h0) * R(1.0 / 3.0);
}

// Their monotonicity constraint (eq. 1.10) on the edge values (l, r) of a
// cell of mean u0.  With dl = u0 - l and dr = r - u0: at a local extremum
// (dl dr <= 0) the cell is flat; otherwise the parabola is monotone in the
// cell iff |dl| <= 2|dr| and |dr| <= 2|dl| (its two tests, dd m6 > dd^2 and
// -dd^2 > dd m6 with dd = dl + dr and m6 = 3 (dl - dr), divided through by
// dd), and an edge beyond that is moved onto it: |dl| <- min(|dl|, 2|dr|),
// |dr| <- min(|dr|, 2|dl|), signs kept.  The constraint is continuous where
// its branches meet, so a tie decided either way changes an edge by
// rounding only.  Returned: the constrained left edge (LEFT) or right edge.
template <bool LEFT, typename R>
__device__ __forceinline__ R ppm_edge(R u0, R l, R r) {
  const R dl = u0 - l, dr = r - u0;
  if (!(dl * dr > R(0))) return u0;
  const R a = LEFT ? dl : dr, b = LEFT ? dr : dl;  // the moved side, the other
  const R m = fmin(fabs(a), R(2) * fabs(b));
  return LEFT ? u0 - copysign(m, a) : u0 + copysign(m, a);
}

// double: the sign tests and minima on the integer pipe (non-negative doubles
// order as their bit patterns; 2|b| = |b + b| exactly)
template <bool LEFT>
__device__ __forceinline__ double ppm_edge_d(double u0, double l, double r) {
  const double dl = u0 - l, dr = r - u0;
  const double a = LEFT ? dl : dr, b = LEFT ? dr : dl;
  const long long ba = dbits(a), bb = dbits(b);
  const long long ma = ba & kMag, mb = bb & kMag;
  const bool mono = ((ba ^ bb) >= 0) & (ma != 0) & (mb != 0);
  const long long m = min(ma, abs_bits(b + b));
  const double s = __longlong_as_double(mono ? (m | (ba & ~kMag)) : 0ll);
  return LEFT ? u0 - s : u0 + s;
}

template <bool LEFT, typename R>
__device__ __forceinline__ R ppm_edge_of(R u0, R l, R r) {
  if constexpr (sizeof(R) == sizeof(double))
    return ppm_edge_d<LEFT>(u0, l, r);
  else
    return ppm_edge<LEFT>(u0, l, r);
}

// States of the face between u[2] and u[3] from cells u[0..5] (the face's
// three cells on each side): the constrained right edge of u[2] | the
// constrained left edge of u[3].
template <typename R>
__device__ __forceinline__ void ppm_face(const R u[6], R& L, R& Rr) {
  const R h1 = half_slope(u[0], u[1], u[2]), h2 = half_slope(u[1], u[2], u[3]);
  const R h3 = half_slope(u[2], u[3], u[4]), h4 = half_slope(u[3], u[4], u[5]);
  const R a12 = ppm_interface(u[1], u[2], h1, h2);
  const R a23 = ppm_interface(u[2], u[3], h2, h3);
  const R a34 = ppm_interface(u[3], u[4], h3, h4);
  L = ppm_edge_of<false>(u[2], a12, a23);
  Rr = ppm_edge_of<true>(u[3], a23, a34);
}

// The PPM limiter of Colella & Sekora (2008) (reconstruction PPM_CS), which
// keeps smooth extrema.  Interface value between cells u0 and up from
// um .. upp: the fourth-order value 7/12 (u0 + up) - 1/12 (um + upp); where it
// leaves [u0, up] its second difference 3 (u0 - 2a + up) is limited against
// those of the two cells (the smallest magnitude, C = 1.25 on its own, if all
// three share a sign, else zero) and a = (u0 + up)/2 - D2_lim/6.
template <typename R>
__device__ __forceinline__ bool same_sign3(R a, R b, R c) {
  return (a > R(0) && b > R(0) && c > R(0)) || (a < R(0) && b < R(0) && c < R(0));
}

template <typename R>
__device__ __forceinline__ R cs_interface(R um, R u0, R up, R upp) {
  R a = R(7.0 / 12.0) * (u0 + up) - R(1.0 / 12.0) * (um + upp);
  if ((a - u0) * (up - a) < R(0)) {
    const R d2 = R(3) * (u0 - R(2) * a + up);
    const R d2l = um - R(2) * u0 + up, d2r = u0 - R(2) * up + upp;
    R lim = R(0);
    if (same_sign3(d2, d2l, d2r))
      lim = copysign(fmin(R(1.25) * fabs(d2), fmin(fabs(d2l), fabs(d2r))), d2);
    a = R(0.5) * (u0 + up) - lim * R(1.0 / 6.0);
  }
  return a;
}

// Edges (l, r) of a cell of mean u0 with neighbours um, up under the
// Colella-Sekora constraint; d2L, d2R: second differences of the cells on
// either side.  At a local extremum (of the edges or of the means) the
// curvature -12 u0 + 6 (l + r) is limited against C = 1.25 times the second
// differences of the three cells and both edges scale towards u0 by the
// ratio; elsewhere an edge more than twice as far from u0 as the other is
// moved to twice that distance.
template <typename R>
__device__ __forceinline__ void cs_edges(R um, R u0, R up, R d2L, R d2R, R& l, R& r) {
  if ((r - u0) * (u0 - l) <= R(0) || (um - u0) * (u0 - up) <= R(0)) {
    const R d2 = R(-12) * u0 + R(6) * (l + r), d2c = um - R(2) * u0 + up;
    R lim = R(0);
    if (same_sign3(d2, d2c, d2L) && same_sign3(d2, d2c, d2R))
      lim = copysign(fmin(fabs(d2), R(1.25) * fmin(fabs(d2c), fmin(fabs(d2L), fabs(d2R)))),
                     d2);
    if (d2 != R(0)) {
      const R fac = lim / d2;
      l = u0 + (l - u0) * fac;
      r = u0 + (r - u0) * fac;
    } else {
      l = u0;
      r = u0;
    }
  } else {
    const R dl = u0 - l, dr = r - u0;
    if (fabs(dr) >= R(2) * fabs(dl))
      r = u0 + R(2) * dl;
    else if (fabs(dl) >= R(2) * fabs(dr))
      l = u0 - R(2) * dr;
  }
}

// Colella-Sekora states of the face between u[2] and u[3] from u[0..5]
template <typename R>
__device__ __forceinline__ void ppm_cs_face(const R u[6], R& L, R& Rr) {
  const R a12 = cs_interface(u[0], u[1], u[2], u[3]);
  const R a23 = cs_interface(u[1], u[2], u[3], u[4]);
  const R a34 = cs_interface(u[2], u[3], u[4], u[5]);
  R l2 = a12, r2 = a23, l3 = a23, r3 = a34;
  cs_edges(u[1], u[2], u[3], u[0] - R(2) * u[1] + u[2], u[2] - R(2) * u[3] + u[4], l2, r2);
  cs_edges(u[2], u[3], u[4], u[1] - R(2) * u[2] + u[3], u[3] - R(2) * u[4] + u[5], l3, r3);
  L = r2;
  Rr = l3;
}

// ---------------------------------------------------------------- closure
// Levermore M1 closure (the paper leaves the closure free, Sec. 2.1):
// P = E [(1 - xi)/2 I + (3 xi - 1)/2 n n], xi = (3 + 4 f^2)/(5 + 2 sqrt(4 - 3 f^2)),
// f = |Ft|/E clipped to [0, 1], Ft = F/c.  With s = sqrt(4 E^2 - 3 |Ft|^2)
// the same tensor is exactly
//     P = (s - E)/3 I + 3/(2E + s) Ft Ft^T          (|Ft| <= E),
// which needs one square root and one reciprocal and no division by |Ft|
// (zero flux gives E/3 I without a special case).  Above the free-streaming
// limit f is clipped to 1: P = E n n = (E/|Ft|^2) Ft Ft^T.  m1_coeffs returns
// (ha, hb) with P = ha I + hb Ft Ft^T; m1_row returns row d of P.
template <typename R>
__device__ __forceinline__ void m1_coeffs(R E, const R Ft[3], R& ha, R& hb) {
  R F2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2];
  R E2 = E * E;
  if (F2 > E2) {
    ha = R(0);
    hb = E / F2;
  } else {
    R s = sqrt(R(4) * E2 - R(3) * F2);
    ha = (s - E) * (R(1) / R(3));
    hb = R(3) / (R(2) * E + s);
  }
}

template <>
__device__ __forceinline__ void m1_coeffs<double>(double E, const double Ft[3], double& ha,
                                                  double& hb) {
  double F2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2];
  double E2 = E * E;
  if (lt_nn(E2, F2)) {
    ha = 0.0;
    hb = E * rcp_pos(F2);
  } else {
    double x = 4.0 * E2 - 3.0 * F2;
    double s = x * rsqrt_pos(x);
    ha = (s - E) * (1.0 / 3.0);
    hb = 3.0 * rcp_pos(2.0 * E + s);
  }
}

template <typename R>
__device__ __forceinline__ void m1_row(int d, R E, const R Ft[3], int closure, R P[3]) {
  if (closure == RHD_CLOSURE_EDDINGTON) {
    P[0] = P[1] = P[2] = R(0);
    P[d] = E * (R(1) / R(3));
    return;
  }
  R ha, hb;
  m1_coeffs(E, Ft, ha, hb);
  R t = hb * Ft[d];
#pragma unroll
  for (int j = 0; j < 3; ++j) P[j] = t * Ft[j];
  P[d] += ha;
}

// ------------------------------------------------------------------- HLL
// Flux through one face along axis d (Sec. 3.3 Godunov step, Sec. 4.3 wave
// speeds) for the RSLA system dE/dt = -chat div(Ft), dFt/dt = -chat div(P),
// from the reconstructed face states L and R (E, Ft).  Reconstructed fluxes
// above the free-streaming limit are scaled back onto |Ft| = E.  Symmetric
// speeds S_R = -S_L = chat sqrt(max(D_dd,L, D_dd,R, 1/3)), D = P/E, so HLL is
//   Phi = (Phi_L + Phi_R)/2 - S (U_R - U_L)/2,
// with the optical-depth factor eps on the energy part (1 for HLL NONE).
// Returns false for a face state with E <= 0 (or NaN).
// a > 0 and a < b for a, b >= 0 in the transport precision (integer pipe for
// double, plain compares for float)
template <typename R>
__device__ __forceinline__ bool positive(R a) {
  if constexpr (sizeof(R) == 8) return dbits(a) > 0 && dbits(a) < kInfBits;
  else return a > R(0);
}
template <typename R>
__device__ __forceinline__ bool less_nn(R a, R b) {
  if constexpr (sizeof(R) == 8) return lt_nn(a, b);
  else return a < b;
}

template <typename R>
__device__ __forceinline__ bool hll_states(int d, R L[4], R Rr[4], R eps, R chat,
                                           int closure, R out[4]) {
  if (!positive(L[0]) || !positive(Rr[0])) {
    out[0] = out[1] = out[2] = out[3] = R(0);
    return false;
  }
  {
    R n2 = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
    if (less_nn(L[0] * L[0], n2)) {
      R sc;
      if constexpr (sizeof(R) == 8) sc = L[0] * rsqrt_pos(n2);
      else sc = L[0] / sqrt(n2);
      L[1] *= sc; L[2] *= sc; L[3] *= sc;
    }
    n2 = Rr[1] * Rr[1] + Rr[2] * Rr[2] + Rr[3] * Rr[3];
    if (less_nn(Rr[0] * Rr[0], n2)) {
      R sc;
      if constexpr (sizeof(R) == 8) sc = Rr[0] * rsqrt_pos(n2);
      else sc = Rr[0] / sqrt(n2);
      Rr[1] *= sc; Rr[2] *= sc; Rr[3] *= sc;
    }
  }
  R PL[3], PR[3];
  m1_row(d, L[0], &L[1], closure, PL);
  m1_row(d, Rr[0], &Rr[1], closure, PR);
  // largest of D_dd,L, D_dd,R and 1/3 without dividing each (P_dd >= 0)
  R num = PL[d], den = L[0];
  if (less_nn(PL[d] * Rr[0], PR[d] * L[0])) { num = PR[d]; den = Rr[0]; }
  if (less_nn(R(3) * num, den)) { num = R(1); den = R(3); }
  R S;
  if constexpr (sizeof(R) == 8) S = chat * num * rsqrt_pos(num * den);  // sqrt(num/den)
  else S = chat * sqrt(num / den);
  R hc = R(0.5) * chat;
  R hS = R(0.5) * S;
  out[0] = hc * (L[1 + d] + Rr[1 + d]) - eps * hS * (Rr[0] - L[0]);
#pragma unroll
  for (int j = 0; j < 3; ++j) out[1 + j] = hc * (PL[j] + PR[j]) - hS * (Rr[1 + j] - L[1 + j]);
  return true;
}

// Mixed precision: row d of the deviation P - (E/3) I of the closure tensor,
// in single precision.  From the form above, P - (E/3) I =
// (3 Ft Ft^T - |Ft|^2 I)/(2E + s) below the free-streaming limit (E n n - E/3 I
// above it; zero for the Eddington closure).  It is O(|Ft|^2/E), so its
// single-precision rounding is small next to the flux, where a rounded P_dd
// ~ E/3 would carry an error of an ulp of E/3 into every face.
__device__ __forceinline__ void m1_dev_row(int d, float E, const float Ft[3], int closure,
                                           float D[3]) {
  D[0] = D[1] = D[2] = 0.f;
  if (closure == RHD_CLOSURE_EDDINGTON) return;
  const float F2 = Ft[0] * Ft[0] + Ft[1] * Ft[1] + Ft[2] * Ft[2];
  const float E2 = E * E;
  float hb, ha;
  if (F2 > E2) {
    hb = E / F2;
    ha = -E * (1.f / 3.f);
  } else {
    const float s = sqrtf(4.f * E2 - 3.f * F2);
    const float w = 1.f / (2.f * E + s);
    hb = 3.f * w;
    ha = -F2 * w;
  }
  const float t = hb * Ft[d];
#pragma unroll
  for (int j = 0; j < 3; ++j) D[j] = t * Ft[j];
  D[d] += ha;
}

// HLL flux of hll_states in mixed precision.  The isotropic part of the
// normal momentum flux, hc (E_L + E_R)/3 (hc = chat/2), is linear in the face
// states: it is returned in double (iso, from the exact single-precision face
// energies and chat6 = chat/6 in double) and left out of out[1 + d], which
// carries the single-precision rest.  The flux of F along d is out[1 + d] +
// iso.  Rounding P_dd in single precision at every face gives each face an
// independent error of an ulp of E/3, which the flux difference turns into
// an error of the flux update of order 1e-7 E/|Ft| relative; near isotropy
// (|Ft| << E) that is the dominant single-precision error.
__device__ __forceinline__ bool hll_states_mixed(int d, float L[4], float Rr[4], float eps,
                                                 float chat, int closure, double chat6,
                                                 float out[4], double& iso) {
  iso = 0.0;
  if (!(L[0] > 0.f) || !(Rr[0] > 0.f)) {
    out[0] = out[1] = out[2] = out[3] = 0.f;
    return false;
  }
  {
    float n2 = L[1] * L[1] + L[2] * L[2] + L[3] * L[3];
    if (L[0] * L[0] < n2) {
      const float sc = L[0] / sqrtf(n2);
      L[1] *= sc; L[2] *= sc; L[3] *= sc;
    }
    n2 = Rr[1] * Rr[1] + Rr[2] * Rr[2] + Rr[3] * Rr[3];
    if (Rr[0] * Rr[0] < n2) {
      const float sc = Rr[0] / sqrtf(n2);
      Rr[1] *= sc; Rr[2] *= sc; Rr[3] *= sc;
    }
  }
  float DL[3], DR[3];
  m1_dev_row(d, L[0], &L[1], closure, DL);
  m1_dev_row(d, Rr[0], &Rr[1], closure, DR);
  // D_dd = 1/3 + dev/E: the larger side and the 1/3 floor by the deviations
  float num = DL[d], den = L[0];
  if (DL[d] * Rr[0] < DR[d] * L[0]) { num = DR[d]; den = Rr[0]; }
  const float S = num > 0.f ? chat * sqrtf(1.f / 3.f + num / den) : chat * sqrtf(1.f / 3.f);
  const float hc = 0.5f * chat;
  const float hS = 0.5f * S;
  out[0] = hc * (L[1 + d] + Rr[1 + d]) - eps * hS * (Rr[0] - L[0]);
#pragma unroll
  for (int j = 0; j < 3; ++j) out[1 + j] = hc * (DL[j] + DR[j]) - hS * (Rr[1 + j] - L[1 + j]);
  iso = chat6 * ((double)L[0] + (double)Rr[0]);
  return true;
}

// The face flux in the transport precision R: hll_states for double (iso =
// 0, unused), hll_states_mixed for float.
template <typename R>
__device__ __forceinline__ bool face_hll(int d, R L[4], R Rr[4], R eps, R chat, int closure,
                                         double chat6, R out[4], double& iso) {
  if constexpr (sizeof(R) == 8) {
    iso = 0.0;
    return hll_states<R>(d, L, Rr, eps, chat, closure, out);
  } else {
    return hll_states_mixed(d, L, Rr, eps, chat, closure, chat6, out, iso);
  }
}

// Optical-depth factor of the HLL energy dissipation (reading of Sec. 4.3):
// (1 - exp(-tau))/tau, 1 in the thin limit, 1/tau in the thick limit.
__device__ __forceinline__ double tau_factor(double tau) {
  return tau > 0.0 ? -expm1(-tau) / tau : 1.0;
}

// ------------------------------------------------------------ local solve
// Start of the inner Newton iteration.  With v and F frozen, eq. (FGFR) and
// eq. (Rnew) reduce exactly to a quartic for the gas temperature:
//   A T^4 + C_v T = C,  A = (c/chat) k g a/(1 + k g),
//   C = Egas(t) - E_kin + (c/chat) k (g E(t) - v.F/c^2)/(1 + k g),
// whose positive root is the converged inner state.  quartic_start solves
// a4 T^4 + T = rhs (a4 = A/C_v, rhs = C/C_v) in single precision in the
// variable t = T/T(t) (alpha t^4 + beta t = 1, coefficients of order one) by
// Newton from the upper bound min(1/beta, alpha^-1/4), where the convex
// quartic converges monotonically.  The double-precision Newton of the paper
// then starts from it instead of from (Egas(t), 0) and needs fewer updates;
// it converges to the same root.  Returns false (cold start) if the
// single-precision numbers are not finite.
__device__ __forceinline__ bool quartic_start(double a4, double rhs, double T0, double& T) {
  float al = (float)(a4 * (T0 * T0) * (T0 * T0) / rhs);
  float be = (float)(T0 / rhs);
  if (!(al >= 0.f) || !(be > 0.f) || !isfinite(al) || !isfinite(be)) return false;
  float t = fminf(1.0f / be, al > 0.f ? rsqrtf(sqrtf(al)) : INFINITY);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    float t2 = t * t;
    float f = fmaf(al * t2, t2, fmaf(be, t, -1.0f));
    float fp = fmaf(4.0f * al * t2, t, be);
    t = t - __fdividef(f, fp);
  }
  if (!(t > 0.f) || !isfinite(t)) return false;
  T = (double)t * T0;
  return true;
}

// Implicit stage of one cell (Sec. 3.3), grey chi.  y = {Egas, m, E, F}
// holds the explicit state on entry and the solution on exit.  tdt = theta dt.
//
// Inner stage: Newton on (Egas, R) for eq. (FGFR) with eq. (Rnew) and the
// paper's Jacobian (beta^2 dropped).  The R-row is multiplied by
// k g (k = chat chi theta dt, g = 1 + beta^2/2), which leaves the Newton
// iterates unchanged and keeps the system regular for small k:
//   r0 = Egas - Egas(t) + (c/chat) R
//   r1 = k g F_R = k g (aT^4 - E(t) - R) + k v.F/c^2 - R
//   J  = [[1, c/chat], [g k 4 a T^3 / C_v, -g (1 + k)]]
// converged when |r0| < eps E_tot and (c/chat)|r1| <= eps E_tot k g,
// E_tot = Egas(t) + (c/chat) E(t).  The first pass starts from quartic_start
// (constant chi) or from (Egas(t), 0) (chi ~ T^p, whose J10 gains the term of
// the T-dependence of k).
// Energy closure: E = E(t) - (chat/c)(Egas - Egas(t)).
// Outer stage: eq. (numF2) (order 2) or (numF1) (order 1) for F with P from
// the new E and the previous outer flux, momentum m = m(t) - (F - F(t))/(c chat),
// repeated until Q = k[(g - 1)(aT^4 - E) + v.F/c^2] settles: its change is at
// most outer_rtol times |Q|, |R| or the magnitude of its terms.
// MIXED: the Newton step's reciprocal of the Jacobian determinant is taken in
// single precision (a step off by 1e-7 only slows the last iteration by that
// factor); residuals, the state, the closure of the exchange term v.P and
// every update stay double, so the solve meets the double-precision
// convergence tests (inner and outer) and conserves to rounding.
// GEN: compiled with the temperature-dependent opacity; the default physics
// (constant chi) uses the GEN = false copy, free of that branch.
template <bool MIXED, bool GEN>
__device__ __forceinline__ int local_solve(const Physics& ph, double tdt, double rho,
                                           double chi, double y[8], int& nn, int& no) {
  nn = 0;
  no = 0;
  if (chi == 0.0) return RHD_OK;
  const double Cv = rho * ph.cv_spec;
  const double inv_Cv = rcp_pos(Cv);
  const double inv_rho = rcp_pos(rho);
  const double cr = ph.c_over_chat;
  const double a = ph.a_rad;
  const double Eg0 = y[0], E0 = y[4];
  const double Etot = Eg0 + cr * E0;
  // k = chat chi theta dt; with a temperature-dependent opacity chi is taken
  // at the current Newton iterate (the paper's chi carry the superscript
  // (t+1)) and held fixed in the Jacobian
  const bool vary = GEN && ph.kappa_T_exp != 0.0;
  const double k0 = ph.chat * chi * tdt;
  double k = k0;
  const double tolG = ph.newton_rtol * Etot;
  double Eg = Eg0, R = 0.0, E = E0;
  double m[3] = {y[1], y[2], y[3]};
  double F[3] = {y[5], y[6], y[7]};

  // v, beta^2, g, v.F/c^2 and the kinetic energy of the frozen (m, F)
  double v[3] = {m[0] * inv_rho, m[1] * inv_rho, m[2] * inv_rho};
  double beta2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * ph.inv_c2;
  double g = (ph.vc_order == 2) ? 1.0 + 0.5 * beta2 : 1.0;
  double w = (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]) * ph.inv_c2;
  double Ekin = 0.5 * (m[0] * v[0] + m[1] * v[1] + m[2] * v[2]);

  // With a temperature-dependent opacity the iteration starts from
  // (Egas(t), 0) like the oracle's: the exact Jacobian below converges
  // quadratically from there, and a common start keeps the two solves on
  // the same iterates near a Marshak front, where the stopping point's
  // rounding is amplified.
  if (!vary) {
    double T0 = (Eg0 - Ekin) * inv_Cv;
    if (pos_finite(T0)) {
      double kg = k * g;
      double inv1 = rcp_pos(1.0 + kg);
      double a4 = cr * kg * a * inv1 * inv_Cv;
      double rhs = T0 + cr * k * (g * E0 - w) * inv1 * inv_Cv;
      double Tg;
      if (pos_finite(rhs) && quartic_start(a4, rhs, T0, Tg)) {
        Eg = Cv * Tg + Ekin;
        R = -ph.chat_over_c * (Eg - Eg0);
      }
    }
  }

  for (int outer = 0; outer < ph.outer_max; ++outer) {
    no = outer + 1;
    double kg = k * g;
    double kw = k * w;
    double c4 = 4.0 * kg * a * inv_Cv;  // J10 / T^3
    double gpk = g * (1.0 + k);
    double tolRg = tolG * k * g;

    bool conv = false;
    double aT4 = 0.0;
    for (int it = 0;; ++it) {
      double T = (Eg - Ekin) * inv_Cv;
      if (!pos_finite(T) || !finite_bits(R)) return RHD_ERR_NONPHYSICAL;
      if (vary) {
        k = k0 * pow(T * ph.inv_kappa_T_ref, ph.kappa_T_exp);
        kg = k * g;
        kw = k * w;
        c4 = 4.0 * kg * a * inv_Cv;
        gpk = g * (1.0 + k);
        tolRg = tolG * k * g;
      }
      double T2 = T * T;
      aT4 = a * T2 * T2;
      double r0 = (Eg - Eg0) + cr * R;
      double r1 = kg * (aT4 - E0 - R) + (kw - R);
      if (lt_nn(fabs(r0), tolG) && le_nn(cr * fabs(r1), tolRg)) {
        conv = true;
        break;
      }
      if (it >= ph.newton_max) break;
      double J10 = c4 * T2 * T;
      // chi ~ T^p: the R/(k g) term of E(Egas, R) varies with T through k,
      // which adds p R/(T C_v) to the scaled J10 (exact dE/dEgas; the
      // paper's J10 holds chi fixed, Sec. 3.3, and converges linearly)
      if (vary) J10 += ph.kappa_T_exp * R / (Eg - Ekin);
      double det = -gpk - cr * J10;  // < 0
      double inv_det = MIXED ? (double)(1.0f / (float)det) : -rcp_pos(-det);
      double dEg = (r0 * gpk + cr * r1) * inv_det;
      double dR = (r0 * J10 - r1) * inv_det;
      Eg += dEg;
      R += dR;
      ++nn;
    }
    if (!conv) return RHD_ERR_NEWTON;

    // energy closure; aT4 is that of the converged Egas
    E = E0 - ph.chat_over_c * (Eg - Eg0);

    // v_j P_ji of the closure at (E, F): P = ha I + hb Ft Ft^T
    double vP[3];
    {
      double Ft[3] = {F[0] * ph.inv_c, F[1] * ph.inv_c, F[2] * ph.inv_c};
      if (ph.closure == RHD_CLOSURE_EDDINGTON) {
        double e3 = E * (1.0 / 3.0);
        vP[0] = v[0] * e3; vP[1] = v[1] * e3; vP[2] = v[2] * e3;
      } else {
        double ha, hb;
        m1_coeffs(E, Ft, ha, hb);  // the cell flux may exceed the free-streaming limit
        double t = hb * (v[0] * Ft[0] + v[1] * Ft[1] + v[2] * Ft[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) vP[i] = ha * v[i] + t * Ft[i];
      }
    }
    double inv_den = rcp_pos(1.0 + kg);
    double Fn[3], mn[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Fn[i] = (y[5 + i] + k * (aT4 * v[i] + vP[i])) * inv_den;
      mn[i] = y[1 + i] - (Fn[i] - y[5 + i]) * ph.inv_cchat;
    }
    double Q_old = k * ((g - 1.0) * (aT4 - E) + w);
    // the updated v, beta^2, g, v.F/c^2: the next pass freezes these
    double vn[3] = {mn[0] * inv_rho, mn[1] * inv_rho, mn[2] * inv_rho};
    double beta2n = (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]) * ph.inv_c2;
    double gn = (ph.vc_order == 2) ? 1.0 + 0.5 * beta2n : 1.0;
    double wn = (vn[0] * Fn[0] + vn[1] * Fn[1] + vn[2] * Fn[2]) * ph.inv_c2;
    double Q_new = k * ((gn - 1.0) * (aT4 - E) + wn);
    // magnitude of the terms of Q: the rounding level of a cancelling v.F
    double Q_scale = k * (fabs((gn - 1.0) * (aT4 - E)) +
                          (fabs(vn[0] * Fn[0]) + fabs(vn[1] * Fn[1]) + fabs(vn[2] * Fn[2])) *
                              ph.inv_c2);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[i] = Fn[i];
      m[i] = mn[i];
      v[i] = vn[i];
    }
    g = gn;
    w = wn;
    Ekin = 0.5 * (m[0] * v[0] + m[1] * v[1] + m[2] * v[2]);
    // |dQ| <= rtol max(|Q_old|, |R|, Q_scale): the three tests of the outer stop
    double dQ = fabs(Q_new - Q_old);
    double big = max_nn(max_nn(fabs(Q_old), fabs(R)), Q_scale);
    if (le_nn(dQ, ph.outer_rtol * big)) {
      y[0] = Eg;
      y[1] = m[0]; y[2] = m[1]; y[3] = m[2];
      y[4] = E;
      y[5] = F[0]; y[6] = F[1]; y[7] = F[2];
      if (!pos_finite(E) || !finite_bits(F[0]) || !finite_bits(F[1]) || !finite_bits(F[2]))
        return RHD_ERR_NONPHYSICAL;
      return RHD_OK;
    }
  }
  return RHD_ERR_OUTER;
}

// Closure tensor D = P/E = dA I + dB Ft Ft^T of a state (E, Ft = F/c).
__device__ __forceinline__ void closure_D(const Physics& ph, double E, const double Ft[3],
                                          double& dA, double& dB) {
  if (ph.closure == RHD_CLOSURE_EDDINGTON) {
    dA = 1.0 / 3.0;
    dB = 0.0;
    return;
  }
  double ha, hb;
  m1_coeffs(E, Ft, ha, hb);
  const double iE = 1.0 / E;
  dA = ha * iE;
  dB = hb * iE;
}

// Implicit stage of one cell for non-grey material (general kernels only):
// chi_0E = chi (times the T factor), chi_0P = rP chi_0E, chi_0F = rF chi_0E in
// eq. (G0)/(G1).  The same inner/outer iteration as local_solve, with
//   R = k [(rP a T^4 - E) g + (2 - rF) v.F/c^2 + (rF - 1)(beta^2 + v.D.v/c^2) E]
// (k = chat chi_0E theta dt; the last term at order 2 only, with the closure
// tensor D frozen like v and F: that of the explicit state, then the one of
// the previous flux update), the R-row scaled by k' = k g - (kF - k)(beta^2 +
// v.D.v/c^2), the paper's Jacobian ((chi_0P/chi_0E) 4aT^3/C_v, -1/k - 1), and
// the flux from eq. (fupdate) with eq. (G1): at order 2
//   [(1 + kF g) I + 2 (kF - k)/c^2 v v^T] F = F(t) + kP a T^4 v + kF v.P + (kF - k) E v,
// solved by the Sherman-Morrison formula; at order 1 eq. (numF1).
template <bool MIXED>
__device__ int local_solve_nongrey(const Physics& ph, double tdt, double rho, double chi,
                                   double y[8], int& nn, int& no) {
  nn = 0;
  no = 0;
  if (chi == 0.0) return RHD_OK;
  const double Cv = rho * ph.cv_spec;
  const double inv_Cv = 1.0 / Cv, inv_rho = 1.0 / rho;
  const double cr = ph.c_over_chat, a = ph.a_rad, ic2 = ph.inv_c2;
  const double Eg0 = y[0], E0 = y[4];
  const double tolG = ph.newton_rtol * (Eg0 + cr * E0);
  const bool o2 = ph.vc_order == 2;
  const bool vary = ph.kappa_T_exp != 0.0;
  const double rP = ph.kappa_P_ratio, rF = ph.kappa_F_ratio;
  const double k0 = ph.chat * chi * tdt;
  double Eg = Eg0, R = 0.0, E = E0;
  double m[3] = {y[1], y[2], y[3]};
  double F[3] = {y[5], y[6], y[7]};
  double v[3] = {m[0] * inv_rho, m[1] * inv_rho, m[2] * inv_rho};
  double beta2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * ic2;
  double g = o2 ? 1.0 + 0.5 * beta2 : 1.0;
  double w = (v[0] * F[0] + v[1] * F[1] + v[2] * F[2]) * ic2;
  double Ekin = 0.5 * (m[0] * v[0] + m[1] * v[1] + m[2] * v[2]);
  double dA, dB, Fd[3] = {F[0] * ph.inv_c, F[1] * ph.inv_c, F[2] * ph.inv_c};
  closure_D(ph, E0, Fd, dA, dB);
  auto vdv_of = [&](const double vv[3]) {
    double vf = vv[0] * Fd[0] + vv[1] * Fd[1] + vv[2] * Fd[2];
    return (dA * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]) + dB * vf * vf) * ic2;
  };
  double vDv = vdv_of(v);
  double kE = k0, kP = rP * k0, kF = rF * k0;
  auto set_k = [&](double T) {
    kE = vary ? k0 * pow(T * ph.inv_kappa_T_ref, ph.kappa_T_exp) : k0;
    kP = rP * kE;
    kF = rF * kE;
  };
  auto kprime = [&]() { return kE * g - (o2 ? (kF - kE) * (beta2 + vDv) : 0.0); };

  if (!vary) {  // start from the frozen-opacity quartic A T^4 + C_v T = C (see quartic_start)
    const double T0 = (Eg0 - Ekin) * inv_Cv;
    if (pos_finite(T0)) {
      set_k(T0);
      const double kp = kprime();
      if (kp > 0.0) {
        const double inv1 = 1.0 / (1.0 + kp);
        const double a4 = cr * kP * g * a * inv1 * inv_Cv;
        const double rhs = T0 + cr * (kp * E0 - (2.0 * kE - kF) * w) * inv1 * inv_Cv;
        double Tg;
        if (pos_finite(rhs) && a4 > 0.0 && quartic_start(a4, rhs, T0, Tg)) {
          Eg = Cv * Tg + Ekin;
          R = -ph.chat_over_c * (Eg - Eg0);
        }
      }
    }
  }

  for (int outer = 0; outer < ph.outer_max; ++outer) {
    no = outer + 1;
    bool conv = false;
    double aT4 = 0.0, kp = 0.0;
    for (int it = 0;; ++it) {
      const double T = (Eg - Ekin) * inv_Cv;
      if (!pos_finite(T) || !finite_bits(R)) return RHD_ERR_NONPHYSICAL;
      set_k(T);
      kp = kprime();
      if (!(kp > 0.0)) return RHD_ERR_NONPHYSICAL;
      const double T2 = T * T;
      aT4 = a * T2 * T2;
      const double Se = kP * aT4 * g + (2.0 * kE - kF) * w;
      const double r0 = (Eg - Eg0) + cr * R;
      const double r1 = Se - R - kp * (E0 + R);
      if (fabs(r0) < tolG && cr * fabs(r1) <= tolG * kp) {
        conv = true;
        break;
      }
      if (it >= ph.newton_max) break;
      double J10 = kp * rP * 4.0 * a * T2 * T * inv_Cv;
      if (vary) J10 += ph.kappa_T_exp * R / (Eg - Ekin);  // as in local_solve
      const double gpk = kp / kE + kp;
      const double det = -gpk - cr * J10;
      const double inv_det = MIXED ? (double)(1.0f / (float)det) : 1.0 / det;
      Eg += (r0 * gpk + cr * r1) * inv_det;
      R += (r0 * J10 - r1) * inv_det;
      ++nn;
    }
    if (!conv) return RHD_ERR_NEWTON;

    E = E0 - ph.chat_over_c * (Eg - Eg0);  // energy closure
    // closure at (E, F of the previous pass): P v for eq. (G1) and the tensor
    // the next inner stage freezes
    double Ft[3] = {F[0] * ph.inv_c, F[1] * ph.inv_c, F[2] * ph.inv_c};
    closure_D(ph, E, Ft, dA, dB);
    Fd[0] = Ft[0]; Fd[1] = Ft[1]; Fd[2] = Ft[2];
    const double vFt = v[0] * Ft[0] + v[1] * Ft[1] + v[2] * Ft[2];
    double rhs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double vP = (dA * v[i] + dB * vFt * Ft[i]) * E;
      rhs[i] = y[5 + i] + kP * aT4 * v[i] + kF * vP + (kF - kE) * E * v[i];
    }
    double Fn[3], mn[3];
    if (o2) {
      const double aa = 1.0 + kF * g;
      const double b = 2.0 * (kF - kE) * ic2;
      const double vr = v[0] * rhs[0] + v[1] * rhs[1] + v[2] * rhs[2];
      const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
      const double corr = b * vr / (aa + b * v2);
#pragma unroll
      for (int i = 0; i < 3; ++i) Fn[i] = (rhs[i] - corr * v[i]) / aa;
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) Fn[i] = rhs[i] / (1.0 + kF);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) mn[i] = y[1 + i] - (Fn[i] - y[5 + i]) * ph.inv_cchat;

    const double Q_old = (kP * aT4 - kE * E) * (g - 1.0) + (2.0 * kE - kF) * w +
                         (o2 ? (kF - kE) * (beta2 + vDv) * E : 0.0);
    double vn[3] = {mn[0] * inv_rho, mn[1] * inv_rho, mn[2] * inv_rho};
    const double beta2n = (vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]) * ic2;
    const double gn = o2 ? 1.0 + 0.5 * beta2n : 1.0;
    const double wn = (vn[0] * Fn[0] + vn[1] * Fn[1] + vn[2] * Fn[2]) * ic2;
    const double vDvn = vdv_of(vn);
    const double Q_new = (kP * aT4 - kE * E) * (gn - 1.0) + (2.0 * kE - kF) * wn +
                         (o2 ? (kF - kE) * (beta2n + vDvn) * E : 0.0);
    const double Q_scale =
        fabs((kP * aT4 - kE * E) * (gn - 1.0)) +
        fabs(2.0 * kE - kF) * (fabs(vn[0] * Fn[0]) + fabs(vn[1] * Fn[1]) + fabs(vn[2] * Fn[2])) *
            ic2 +
        (o2 ? fabs(kF - kE) * (beta2n + fabs(vDvn)) * E : 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[i] = Fn[i];
      m[i] = mn[i];
      v[i] = vn[i];
    }
    beta2 = beta2n;
    g = gn;
    w = wn;
    vDv = vDvn;
    Ekin = 0.5 * (m[0] * v[0] + m[1] * v[1] + m[2] * v[2]);
    const double dQ = fabs(Q_new - Q_old);
    if (dQ <= ph.outer_rtol * fabs(Q_old) || dQ <= ph.outer_rtol * fabs(R) ||
        dQ <= ph.outer_rtol * Q_scale) {
      y[0] = Eg;
      y[1] = m[0]; y[2] = m[1]; y[3] = m[2];
      y[4] = E;
      y[5] = F[0]; y[6] = F[1]; y[7] = F[2];
      if (!pos_finite(E) || !finite_bits(F[0]) || !finite_bits(F[1]) || !finite_bits(F[2]))
        return RHD_ERR_NONPHYSICAL;
      return RHD_OK;
    }
  }
  return RHD_ERR_OUTER;
}

// ------------------------------------------------------------ launchers
// (host side, defined in the .cu files)
// b0, b1: the tile rows [b0, b1) of the slowest axis (b1 < 0: to the end)
cudaError_t launch_stage(int stage, int precision, const StageArgs& A, cudaStream_t s,
                         int b0 = 0, int b1 = -1);
cudaError_t launch_stage_ppm(int stage, int precision, const StageArgs& A, cudaStream_t s,
                             int b0 = 0, int b1 = -1);
// tile rows of a grid along its slowest axis, and the cells of one row
int stage_rows(const Geometry& g);
long long stage_row_cells(const Geometry& g, int row);
cudaError_t launch_status_reset(DevStatus* st, cudaStream_t s);
cudaError_t launch_totals(const Geometry& g, const Physics& ph, const double* y,
                          double* partials, int npart, double* out4, cudaStream_t s);
int totals_partials_needed();
// halo_kappa, halo_rho: plane 0 of the slab above a HALO top face (else null);
// i0, i1: the cells [i0, i1) whose +d faces are computed (i1 < 0: to the end)
cudaError_t launch_tau_eps(const Geometry& g, const double* rho, const double* kappa,
                           double tau_scale, double* const eps[3], cudaStream_t s,
                           const double* halo_kappa = nullptr,
                           const double* halo_rho = nullptr, long long i0 = 0,
                           long long i1 = -1);
cudaError_t launch_check_field(int field, const double* x, int n, int* flag,
                               cudaStream_t s);
// message returned by rhd_last_error(NULL) on this thread
void set_global_error(const char* msg);
// device-side geometry and physics of validated params
void fill_geometry(const rhd_params* p, Geometry& g, Physics& ph);
// whether a grid needs the general kernels (RK2-SSP, a temperature-dependent
// opacity or an inflow face) rather than the lean default ones
inline bool needs_general(const Geometry& g, const Physics& ph) {
  if (ph.scheme != RHD_SCHEME_IMEX_PDARS || ph.kappa_T_exp != 0.0 ||
      ph.reconstruction != RHD_RECON_PLM ||
      ph.kappa_P_ratio != 1.0 || ph.kappa_F_ratio != 1.0)
    return true;
  for (int d = 0; d < g.ndim; ++d)
    if (g.bc[d][0] == RHD_BC_INFLOW || g.bc[d][1] == RHD_BC_INFLOW) return true;
  return false;
}

}  // namespace rhd
