// rhd_tile.cuh -- one tile of one IMEX stage, shared by the grid kernels
// (rhd_stage.cu) and the batched persistent kernel (rhd_batch.cu).
//
// Work layout (3-D): a block owns a TX x TY column of cells and marches
// through a chunk of z planes.  E and F/c of four consecutive planes sit in
// a shared-memory ring, each plane with a 2-cell halo in x and y (3 with PPM
// faces; ghost cells folded in at load time: periodic wrap, or mirror with
// the normal flux negated).  Every face flux is computed exactly once: x- and y-faces of the
// current plane by one thread each (into shared memory), z-faces by the thread
// that owns the column (kept in registers from one plane to the next,
// together with the half z-slope of the current cell).  The thread then
// applies the conservative update and runs the cell's local implicit solve in
// registers, so the explicit state never reaches HBM.  2-D grids use one
// plane; 1-D grids use rows of TX cells.
#pragma once

#include <type_traits>

#include "rhd_internal.cuh"

namespace rhd {

// A tile: TX x TY threads (one per cell of a plane), LZ planes per block in
// 3-D.  PPM: piecewise parabolic faces (else PLM).  HX, HY: halo widths; NPL:
// planes kept in the shared-memory ring.
template <int NDIM_, int TX_, int TY_, int LZ_, bool PPM_ = false>
struct TileT {
  static constexpr int NDIM = NDIM_, TX = TX_, TY = TY_, LZ = LZ_;
  static constexpr bool PPM = PPM_;
  static constexpr int HX = PPM ? 3 : 2, HY = NDIM >= 2 ? HX : 0;
  static constexpr int NPL = NDIM == 3 ? 4 : 1;
  static constexpr int NT = TX * TY;
};

template <int NDIM>
struct DefaultTileOf;
// 3-D: 8 planes per block.  Longer z-chunks load fewer halo planes, but the
// per-block cost varies with the local physics (iteration counts), and short
// chunks balance the SMs better (256^3: 8 planes 2.6 % faster than 32).
// Build-time shape of the 3-D tile (rows TY of 32 cells, LZ planes per
// block) and the blocks per SM its stage kernels are compiled for.
#ifndef RHD_TILE3_TY
#define RHD_TILE3_TY 8
#endif
#ifndef RHD_TILE3_LZ
#define RHD_TILE3_LZ 8
#endif
template <>
struct DefaultTileOf<3> { using type = TileT<3, 32, RHD_TILE3_TY, RHD_TILE3_LZ>; };
template <>
struct DefaultTileOf<2> { using type = TileT<2, 32, 8, 1>; };
template <>
struct DefaultTileOf<1> { using type = TileT<1, 256, 1, 1>; };
template <int NDIM>
using Tile = typename DefaultTileOf<NDIM>::type;

// PPM tiles: the same shapes with the wider halo (3-D, FP64: 86 KB of
// shared memory, two blocks per SM).
template <int NDIM>
using TilePPM = TileT<NDIM, DefaultTileOf<NDIM>::type::TX, DefaultTileOf<NDIM>::type::TY,
                      DefaultTileOf<NDIM>::type::LZ, true>;

// ring slot of plane p (p >= -3)
template <class T>
__device__ __forceinline__ int ring_slot(int p) {
  return T::NPL == 4 ? (p & 3) : 0;
}

template <class T, typename R>
struct SmemT {
  static constexpr int PW = T::TX + 2 * T::HX;
  static constexpr int PH = T::TY + 2 * T::HY;
  static constexpr int PS = PW * PH;                   // cells per plane
  // values per cell: E, Ft (FP64); mixed: their hi and lo single-precision
  // parts, E_hi .. Fz_hi then E_lo .. Fz_lo (split_hilo)
  static constexpr int NV = sizeof(R) == sizeof(float) ? 8 : 4;
  static constexpr int PLANE = NV * PS;                // R values per ring plane
  static constexpr int RING = T::NPL * PLANE;
  static constexpr int FX = 4 * T::TY * (T::TX + 1);   // x-face fluxes
  static constexpr int FY = T::NDIM >= 2 ? 4 * (T::TY + 1) * T::TX : 0;
  // PPM z march: each thread's carried right edge and interface value (kept
  // in shared memory: in registers they push the FP64 kernel past its budget)
  static constexpr int CZ = (T::PPM && T::NDIM == 3) ? 12 * T::NT : 0;
  // mixed precision: the isotropic part of each x-/y-face's normal momentum
  // flux in double (hll_states_mixed), after the R arrays (16-byte aligned)
  static constexpr bool ISO = sizeof(R) == sizeof(float);
  static constexpr int FXI = ISO ? T::TY * (T::TX + 1) : 0;
  static constexpr int FYI = ISO && T::NDIM >= 2 ? (T::TY + 1) * T::TX : 0;
  static constexpr size_t ISO_OFF = sizeof(R) * (RING + FX + FY + CZ);
  // local solves in cost order (stages 1 and 2, where the launch supplies
  // the predicted costs): per slot the explicit state (8 doubles,
  // slot-minor), then per slot the solve flag and source thread / the
  // status, the Newton and outer counts, and the per-warp counts of each cost
  // bucket.  The FP64 3-D PPM tile, whose two blocks per SM leave no room for
  // more, stages the states in its face-flux arrays, which hold nothing
  // between a plane's flux differences and the next plane's faces.
  static constexpr int NB = 32;  // cost buckets
  static constexpr bool SORT_ALIAS = T::PPM && T::NDIM == 3 && sizeof(R) == sizeof(double);
  static_assert(!SORT_ALIAS || sizeof(R) * (FX + FY) >= sizeof(double) * 8 * T::NT,
                "the face-flux arrays hold the staged states");
  static constexpr size_t SORT_Y_OFF =
      SORT_ALIAS ? sizeof(R) * RING : ISO_OFF + sizeof(double) * (FXI + FYI);
  static constexpr size_t SORT_I_OFF = ISO_OFF + sizeof(double) * (FXI + FYI) +
                                       (SORT_ALIAS ? 0 : sizeof(double) * 8 * T::NT);
  static constexpr size_t BYTES = SORT_I_OFF + sizeof(int) * (3 * T::NT + (T::NT / 32) * NB);
};

// Coordinate x >= -3 folded onto [0, n) by the boundary condition (padding
// of a partial tile beyond n + hmax is clamped first; a mirror needs
// n >= hmax + 1); flip = mirror image.
__device__ __forceinline__ int fold(int x, int n, int bclo, int bchi, bool& flip,
                                    int hmax = 1) {
  flip = false;
  x = min(x, n + hmax);
  if (x < 0) {
    if (bclo == RHD_BC_PERIODIC) {
      x = ((x % n) + n) % n;
    } else {
      x = -1 - x;
      flip = true;
    }
  } else if (x >= n) {
    if (bchi == RHD_BC_PERIODIC) {
      x = x % n;
    } else {
      x = 2 * n - 1 - x;
      flip = true;
    }
  }
  return x;
}

// Side (0 low, 1 high) of an inflow ghost at coordinate x along axis d, or -1
// for an interior cell or a ghost of another boundary kind.
__device__ __forceinline__ int inflow_side(const Geometry& g, int d, int x) {
  if (x < 0) return g.bc[d][0] == RHD_BC_INFLOW ? 0 : -1;
  if (x >= g.n[d]) return g.bc[d][1] == RHD_BC_INFLOW ? 1 : -1;
  return -1;
}

// Side (0 low, 1 high) of a ghost plane z that a neighbouring slab supplies
// (an RHD_BC_HALO z face), or -1.
__device__ __forceinline__ int halo_side(const Geometry& g, int z) {
  if (z < 0) return g.bc[2][0] == RHD_BC_HALO ? 0 : -1;
  if (z >= g.n[2]) return g.bc[2][1] == RHD_BC_HALO ? 1 : -1;
  return -1;
}

// Field E of ghost plane z in its halo buffer (F_x, F_y, F_z follow at
// strides of HALO_PLANES planes).
__device__ __forceinline__ const double* halo_plane(const StageArgs& A, int side, int z) {
  const int i = side == 0 ? z + HALO_PLANES : z - A.g.n[2];
  return A.halo[side] + (size_t)i * A.g.n[0] * A.g.n[1];
}

// optical depth of the face from the flux-mean opacity chi_0F
__device__ __forceinline__ double eps_direct(const StageArgs& A, int ia, int ib, int d) {
  const long long n = A.g.ncell;
  double tau = 0.5 * (RHD_LD(A.st, A.kappa, ia, n) * RHD_LD(A.st, A.rho, ia, n) +
                      RHD_LD(A.st, A.kappa, ib, n) * RHD_LD(A.st, A.rho, ib, n)) * A.g.dx[d];
  return tau_factor(tau * A.ph.kappa_F_ratio);
}

// Optical-depth factor of the face on the +d side of the cell c (c[d] may be
// -1: the low wall face).  TAU mode only; 1 otherwise.
__device__ __forceinline__ double face_eps(const StageArgs& A, int d, int cx, int cy, int cz) {
  if (A.ph.hll_mode != RHD_HLL_TAU) return 1.0;
  const Geometry& g = A.g;
  int c[3] = {cx, cy, cz};
  if (c[d] < 0) {
    // the low face of a slab: the factor its neighbour below computed
    if (g.bc[d][0] == RHD_BC_HALO)
      return RHD_LDG(A.st, A.eps_zlo, c[0] + g.n[0] * c[1], (long long)g.n[0] * g.n[1]);
    if (g.bc[d][0] != RHD_BC_PERIODIC) {
      c[d] = 0;  // reflecting wall: the ghost mirrors cell 0
      int i0 = c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
      return eps_direct(A, i0, i0, d);
    }
    c[d] = g.n[d] - 1;  // periodic: the same face as the top one
  }
  int il = c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
  if (A.eps[d]) return RHD_LDG(A.st, A.eps[d], il, g.ncell);
  bool flip;
  int xb = fold(c[d] + 1, g.n[d], g.bc[d][0], g.bc[d][1], flip);
  return eps_direct(A, il, il + (xb - c[d]) * g.stride[d], d);
}

// Mixed precision: x as a pair of floats with hi + lo = x to 2^-47 |x|.  hi
// is x with its mantissa cut to 24 bits (integer operations; exact in float
// within the float exponent range), lo = x - hi rounded to float.  A
// difference of two neighbours, (b_hi - a_hi) + (b_lo - a_lo), is then good
// to single precision of the difference itself, where the difference of the
// rounded values would carry an error of an ulp of the values: the MC slopes
// and face states of the mixed transport are formed that way.
__device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e >= 1023 - 126 && e <= 1023 + 127) {
    const double xt = __longlong_as_double(b & ~((1ll << 29) - 1));
    hi = __uint_as_float((unsigned)((b >> 32) & 0x80000000ll) |
                         ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff));
    lo = (float)(x - xt);
  } else {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
}

// load plane zg (global z, may be a ghost plane) into ring slot `slot`,
// converting to the transport precision R (mixed: hi/lo pairs)
template <class T, typename R, bool GEN>
__device__ __forceinline__ void load_plane(const StageArgs& A, R* ring, int slot, int zg,
                                           int x0, int y0) {
  constexpr int NDIM = T::NDIM;
  using S = SmemT<T, R>;
  const Geometry& g = A.g;
  bool fz = false;
  int zf = NDIM == 3 ? fold(zg, g.n[2], g.bc[2][0], g.bc[2][1], fz, T::HX - 1) : 0;
  const int zin = GEN && NDIM == 3 ? inflow_side(g, 2, zg) : -1;
  // a ghost plane of a HALO face: the neighbour's plane, not mirrored
  const int hs = NDIM == 3 ? halo_side(g, zg) : -1;
  const double* hp = hs >= 0 ? halo_plane(A, hs, zg) : nullptr;
  const size_t hq = (size_t)HALO_PLANES * g.n[0] * g.n[1];
  if (hs >= 0) fz = false;
  R* pl = ring + slot * S::PLANE;
  for (int c = threadIdx.x; c < S::PS; c += T::TX * T::TY) {
    int ii = c % S::PW, jj = c / S::PW;
    bool fx = false, fy = false;
    int xf = fold(x0 + ii - T::HX, g.n[0], g.bc[0][0], g.bc[0][1], fx, T::HX - 1);
    int yf = NDIM >= 2 ? fold(y0 + jj - T::HY, g.n[1], g.bc[1][0], g.bc[1][1], fy, T::HX - 1)
                       : 0;
    // the values in double (mixed: split into hi/lo pairs below); F/c is
    // rounded explicitly, like column_cell's
    const double wic = A.ph.inv_c;
    double E, Fx, Fy, Fz;
    if (hs >= 0) {
      // index into the side's halo buffer [4 fields][HALO_PLANES][n0 n1]
      const long long hi = (hp - A.halo[hs]) + xf + (long long)g.n[0] * yf;
      const double* hb = A.halo[hs];
      E = RHD_LDG(A.st, hb, hi, 4 * (long long)hq);
      Fx = __dmul_rn(RHD_LDG(A.st, hb, hi + hq, 4 * (long long)hq), wic);
      Fy = __dmul_rn(RHD_LDG(A.st, hb, hi + 2 * hq, 4 * (long long)hq), wic);
      Fz = __dmul_rn(RHD_LDG(A.st, hb, hi + 3 * hq, 4 * (long long)hq), wic);
    } else {
      int idx = xf + g.n[0] * (yf + g.n[1] * zf);
      E = RHD_LDG(A.st, A.yt[Y_ERAD], idx, g.ncell);
      Fx = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FX], idx, g.ncell), wic);
      Fy = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FY], idx, g.ncell), wic);
      Fz = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FZ], idx, g.ncell), wic);
    }
    Fx = fx ? -Fx : Fx;
    Fy = fy ? -Fy : Fy;
    Fz = fz ? -Fz : Fz;
    // ghost cells of an inflow face hold its fixed radiation state
    int ax = zin >= 0 ? 2 : -1, side = zin;
    if (GEN && ax < 0) {
      side = inflow_side(g, 0, x0 + ii - T::HX);
      ax = side >= 0 ? 0 : -1;
    }
    if (GEN && ax < 0 && NDIM >= 2) {
      side = inflow_side(g, 1, y0 + jj - T::HY);
      ax = side >= 0 ? 1 : -1;
    }
    if (ax >= 0) {
      const double* st = g.bc_state[ax][side];
      E = st[0];
      Fx = __dmul_rn(st[1], wic);
      Fy = __dmul_rn(st[2], wic);
      Fz = __dmul_rn(st[3], wic);
    }
    if constexpr (S::NV == 8) {
      const double v[4] = {E, Fx, Fy, Fz};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float hi, lo;
        split_hilo(v[q], hi, lo);
        pl[q * S::PS + c] = hi;
        pl[(4 + q) * S::PS + c] = lo;
      }
    } else {
      pl[0 * S::PS + c] = (R)E;
      pl[1 * S::PS + c] = (R)Fx;
      pl[2 * S::PS + c] = (R)Fy;
      pl[3 * S::PS + c] = (R)Fz;
    }
  }
}

#ifdef RHD_BOUNDS_CHECK
// the status block of the block's launch, for the checks of ring reads
static __shared__ DevStatus* s_chk_status;
#define RHD_RING_OK(c, n) chk_index(s_chk_status, (c), (n))
#else
#define RHD_RING_OK(c, n) true
#endif

template <class T, typename R>
__device__ __forceinline__ void cell_of(const R* pl, int c, R u[4]) {
  using S = SmemT<T, R>;
  if (!RHD_RING_OK(c, S::PS)) c = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) u[q] = pl[q * S::PS + c];
}

// mixed: the hi/lo parts of cell c of a ring plane
template <class T>
__device__ __forceinline__ void cell_hl(const float* pl, int c, float hi[4], float lo[4]) {
  using S = SmemT<T, float>;
  if (!RHD_RING_OK(c, S::PS)) c = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    hi[q] = pl[q * S::PS + c];
    lo[q] = pl[(4 + q) * S::PS + c];
  }
}

// difference b - a of two hi/lo values
__device__ __forceinline__ float diff_hl(float bh, float bl, float ah, float al) {
  return (bh - ah) + (bl - al);
}

// half of the MC-limited slope from the differences dm = u0 - um, dp = up - u0
// (the limiter of half_slope)
__device__ __forceinline__ float half_slope_d(float dm, float dp) {
  const float m = fminf(fminf(fabsf(dm), fabsf(dp)), 0.25f * fabsf(dm + dp));
  return (dm > 0.f && dp > 0.f) ? m : ((dm < 0.f && dp < 0.f) ? -m : 0.f);
}

// PPM states of the face between cells u[2] and u[3] of the six cells u
// (cs: the Colella-Sekora limiter)
template <typename R>
__device__ __forceinline__ void ppm_states(const R u[6][4], R L[4], R Rr[4], bool cs) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    R v[6];
#pragma unroll
    for (int o = 0; o < 6; ++o) v[o] = u[o][q];
    if (cs)
      ppm_cs_face(v, L[q], Rr[q]);
    else
      ppm_face(v, L[q], Rr[q]);
  }
}

// flux through the face between plane cells c - st and c (stride st); cs:
// PPM tiles with the Colella-Sekora limiter; iso: see face_hll
template <class T, typename R>
__device__ __forceinline__ bool plane_face(const R* pl, int c, int st, int d, R eps, R chat,
                                           int closure, double chat6, R out[4], double& iso,
                                           bool cs = false) {
  R L[4], Rr[4];
  if constexpr (T::PPM) {
    R u[6][4];
#pragma unroll
    for (int o = 0; o < 6; ++o) cell_of<T, R>(pl, c + (o - 3) * st, u[o]);
    ppm_states(u, L, Rr, cs);
  } else if constexpr (sizeof(R) == sizeof(float)) {
    // face states from the hi/lo differences of the four cells
    float hm[4], lm[4], ha[4], la[4], hb[4], lb[4], hp[4], lp[4];
    cell_hl<T>(pl, c - 2 * st, hm, lm);
    cell_hl<T>(pl, c - st, ha, la);
    cell_hl<T>(pl, c, hb, lb);
    cell_hl<T>(pl, c + st, hp, lp);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float d0 = diff_hl(ha[q], la[q], hm[q], lm[q]);
      const float d1 = diff_hl(hb[q], lb[q], ha[q], la[q]);
      const float d2 = diff_hl(hp[q], lp[q], hb[q], lb[q]);
      L[q] = ha[q] + (la[q] + half_slope_d(d0, d1));
      Rr[q] = hb[q] + (lb[q] - half_slope_d(d1, d2));
    }
  } else {
    R am[4], a[4], b[4], bp[4];
    cell_of<T, R>(pl, c - 2 * st, am);
    cell_of<T, R>(pl, c - st, a);
    cell_of<T, R>(pl, c, b);
    cell_of<T, R>(pl, c + st, bp);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      L[q] = a[q] + half_slope(am[q], a[q], b[q]);
      Rr[q] = b[q] - half_slope(a[q], b[q], bp[q]);
    }
  }
  return face_hll<R>(d, L, Rr, eps, chat, closure, chat6, out, iso);
}

// One cell (E, F/c) of the own column (cx, cy inside the grid) at plane zg,
// a ghost plane folded or taken from its inflow state exactly as load_plane
// does.
template <class T, typename R, bool GEN>
__device__ __forceinline__ void column_cell(const StageArgs& A, int cx, int cy, int zg,
                                            R u[4]) {
  // the values load_plane puts in the ring: double, or the hi part of a
  // mixed-precision hi/lo pair (a face shared by two z-chunks is then
  // computed from the same inputs by both, and the flux telescopes); the
  // products F/c are rounded explicitly, as the ring's stores round them,
  // so that no contraction into a later operation can make them differ
  const Geometry& g = A.g;
  const double inv_c = A.ph.inv_c;
  bool fz = false;
  const int zf = fold(zg, g.n[2], g.bc[2][0], g.bc[2][1], fz, T::HX - 1);
  const int hs = halo_side(g, zg);
  double w[4];
  if (hs >= 0) {
    const double* hb = A.halo[hs];
    const long long hi = (halo_plane(A, hs, zg) - hb) + cx + (long long)g.n[0] * cy;
    const long long hq = (long long)HALO_PLANES * g.n[0] * g.n[1];
    w[0] = RHD_LDG(A.st, hb, hi, 4 * hq);
    w[1] = __dmul_rn(RHD_LDG(A.st, hb, hi + hq, 4 * hq), inv_c);
    w[2] = __dmul_rn(RHD_LDG(A.st, hb, hi + 2 * hq, 4 * hq), inv_c);
    w[3] = __dmul_rn(RHD_LDG(A.st, hb, hi + 3 * hq, 4 * hq), inv_c);
  } else {
    const int idx = cx + g.n[0] * (cy + g.n[1] * zf);
    w[0] = RHD_LDG(A.st, A.yt[Y_ERAD], idx, g.ncell);
    w[1] = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FX], idx, g.ncell), inv_c);
    w[2] = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FY], idx, g.ncell), inv_c);
    const double Fz = __dmul_rn(RHD_LDG(A.st, A.yt[Y_FZ], idx, g.ncell), inv_c);
    w[3] = fz ? -Fz : Fz;
  }
  const int side = GEN ? inflow_side(g, 2, zg) : -1;
  if (side >= 0) {
    const double* st = g.bc_state[2][side];
    w[0] = st[0];
    w[1] = __dmul_rn(st[1], inv_c);
    w[2] = __dmul_rn(st[2], inv_c);
    w[3] = __dmul_rn(st[3], inv_c);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if constexpr (sizeof(R) == sizeof(float)) {
      float lo;
      split_hilo(w[q], u[q], lo);
    } else {
      u[q] = w[q];
    }
  }
}

// Per-thread iteration statistics of the cells a thread has solved.
// ------------------------------------------------ local solves in cost order
// Shared arrays of the sorted solves: 8 doubles per slot (the explicit state
// y*), then per slot the solve flag and source thread (in) / the status
// (out), the Newton and the outer counts, then the per-warp counts of each
// cost bucket.
template <class T, typename R>
struct SortSmem {
  double* v;
  int* flag;
  int* nn;
  int* no;
  int* tab;
  __device__ __forceinline__ explicit SortSmem(unsigned char* smem) {
    using S = SmemT<T, R>;
    v = reinterpret_cast<double*>(smem + S::SORT_Y_OFF);
    flag = reinterpret_cast<int*>(smem + S::SORT_I_OFF);
    nn = flag + T::NT;
    no = nn + T::NT;
    tab = no + T::NT;
  }
};

// Solve cost of a cell as kept between steps: its outer passes (1..8) in the
// top 3 bits, its Newton updates (0..31) in the low 5; 0 before the first.
__device__ __forceinline__ unsigned char cost_byte(int nn, int no) {
  return (unsigned char)((min(max(no, 1), 8) - 1) << 5 | min(nn, 31));
}

// Cost bucket of a kept cost: nn + 4 no - 8, within [0, 31] (the work of a
// Newton update counting 1 and of an outer pass about 4).
__device__ __forceinline__ int cost_key(int b) {
  if (b == 0) return 0;
  const int no = (b >> 5) + 1, nn = b & 31;
  return max(0, min(31, nn + 4 * no - 8));
}

// Slot of this thread's cell in the block's cost order: a stable counting
// sort on the cost bucket of the previous step's cost (cells without a solve
// in bucket 0).  Sorted rank r goes to warp r / 32 in the first half of
// the warps and to the mirrored warp in the second (ranks 128..255 of 256 to
// warps 7..4), so that each of the SM's schedulers (warp w runs on scheduler
// w mod 4) holds one cheaper and one dearer warp of the block.  The bucket
// counts must be zero on entry; every thread of the block calls this.
template <class T, typename R>
__device__ __forceinline__ int sort_slot(unsigned char* smem, const StageArgs& A, bool need,
                                         int idx, int ncell) {
  using S = SmemT<T, R>;
  constexpr int NT = T::NT, NW = NT / 32, NB = S::NB;
  static_assert(NB == 32 && NT % 32 == 0 && (NW % 2 == 0), "one lane per bucket, warp pairs");
  SortSmem<T, R> q(smem);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int key = 0;
  if (need) key = cost_key((int)RHD_LD(A.st, A.cost, idx, ncell));
  const unsigned m = __match_any_sync(full, key);
  const int wrank = __popc(m & ((1u << lane) - 1u));
  if (wrank == 0) RHD_ST(A.st, q.tab, warp * NB + key, NW * NB, __popc(m));
  __syncthreads();
  if (warp == 0) {  // lane b: the start of bucket b in each warp
    int tot = 0;
    for (int w = 0; w < NW; ++w) tot += q.tab[w * NB + lane];
    int base = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, base, o);
      if (lane >= o) base += v;
    }
    base -= tot;
    for (int w = 0; w < NW; ++w) {
      const int c = q.tab[w * NB + lane];
      q.tab[w * NB + lane] = base;
      base += c;
    }
  }
  __syncthreads();
  const int r = (int)RHD_LD(A.st, q.tab, warp * NB + key, NW * NB) + wrank;
  const int gw = r >> 5;
  const int tw = gw < NW / 2 ? gw : (3 * NW / 2 - 1) - gw;
  return tw * 32 + (r & 31);
}

// this thread's cell (its explicit state; whether it needs a solve) into its
// sorted slot
template <class T, typename R>
__device__ __forceinline__ void stage_slot_put(unsigned char* smem, const StageArgs& A, int slot,
                                               const double y[8], bool need) {
  constexpr int NT = T::NT;
  SortSmem<T, R> q(smem);
#pragma unroll
  for (int j = 0; j < 8; ++j) RHD_ST(A.st, q.v, j * NT + slot, 8 * NT, y[j]);
  RHD_ST(A.st, q.flag, slot, NT, need ? (int)(threadIdx.x << 1) | 1 : 0);
}

// the cell of slot (this thread's solve): its state, and through src the
// thread that owns it; clears the bucket counts for the next plane (all
// threads have read them before the barrier that precedes this call);
// returns whether the cell needs a solve
template <class T, typename R>
__device__ __forceinline__ bool stage_slot_get(unsigned char* smem, const StageArgs& A, int slot,
                                               double y[8], int& src) {
  using S = SmemT<T, R>;
  constexpr int NT = T::NT, NTAB = (NT / 32) * S::NB;
  SortSmem<T, R> q(smem);
  for (int i = threadIdx.x; i < NTAB; i += NT) q.tab[i] = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) y[j] = RHD_LD(A.st, q.v, j * NT + slot, 8 * NT);
  const int f = (int)RHD_LD(A.st, q.flag, slot, NT);
  src = f >> 1;
  return (f & 1) != 0;
}

// the solved cell of slot back into its slot
template <class T, typename R>
__device__ __forceinline__ void stage_slot_result(unsigned char* smem, const StageArgs& A,
                                                  int slot, const double y[8], int code, int nn,
                                                  int no) {
  constexpr int NT = T::NT;
  SortSmem<T, R> q(smem);
#pragma unroll
  for (int j = 0; j < 8; ++j) RHD_ST(A.st, q.v, j * NT + slot, 8 * NT, y[j]);
  RHD_ST(A.st, q.flag, slot, NT, code);
  RHD_ST(A.st, q.nn, slot, NT, nn);
  RHD_ST(A.st, q.no, slot, NT, no);
}

// this thread's own cell, solved, from its sorted slot
template <class T, typename R>
__device__ __forceinline__ void stage_slot_take(unsigned char* smem, const StageArgs& A, int slot,
                                                double y[8], int& code, int& nn, int& no) {
  constexpr int NT = T::NT;
  SortSmem<T, R> q(smem);
#pragma unroll
  for (int j = 0; j < 8; ++j) y[j] = RHD_LD(A.st, q.v, j * NT + slot, 8 * NT);
  code = (int)RHD_LD(A.st, q.flag, slot, NT);
  nn = (int)RHD_LD(A.st, q.nn, slot, NT);
  no = (int)RHD_LD(A.st, q.no, slot, NT);
}

struct TileStats {
  int nn_max = 0, no_max = 0;
  unsigned long long nn_sum = 0, no_sum = 0, cnt = 0;
};

// One tile of one stage (STAGE 1, 2, or 0 = transport rates only; GEN: with
// the general physics, RK2-SSP, a temperature-dependent opacity and inflow
// faces, which the default physics compiles out): the block
// of T::NT threads owns the cells x0 + [0, TX) x y0 + [0, TY) x planes
// [kbeg, kbeg + LZ) of the grid described by A.  R: precision of
// reconstruction, closure and HLL fluxes (double for FP64, float for MIXED);
// the state, the flux differences, the updates and the local solve are double
// in both.  Every thread of the block must call it (it synchronises).
template <int STAGE, class T, typename R, bool GEN>
__device__ __forceinline__ void stage_tile(const StageArgs& A, int x0, int y0, int kbeg,
                                           unsigned char* smem_raw, TileStats& ts) {
  using S = SmemT<T, R>;
  constexpr int NDIM = T::NDIM;
  constexpr int TX = T::TX, TY = T::TY, NT = TX * TY;
  constexpr bool MIXED = sizeof(R) == sizeof(float);
  R* ring = reinterpret_cast<R*>(smem_raw);
  R* fxs = ring + S::RING;
  R* fys = fxs + S::FX;
  double* fxi = reinterpret_cast<double*>(smem_raw + S::ISO_OFF);  // MIXED only
  double* fyi = fxi + S::FXI;

  const Geometry& g = A.g;
  const Physics& ph = A.ph;
#ifdef RHD_BOUNDS_CHECK
  if (threadIdx.x == 0) s_chk_status = A.st;
  __syncthreads();
#endif
  if constexpr (STAGE != 0) {
    if (A.cost != nullptr) {  // the sorted solves' bucket counts start at zero
      SortSmem<T, R> q(smem_raw);
      for (int i = threadIdx.x; i < (NT / 32) * S::NB; i += NT) q.tab[i] = 0;
      __syncthreads();
    }
  }
  const R chat = (R)ph.chat;
  const double chat6 = ph.chat * (1.0 / 6.0);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int ix = x0 + tx, iy = y0 + ty;
  const bool col = ix < g.n[0] && (NDIM < 2 || iy < g.n[1]);
  const int cy = NDIM >= 2 ? min(iy, g.n[1] - 1) : 0;  // clamped row of the column
  const int cx = min(ix, g.n[0] - 1);
  const int kend = min(kbeg + T::LZ, g.n[2]);
  const int own = (tx + T::HX) + (ty + T::HY) * S::PW;  // own cell in a plane

  bool zbad = false;

  R zlo[4] = {R(0), R(0), R(0), R(0)};  // z-face flux below the current cell
  double zlo_iso = 0.0;                 // its isotropic momentum part (MIXED)
  R hz[4] = {R(0), R(0), R(0), R(0)};   // half z-slope of the current cell (PLM)
  // PPM z march: the constrained right edge of the current cell and the
  // interface value above it, carried from plane to plane, so each plane
  // adds one cell's edges; the start reads the own column from memory
  R* rz = fys + S::FY + threadIdx.x;       // rz[q * NT]: right edge of cell k
  R* az = rz + 4 * NT;                      // az[q * NT]: interface value a(k+1/2)
  R* dz = az + 4 * NT;                      // dz[q * NT]: second difference of cell k
  const bool cs = T::PPM && ph.reconstruction == RHD_RECON_PPM_CS;
  if constexpr (NDIM == 3 && T::PPM) {
    R u[6][4];
#pragma unroll
    for (int o = 0; o < 6; ++o) column_cell<T, R, GEN>(A, cx, cy, kbeg - 3 + o, u[o]);
    R L[4], Rr[4];
    if (cs) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        R w[6];
#pragma unroll
        for (int o = 0; o < 6; ++o) w[o] = u[o][q];
        const R a12 = cs_interface(w[0], w[1], w[2], w[3]);
        const R a23 = cs_interface(w[1], w[2], w[3], w[4]);
        const R a34 = cs_interface(w[2], w[3], w[4], w[5]);
        const R d2a = w[1] - R(2) * w[2] + w[3], d2b = w[2] - R(2) * w[3] + w[4];
        R l2 = a12, r2 = a23, l3 = a23, r3 = a34;
        cs_edges(w[1], w[2], w[3], w[0] - R(2) * w[1] + w[2], d2b, l2, r2);
        cs_edges(w[2], w[3], w[4], d2a, w[3] - R(2) * w[4] + w[5], l3, r3);
        L[q] = r2;
        Rr[q] = l3;
        rz[q * NT] = r3;
        az[q * NT] = a34;
        dz[q * NT] = d2b;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const R h1 = half_slope(u[0][q], u[1][q], u[2][q]);
        const R h2 = half_slope(u[1][q], u[2][q], u[3][q]);
        const R h3 = half_slope(u[2][q], u[3][q], u[4][q]);
        const R h4 = half_slope(u[3][q], u[4][q], u[5][q]);
        const R a12 = ppm_interface(u[1][q], u[2][q], h1, h2);
        const R a23 = ppm_interface(u[2][q], u[3][q], h2, h3);
        const R a34 = ppm_interface(u[3][q], u[4][q], h3, h4);
        L[q] = ppm_edge_of<false>(u[2][q], a12, a23);
        Rr[q] = ppm_edge_of<true>(u[3][q], a23, a34);
        rz[q * NT] = ppm_edge_of<false>(u[3][q], a23, a34);
        az[q * NT] = a34;
      }
    }
    R eps = (R)face_eps(A, 2, cx, cy, kbeg - 1);
    zbad = !face_hll<R>(2, L, Rr, eps, chat, ph.closure, chat6, zlo, zlo_iso);
    for (int o = 0; o <= 2; ++o)
      load_plane<T, R, GEN>(A, ring, ring_slot<T>(kbeg + o), kbeg + o, x0, y0);
  } else if constexpr (NDIM == 3) {
    for (int o = -2; o <= 1; ++o)
      load_plane<T, R, GEN>(A, ring, (kbeg + o) & 3, kbeg + o, x0, y0);
    __syncthreads();
    R L[4], Rr[4];
    if constexpr (MIXED) {
      float hm[4], lm[4], h0[4], l0[4], hp[4], lp[4], hpp[4], lpp[4];
      cell_hl<T>(ring + ((kbeg - 2) & 3) * S::PLANE, own, hm, lm);
      cell_hl<T>(ring + ((kbeg - 1) & 3) * S::PLANE, own, h0, l0);
      cell_hl<T>(ring + ((kbeg + 0) & 3) * S::PLANE, own, hp, lp);
      cell_hl<T>(ring + ((kbeg + 1) & 3) * S::PLANE, own, hpp, lpp);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float d0 = diff_hl(h0[q], l0[q], hm[q], lm[q]);
        const float d1 = diff_hl(hp[q], lp[q], h0[q], l0[q]);
        const float d2 = diff_hl(hpp[q], lpp[q], hp[q], lp[q]);
        hz[q] = half_slope_d(d1, d2);
        L[q] = h0[q] + (l0[q] + half_slope_d(d0, d1));
        Rr[q] = hp[q] + (lp[q] - hz[q]);
      }
    } else {
      R um[4], u0[4], up[4], upp[4];
      cell_of<T, R>(ring + ((kbeg - 2) & 3) * S::PLANE, own, um);
      cell_of<T, R>(ring + ((kbeg - 1) & 3) * S::PLANE, own, u0);
      cell_of<T, R>(ring + ((kbeg + 0) & 3) * S::PLANE, own, up);
      cell_of<T, R>(ring + ((kbeg + 1) & 3) * S::PLANE, own, upp);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        hz[q] = half_slope(u0[q], up[q], upp[q]);
        L[q] = u0[q] + half_slope(um[q], u0[q], up[q]);
        Rr[q] = up[q] - hz[q];
      }
    }
    R eps = (R)face_eps(A, 2, cx, cy, kbeg - 1);
    zbad = !face_hll<R>(2, L, Rr, eps, chat, ph.closure, chat6, zlo, zlo_iso);
    __syncthreads();  // plane kbeg-2's slot is reloaded by the first iteration
  }

  for (int k = kbeg; k < kend; ++k) {
    if (NDIM == 3) {
      constexpr int AHEAD = T::PPM ? 3 : 2;
      load_plane<T, R, GEN>(A, ring, ring_slot<T>(k + AHEAD), k + AHEAD, x0, y0);
    } else {
      load_plane<T, R, GEN>(A, ring, 0, 0, x0, y0);
    }
    __syncthreads();
    const R* pl = ring + (NDIM == 3 ? ring_slot<T>(k) : 0) * S::PLANE;
    bool bad = zbad;

    // ---- z-face k+1/2 of the own column
    R zhi[4] = {R(0), R(0), R(0), R(0)};
    double zhi_iso = 0.0;
    R hz1[4] = {R(0), R(0), R(0), R(0)};
    if constexpr (NDIM == 3 && T::PPM) {
      // face k+1/2: the carried right edge of cell k | the left edge of
      // cell k+1, whose edges come from a(k+1/2) and a new a(k+3/2)
      R v0[4], v1[4], v2[4], v3[4];
      cell_of<T, R>(pl, own, v0);
      cell_of<T, R>(ring + ring_slot<T>(k + 1) * S::PLANE, own, v1);
      cell_of<T, R>(ring + ring_slot<T>(k + 2) * S::PLANE, own, v2);
      cell_of<T, R>(ring + ring_slot<T>(k + 3) * S::PLANE, own, v3);
      R L[4], Rr[4];
      if (cs) {
        // the cell k+1 needs the second difference of cell k, carried
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R an = cs_interface(v0[q], v1[q], v2[q], v3[q]);
          R l1 = az[q * NT], r1 = an;
          cs_edges(v0[q], v1[q], v2[q], dz[q * NT], v1[q] - R(2) * v2[q] + v3[q], l1, r1);
          L[q] = rz[q * NT];
          Rr[q] = l1;
          rz[q * NT] = r1;
          az[q * NT] = an;
          dz[q * NT] = v0[q] - R(2) * v1[q] + v2[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R ha = half_slope(v0[q], v1[q], v2[q]);
          const R hb = half_slope(v1[q], v2[q], v3[q]);
          const R an = ppm_interface(v1[q], v2[q], ha, hb);
          L[q] = rz[q * NT];
          Rr[q] = ppm_edge_of<true>(v1[q], az[q * NT], an);
          rz[q * NT] = ppm_edge_of<false>(v1[q], az[q * NT], an);
          az[q * NT] = an;
        }
      }
      R eps = (R)face_eps(A, 2, cx, cy, k);
      zbad = !face_hll<R>(2, L, Rr, eps, chat, ph.closure, chat6, zhi, zhi_iso);
      bad = bad || zbad;
    } else if constexpr (NDIM == 3) {
      R L[4], Rr[4];
      if constexpr (MIXED) {
        float h0[4], l0[4], h1[4], l1[4], h2[4], l2[4];
        cell_hl<T>(pl, own, h0, l0);
        cell_hl<T>(ring + ((k + 1) & 3) * S::PLANE, own, h1, l1);
        cell_hl<T>(ring + ((k + 2) & 3) * S::PLANE, own, h2, l2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          hz1[q] = half_slope_d(diff_hl(h1[q], l1[q], h0[q], l0[q]),
                                diff_hl(h2[q], l2[q], h1[q], l1[q]));
          L[q] = h0[q] + (l0[q] + hz[q]);
          Rr[q] = h1[q] + (l1[q] - hz1[q]);
        }
      } else {
        R u0[4], u1[4], u2[4];
        cell_of<T, R>(pl, own, u0);
        cell_of<T, R>(ring + ((k + 1) & 3) * S::PLANE, own, u1);
        cell_of<T, R>(ring + ((k + 2) & 3) * S::PLANE, own, u2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          hz1[q] = half_slope(u0[q], u1[q], u2[q]);
          L[q] = u0[q] + hz[q];
          Rr[q] = u1[q] - hz1[q];
        }
      }
      R eps = (R)face_eps(A, 2, cx, cy, k);
      zbad = !face_hll<R>(2, L, Rr, eps, chat, ph.closure, chat6, zhi, zhi_iso);
      bad = bad || zbad;
    }

    // ---- x-faces of plane k: face f lies between tile cells fi-1 and fi
    for (int f = threadIdx.x; f < (TX + 1) * TY; f += NT) {
      int fi = f % (TX + 1), fj = f / (TX + 1);
      int c = fi + T::HX + (fj + T::HY) * S::PW;
      int xl = x0 + fi - 1;
      int yr = NDIM >= 2 ? y0 + fj : 0;
      bool real = xl < g.n[0] && (NDIM < 2 || yr < g.n[1]);
      R eps = real ? (R)face_eps(A, 0, xl, yr, k) : R(1);
      R out[4];
      double iso;
      if (!plane_face<T, R>(pl, c, 1, 0, eps, chat, ph.closure, chat6, out, iso, cs) && real) {
        // a face with E <= 0 poisons both neighbours' fluxes
#pragma unroll
        for (int q = 0; q < 4; ++q) out[q] = (R)__longlong_as_double(0x7ff8000000000000ll);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) fxs[q * TY * (TX + 1) + f] = out[q];
      if constexpr (MIXED) fxi[f] = iso;
    }
    // ---- y-faces of plane k: face f lies between rows fj-1 and fj
    if (NDIM >= 2) {
      for (int f = threadIdx.x; f < TX * (TY + 1); f += NT) {
        int fi = f % TX, fj = f / TX;
        int c = fi + T::HX + (fj + T::HY) * S::PW;
        int xr = x0 + fi, yl = y0 + fj - 1;
        bool real = xr < g.n[0] && yl < g.n[1];
        R eps = real ? (R)face_eps(A, 1, xr, yl, k) : R(1);
        R out[4];
        double iso;
        if (!plane_face<T, R>(pl, c, S::PW, 1, eps, chat, ph.closure, chat6, out, iso, cs) &&
            real) {
#pragma unroll
          for (int q = 0; q < 4; ++q) out[q] = (R)__longlong_as_double(0x7ff8000000000000ll);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) fys[q * (TY + 1) * TX + f] = out[q];
        if constexpr (MIXED) fyi[f] = iso;
      }
    }
    __syncthreads();

    // this thread's cell: its explicit state y* (stages 1, 2), rho, chi
    double y[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double rho = 0.0, chi = 0.0;
    int idx = 0;
    int nn = 0, no = 0;
    int code = RHD_OK;
    bool need = false;  // a local solve to run for it
    // RK2-SSP (Sec. 4.2): no exchange in stage 1, the full dt f(y(n+1)) in
    // stage 2; IMEX PD-ARS: theta = 1, then theta = 1/2
    const bool rk2 = GEN && ph.scheme == RHD_SCHEME_RK2_SSP;
    if (col) {
      idx = ix + g.n[0] * (iy + g.n[1] * k);
      double rate[4];
      const int fl = tx + ty * (TX + 1);
      // flux differences in double: the difference of two floats is exact in
      // double, so the update telescopes across cells in both precisions
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const R* fq = fxs + q * TY * (TX + 1);
        double df = (double)fq[fl + 1] - (double)fq[fl];
        if (MIXED && q == 1) df += fxi[fl + 1] - fxi[fl];
        rate[q] = -df * g.inv_dx[0];
      }
      if (NDIM >= 2) {
        const int fb = tx + ty * TX;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const R* fq = fys + q * (TY + 1) * TX;
          double df = (double)fq[fb + TX] - (double)fq[fb];
          if (MIXED && q == 2) df += fyi[fb + TX] - fyi[fb];
          rate[q] -= df * g.inv_dx[1];
        }
      }
      if (NDIM == 3) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          double df = (double)zhi[q] - (double)zlo[q];
          if (MIXED && q == 3) df += zhi_iso - zlo_iso;
          rate[q] -= df * g.inv_dx[2];
        }
      }
      bad = bad || !isfinite(rate[0]) || !isfinite(rate[1]) || !isfinite(rate[2]) ||
            !isfinite(rate[3]);

      if (STAGE == 0) {
        // transport only: s(y) of eq. (yrsla) for E and the physical flux F
        RHD_ST(A.st, A.rate[0], idx, g.ncell, rate[0]);
#pragma unroll
        for (int j = 0; j < 3; ++j) RHD_ST(A.st, A.rate[1 + j], idx, g.ncell, ph.c * rate[1 + j]);
        if (bad) {
          atomicMin(&A.st->fail_key, ((unsigned long long)(A.cell_base + idx) << 8) | RHD_ERR_NONPHYSICAL);
          A.st->fail_step = A.step;
          A.st->fail_stage = 0;
        }
      } else if (STAGE == 1) {
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = RHD_LD(A.st, A.yt[q], idx, g.ncell);
        y[Y_ERAD] += A.dt * rate[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) y[Y_FX + j] += A.dt * ph.c * rate[1 + j];
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          y[q] = 0.5 * (RHD_LD(A.st, A.yn[q], idx, g.ncell) + RHD_LD(A.st, A.yt[q], idx, g.ncell));
        y[Y_ERAD] += 0.5 * A.dt * rate[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) y[Y_FX + j] += 0.5 * A.dt * ph.c * rate[1 + j];
      }
      rho = RHD_LD(A.st, A.rho, idx, g.ncell);
      chi = RHD_LD(A.st, A.kappa, idx, g.ncell) * rho;
      if (STAGE != 0) {
        if (bad)
          code = RHD_ERR_NONPHYSICAL;
        else
          need = !(rk2 && STAGE == 1);
      }
    }
    if constexpr (STAGE != 0) {
      const double tdt = (STAGE == 1 || rk2) ? A.dt : 0.5 * A.dt;
      // with predicted costs the block's solves run in cost order: each
      // thread solves the cell of its sorted slot, so that a warp's lanes
      // take similar numbers of iterations; a cell's arithmetic does not
      // depend on the lane that runs it, so the results are the same bits
      const bool sorted = A.cost != nullptr && !(rk2 && STAGE == 1);
      int myslot = threadIdx.x;
      bool run = need;
      if (sorted) {
        myslot = sort_slot<T, R>(smem_raw, A, need, idx, g.ncell);
        stage_slot_put<T, R>(smem_raw, A, myslot, y, need);
        __syncthreads();
        int src = 0;
        run = stage_slot_get<T, R>(smem_raw, A, threadIdx.x, y, src);
        if (run) {  // rho and chi of the slot's cell, as its own thread took them
          const int sidx = (x0 + src % TX) + g.n[0] * ((y0 + src / TX) + g.n[1] * k);
          rho = RHD_LD(A.st, A.rho, sidx, g.ncell);
          chi = RHD_LD(A.st, A.kappa, sidx, g.ncell) * rho;
        }
      }
      int scode = RHD_OK, snn = 0, sno = 0;
      if (run) {
        if (GEN && (ph.kappa_P_ratio != 1.0 || ph.kappa_F_ratio != 1.0))
          scode = local_solve_nongrey<MIXED>(ph, tdt, rho, chi, y, snn, sno);
        else
          scode = local_solve<MIXED, GEN>(ph, tdt, rho, chi, y, snn, sno);
      }
      if (sorted) {
        if (run) stage_slot_result<T, R>(smem_raw, A, threadIdx.x, y, scode, snn, sno);
        __syncthreads();
        if (need) stage_slot_take<T, R>(smem_raw, A, myslot, y, scode, snn, sno);
      }
      if (need) {
        code = scode;
        nn = snn;
        no = sno;
      }
    }
    if (col) {
      if (STAGE != 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) RHD_ST(A.st, A.yo[q], idx, g.ncell, y[q]);
        if (A.cost != nullptr && need)
          RHD_ST(A.st, A.cost, idx, g.ncell, cost_byte(nn, no));
      }
      if (code != RHD_OK) {
        atomicMin(&A.st->fail_key, ((unsigned long long)(A.cell_base + idx) << 8) | (unsigned)code);
        A.st->fail_step = A.step;
        A.st->fail_stage = STAGE;
      }
      ts.nn_max = max(ts.nn_max, nn);
      ts.no_max = max(ts.no_max, no);
      ts.nn_sum += nn;
      ts.no_sum += no;
      ts.cnt += (STAGE != 0 && rk2 && STAGE == 1) ? 0 : 1;
    }
    if (NDIM == 3) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        zlo[q] = zhi[q];
        hz[q] = hz1[q];
      }
      zlo_iso = zhi_iso;
    }
    __syncthreads();
  }

}

// Block reduction of TileStats (warp shuffles, then one atomic per block).
template <int NT>
__device__ __forceinline__ void flush_stats(DevStatus* st, TileStats& ts) {
  __shared__ int s_max_nn[NT / 32], s_max_no[NT / 32];
  __shared__ unsigned long long s_sum_nn[NT / 32], s_cnt[NT / 32], s_sum_no[NT / 32];
  const unsigned full = 0xffffffffu;
  int wmax_nn = __reduce_max_sync(full, ts.nn_max);
  int wmax_no = __reduce_max_sync(full, ts.no_max);
  unsigned long long nn_sum = ts.nn_sum, no_sum = ts.no_sum, cnt = ts.cnt;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    nn_sum += __shfl_down_sync(full, nn_sum, off);
    no_sum += __shfl_down_sync(full, no_sum, off);
    cnt += __shfl_down_sync(full, cnt, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_max_nn[warp] = wmax_nn;
    s_max_no[warp] = wmax_no;
    s_sum_nn[warp] = nn_sum;
    s_sum_no[warp] = no_sum;
    s_cnt[warp] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int bmn = 0, bmo = 0;
    unsigned long long bs = 0, bc = 0, bo = 0;
    for (int w = 0; w < NT / 32; ++w) {
      bmn = max(bmn, s_max_nn[w]);
      bmo = max(bmo, s_max_no[w]);
      bs += s_sum_nn[w];
      bc += s_cnt[w];
      bo += s_sum_no[w];
    }
    if (bmn > 0) atomicMax(&st->max_newton, bmn);
    if (bmo > 0) atomicMax(&st->max_outer, bmo);
    if (bs) atomicAdd(&st->sum_newton, bs);
    if (bc) atomicAdd(&st->n_solves, bc);
    if (bo) atomicAdd(&st->sum_outer, bo);
  }
}

}  // namespace rhd
