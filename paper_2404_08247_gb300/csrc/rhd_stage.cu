// rhd_stage.cu -- the two stage kernels of one IMEX PD-ARS step on one grid.
//
// Stage 1 (eq. imex1):  y* = y(n) + dt s(y(n)),       y(n+1/2) = y* + dt f(y(n+1/2))
// Stage 2 (eq. imex2):  y** = (y(n) + y(n+1/2))/2 + dt s(y(n+1/2))/2,
//                       y(n+1) = y** + (dt/2) f(y(n+1))
// The stage-2 explicit state is eq. (imex2) with dt f(y(n+1/2)) replaced by
// y(n+1/2) - y*, which eq. (imex1) makes exact.  One block per tile; the tile
// body is stage_tile (rhd_tile.cuh), the kernel stage_kernel (rhd_stage.cuh).
#include <algorithm>

#include "rhd_stage.cuh"

namespace rhd {

__global__ void status_reset_kernel(DevStatus* st) {
  st->fail_key = ~0ull;
  st->fail_step = -1;
  st->fail_stage = 0;
  st->max_newton = 0;
  st->max_outer = 0;
  st->sum_newton = 0;
  st->n_solves = 0;
  st->sum_outer = 0;
}

cudaError_t launch_status_reset(DevStatus* st, cudaStream_t s) {
  status_reset_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

// Optical-depth factors of every face (TAU mode): eps_d[i] belongs to the face
// between cell i and its +d neighbour (periodic wrap, or the mirror of cell i
// at a reflecting wall).  Depends on the static rho and kappa only; tau_scale
// is chi_0F / chi_0E (the face depth is that of the flux-mean opacity).
__global__ void tau_eps_kernel(const Geometry g, const double* __restrict__ rho,
                               const double* __restrict__ kappa, double tau_scale, double* e0,
                               double* e1, double* e2, const double* __restrict__ hk,
                               const double* __restrict__ hr, int i0, int i1) {
  int idx = i0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= i1) return;
  int c[3];
  c[0] = idx % g.n[0];
  int r = idx / g.n[0];
  c[1] = r % g.n[1];
  c[2] = r / g.n[1];
  double* out[3] = {e0, e1, e2};
  double chi_a = kappa[idx] * rho[idx];
  for (int d = 0; d < g.ndim; ++d) {
    bool flip;
    int xb = fold(c[d] + 1, g.n[d], g.bc[d][0], g.bc[d][1], flip);
    int nb = idx + (xb - c[d]) * g.stride[d];
    const double* kb = kappa;
    const double* rb = rho;
    if (d == 2 && c[2] == g.n[2] - 1 && g.bc[2][1] == RHD_BC_HALO) {
      // the top face of a slab: its neighbour is plane 0 of the slab above
      kb = hk;
      rb = hr;
      nb = c[0] + g.n[0] * c[1];
    }
    double tau = 0.5 * (chi_a + kb[nb] * rb[nb]) * g.dx[d];
    out[d][idx] = tau_factor(tau * tau_scale);
  }
}

cudaError_t launch_tau_eps(const Geometry& g, const double* rho, const double* kappa,
                           double tau_scale, double* const eps[3], cudaStream_t s,
                           const double* halo_kappa, const double* halo_rho, long long i0,
                           long long i1) {
  if (g.bc[2][1] == RHD_BC_HALO && (!halo_kappa || !halo_rho)) return cudaErrorInvalidValue;
  if (i1 < 0 || i1 > g.ncell) i1 = g.ncell;
  if (i0 < 0 || i0 >= i1) return cudaErrorInvalidValue;
  int blocks = (int)((i1 - i0 + 255) / 256);
  tau_eps_kernel<<<blocks, 256, 0, s>>>(g, rho, kappa, tau_scale, eps[0], eps[1], eps[2],
                                        halo_kappa, halo_rho, (int)i0, (int)i1);
  return cudaGetLastError();
}

// The lean kernels (GEN = false) serve the default physics; RK2-SSP, a
// temperature-dependent or non-grey opacity or an inflow face select the
// general ones; PPM faces the PPM unit's (general physics, wider halo).
template <int STAGE>
static cudaError_t launch_stage_t(int precision, const StageArgs& A, cudaStream_t s, int b0,
                                  int b1) {
  if (A.ph.reconstruction != RHD_RECON_PLM)
    return launch_stage_ppm(STAGE, precision, A, s, b0, b1);
  const bool gen = needs_general(A.g, A.ph);
  if (precision == RHD_PREC_MIXED)
    return gen ? launch_prec<STAGE, float, true, false>(A, s, b0, b1)
               : launch_prec<STAGE, float, false, false>(A, s, b0, b1);
  return gen ? launch_prec<STAGE, double, true, false>(A, s, b0, b1)
             : launch_prec<STAGE, double, false, false>(A, s, b0, b1);
}

cudaError_t launch_stage(int stage, int precision, const StageArgs& A, cudaStream_t s, int b0,
                         int b1) {
  if (stage == 0) return launch_stage_t<0>(precision, A, s, b0, b1);
  return stage == 1 ? launch_stage_t<1>(precision, A, s, b0, b1)
                    : launch_stage_t<2>(precision, A, s, b0, b1);
}

// Tile rows along the slowest axis, and the cells one row covers (PLM and
// PPM tiles have the same shape).
int stage_rows(const Geometry& g) {
  switch (g.ndim) {
    case 1: return (g.n[0] + Tile<1>::TX - 1) / Tile<1>::TX;
    case 2: return (g.n[1] + Tile<2>::TY - 1) / Tile<2>::TY;
    default: return (g.n[2] + Tile<3>::LZ - 1) / Tile<3>::LZ;
  }
}

long long stage_row_cells(const Geometry& g, int row) {
  const int ax = g.ndim - 1;
  const int w = g.ndim == 1 ? Tile<1>::TX : g.ndim == 2 ? Tile<2>::TY : Tile<3>::LZ;
  long long plane = 1;
  for (int d = 0; d < ax; ++d) plane *= g.n[d];
  const int lo = row * w, hi = std::min(g.n[ax], lo + w);
  return hi > lo ? plane * (hi - lo) : 0;
}

}  // namespace rhd
