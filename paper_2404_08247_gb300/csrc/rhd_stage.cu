// rhd_stage.cu -- the two stage kernels of one IMEX PD-ARS step on one grid.
//
// Stage 1 (eq. imex1):  y* = y(n) + dt s(y(n)),       y(n+1/2) = y* + dt f(y(n+1/2))
// Stage 2 (eq. imex2):  y** = (y(n) + y(n+1/2))/2 + dt s(y(n+1/2))/2,
//                       y(n+1) = y** + (dt/2) f(y(n+1))
// The stage-2 explicit state is eq. (imex2) with dt f(y(n+1/2)) replaced by
// y(n+1/2) - y*, which eq. (imex1) makes exact.  One block per tile; the tile
// body is stage_tile (rhd_tile.cuh).
#include "rhd_tile.cuh"

namespace rhd {

template <int STAGE, int NDIM, typename R, bool GEN>
__global__ void __launch_bounds__(Tile<NDIM>::NT, 2) stage_kernel(const StageArgs A) {
  using T = Tile<NDIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (A.st->fail_key != ~0ull) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // a previous launch of this batch failed
  TileStats ts;
  stage_tile<STAGE, T, R, GEN>(A, blockIdx.x * T::TX, blockIdx.y * T::TY, blockIdx.z * T::LZ,
                          smem_raw, ts);
  flush_stats<T::NT>(A.st, ts);
}

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
                               double* e1, double* e2) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ncell) return;
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
    double tau = 0.5 * (chi_a + kappa[nb] * rho[nb]) * g.dx[d];
    out[d][idx] = tau_factor(tau * tau_scale);
  }
}

cudaError_t launch_tau_eps(const Geometry& g, const double* rho, const double* kappa,
                           double tau_scale, double* const eps[3], cudaStream_t s) {
  int blocks = (g.ncell + 255) / 256;
  tau_eps_kernel<<<blocks, 256, 0, s>>>(g, rho, kappa, tau_scale, eps[0], eps[1], eps[2]);
  return cudaGetLastError();
}

template <int STAGE, int NDIM, typename R, bool GEN>
static cudaError_t launch_nd(const StageArgs& A, cudaStream_t s) {
  using T = Tile<NDIM>;
  using S = SmemT<T, R>;
  // opt in to more than 48 KiB of dynamic shared memory (idempotent)
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<STAGE, NDIM, R, GEN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((A.g.n[0] + T::TX - 1) / T::TX, (A.g.n[1] + T::TY - 1) / T::TY,
            (A.g.n[2] + T::LZ - 1) / T::LZ);
  stage_kernel<STAGE, NDIM, R, GEN><<<grid, T::TX * T::TY, S::BYTES, s>>>(A);
  return cudaGetLastError();
}

template <int STAGE, typename R, bool GEN>
static cudaError_t launch_prec(const StageArgs& A, cudaStream_t s) {
  switch (A.g.ndim) {
    case 1: return launch_nd<STAGE, 1, R, GEN>(A, s);
    case 2: return launch_nd<STAGE, 2, R, GEN>(A, s);
    default: return launch_nd<STAGE, 3, R, GEN>(A, s);
  }
}

// The lean kernels (GEN = false) serve the default physics; RK2-SSP, a
// temperature-dependent opacity or an inflow face select the general ones.
template <int STAGE>
static cudaError_t launch_stage_t(int precision, const StageArgs& A, cudaStream_t s) {
  const bool gen = needs_general(A.g, A.ph);
  if (precision == RHD_PREC_MIXED)
    return gen ? launch_prec<STAGE, float, true>(A, s) : launch_prec<STAGE, float, false>(A, s);
  return gen ? launch_prec<STAGE, double, true>(A, s) : launch_prec<STAGE, double, false>(A, s);
}

cudaError_t launch_stage(int stage, int precision, const StageArgs& A, cudaStream_t s) {
  if (stage == 0) return launch_stage_t<0>(precision, A, s);
  return stage == 1 ? launch_stage_t<1>(precision, A, s) : launch_stage_t<2>(precision, A, s);
}

}  // namespace rhd
