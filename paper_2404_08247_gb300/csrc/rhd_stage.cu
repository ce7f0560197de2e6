// rhd_stage.cu -- the two stage kernels of one IMEX PD-ARS step (FP64).
//
// Stage 1 (eq. imex1):  y* = y(n) + dt s(y(n)),       y(n+1/2) = y* + dt f(y(n+1/2))
// Stage 2 (eq. imex2):  y** = (y(n) + y(n+1/2))/2 + dt s(y(n+1/2))/2,
//                       y(n+1) = y** + (dt/2) f(y(n+1))
// The stage-2 explicit state is eq. (imex2) with dt f(y(n+1/2)) replaced by
// y(n+1/2) - y*, which eq. (imex1) makes exact.
//
// One thread per cell: the thread gathers the 5-cell stencil of E and F along
// each active axis (ghost cells by index folding: periodic wrap or mirror with
// the normal flux negated), builds both face fluxes, applies the conservative
// update and then runs the cell's local implicit solve, so the explicit state
// never leaves registers.
#include "rhd_internal.cuh"

namespace rhd {

// Neighbour of cell idx (coordinate q along axis d) at offset o, with the
// boundary condition applied; flip = the normal flux changes sign (mirror).
__device__ __forceinline__ int neighbour(const Geometry& g, int d, int q, int idx, int o,
                                         bool& flip) {
  const int n = g.n[d];
  int x = q + o;
  flip = false;
  if (x < 0) {
    if (g.bc[d][0] == RHD_BC_PERIODIC) {
      x = ((x % n) + n) % n;
    } else {
      x = -1 - x;
      flip = true;
    }
  } else if (x >= n) {
    if (g.bc[d][1] == RHD_BC_PERIODIC) {
      x = x % n;
    } else {
      x = 2 * n - 1 - x;
      flip = true;
    }
  }
  return idx + (x - q) * g.stride[d];
}

template <int STAGE, int NDIM>
__global__ void __launch_bounds__(128) stage_fp64(const StageArgs A) {
  __shared__ int s_skip;
  __shared__ int s_max_nn[4], s_max_no[4];
  __shared__ unsigned long long s_sum_nn[4], s_cnt[4], s_sum_no[4];
  if (threadIdx.x == 0) s_skip = (A.st->fail_key != ~0ull) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // a previous launch of this batch failed

  const Geometry& g = A.g;
  const Physics& ph = A.ph;
  const int N = g.ncell;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = idx < N;
  int nn = 0, no = 0, code = RHD_OK;

  if (active) {
    int coord[3];
    coord[0] = idx % g.n[0];
    int r = idx / g.n[0];
    coord[1] = r % g.n[1];
    coord[2] = r / g.n[1];

    double rate[4] = {0.0, 0.0, 0.0, 0.0};  // dE/dt, dFt/dt (Ft = F/c)
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      double c5[5][4];
      double chi3[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        bool flip;
        int nb = neighbour(g, d, coord[d], idx, o, flip);
        c5[o + 2][0] = __ldg(A.yt[Y_ERAD] + nb);
        c5[o + 2][1] = __ldg(A.yt[Y_FX] + nb) * ph.inv_c;
        c5[o + 2][2] = __ldg(A.yt[Y_FY] + nb) * ph.inv_c;
        c5[o + 2][3] = __ldg(A.yt[Y_FZ] + nb) * ph.inv_c;
        if (flip) c5[o + 2][1 + d] = -c5[o + 2][1 + d];
        if (ph.hll_mode == RHD_HLL_TAU && o >= -1 && o <= 1)
          chi3[o + 1] = __ldg(A.kappa + nb) * __ldg(A.rho + nb);
      }
      double eps_lo = 1.0, eps_hi = 1.0;
      if (ph.hll_mode == RHD_HLL_TAU) {
        eps_lo = tau_factor(0.5 * (chi3[0] + chi3[1]) * g.dx[d]);
        eps_hi = tau_factor(0.5 * (chi3[1] + chi3[2]) * g.dx[d]);
      }
      double lo[4], hi[4];
      bool ok_lo = hll_face<double>(d, c5[0], c5[1], c5[2], c5[3], eps_lo, ph.chat,
                                    ph.closure, lo);
      bool ok_hi = hll_face<double>(d, c5[1], c5[2], c5[3], c5[4], eps_hi, ph.chat,
                                    ph.closure, hi);
      if (!ok_lo || !ok_hi) code = RHD_ERR_NONPHYSICAL;
#pragma unroll
      for (int q = 0; q < 4; ++q) rate[q] -= (hi[q] - lo[q]) * g.inv_dx[d];
    }

    double y[8];
    if (STAGE == 1) {
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] = A.yt[q][idx];
      y[Y_ERAD] += A.dt * rate[0];
#pragma unroll
      for (int j = 0; j < 3; ++j) y[Y_FX + j] += A.dt * ph.c * rate[1 + j];
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        y[q] = 0.5 * (A.yn[q][idx] + A.yt[q][idx]);
      y[Y_ERAD] += 0.5 * A.dt * rate[0];
#pragma unroll
      for (int j = 0; j < 3; ++j) y[Y_FX + j] += 0.5 * A.dt * ph.c * rate[1 + j];
    }

    const double rho = A.rho[idx];
    const double chi = A.kappa[idx] * rho;
    if (code == RHD_OK)
      code = local_solve(ph, STAGE == 1 ? A.dt : 0.5 * A.dt, rho, chi, y, nn, no);
#pragma unroll
    for (int q = 0; q < 8; ++q) A.yo[q][idx] = y[q];
    if (code != RHD_OK) {
      atomicMin(&A.st->fail_key, ((unsigned long long)idx << 8) | (unsigned)code);
      A.st->fail_step = A.step;
      A.st->fail_stage = STAGE;
    }
  }

  // iteration statistics: warp, then block, then one atomic per block
  const unsigned full = 0xffffffffu;
  int wmax_nn = __reduce_max_sync(full, nn);
  int wmax_no = __reduce_max_sync(full, no);
  unsigned long long wsum = (unsigned long long)nn;
  unsigned long long wcnt = active ? 1ull : 0ull;
  unsigned long long wso = (unsigned long long)no;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    wsum += __shfl_down_sync(full, wsum, off);
    wcnt += __shfl_down_sync(full, wcnt, off);
    wso += __shfl_down_sync(full, wso, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_max_nn[warp] = wmax_nn;
    s_max_no[warp] = wmax_no;
    s_sum_nn[warp] = wsum;
    s_cnt[warp] = wcnt;
    s_sum_no[warp] = wso;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int bmn = 0, bmo = 0;
    unsigned long long bs = 0, bc = 0, bo = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      bmn = max(bmn, s_max_nn[w]);
      bmo = max(bmo, s_max_no[w]);
      bs += s_sum_nn[w];
      bc += s_cnt[w];
      bo += s_sum_no[w];
    }
    if (bmn > 0) atomicMax(&A.st->max_newton, bmn);
    if (bmo > 0) atomicMax(&A.st->max_outer, bmo);
    if (bs) atomicAdd(&A.st->sum_newton, bs);
    if (bc) atomicAdd(&A.st->n_solves, bc);
    if (bo) atomicAdd(&A.st->sum_outer, bo);
  }
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

template <int STAGE>
static cudaError_t launch_fp64(const StageArgs& A, cudaStream_t s) {
  const int block = 128;
  const int grid = (A.g.ncell + block - 1) / block;
  switch (A.g.ndim) {
    case 1: stage_fp64<STAGE, 1><<<grid, block, 0, s>>>(A); break;
    case 2: stage_fp64<STAGE, 2><<<grid, block, 0, s>>>(A); break;
    default: stage_fp64<STAGE, 3><<<grid, block, 0, s>>>(A); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_stage(int stage, int precision, const StageArgs& A, cudaStream_t s) {
  (void)precision;
  return stage == 1 ? launch_fp64<1>(A, s) : launch_fp64<2>(A, s);
}

}  // namespace rhd
