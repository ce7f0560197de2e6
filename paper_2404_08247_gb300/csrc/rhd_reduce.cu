// rhd_reduce.cu -- conserved totals (Sec. 3.3) and input validation.
//
// Totals: sum over cells of (Egas + (c/chat) E) V and (m + F/(c chat)) V, the
// quantities the energy closure and the momentum update conserve.  Two passes
// with a fixed grid and fixed tree order, so the result is bit-reproducible:
// pass 1 writes one partial per block (grid-stride accumulation, warp shuffles,
// then shared memory), pass 2 reduces the partials in one block.
#include "rhd_internal.cuh"

namespace rhd {

static const int kTotBlocks = 608;  // 4 x 152 SMs
static const int kTotThreads = 256;

int totals_partials_needed() { return kTotBlocks * 4; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kTotThreads)
totals_pass1(const double* __restrict__ y, int N, double cr, double inv_cchat, double V,
             double* __restrict__ partials) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    s[0] += y[(size_t)Y_EGAS * N + i] + cr * y[(size_t)Y_ERAD * N + i];
    s[1] += y[(size_t)Y_MX * N + i] + y[(size_t)Y_FX * N + i] * inv_cchat;
    s[2] += y[(size_t)Y_MY * N + i] + y[(size_t)Y_FY * N + i] * inv_cchat;
    s[3] += y[(size_t)Y_MZ * N + i] + y[(size_t)Y_FZ * N + i] * inv_cchat;
  }
  __shared__ double sm[4][kTotThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double w = warp_sum(s[q]);
    if (lane == 0) sm[q][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double w = lane < kTotThreads / 32 ? sm[q][lane] : 0.0;
      w = warp_sum(w);
      if (lane == 0) partials[blockIdx.x * 4 + q] = w * V;
    }
  }
}

__global__ void __launch_bounds__(kTotThreads)
totals_pass2(const double* __restrict__ partials, int nb, double* __restrict__ out4) {
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += partials[b * 4 + q];
  __shared__ double sm[4][kTotThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double w = warp_sum(s[q]);
    if (lane == 0) sm[q][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double w = lane < kTotThreads / 32 ? sm[q][lane] : 0.0;
      w = warp_sum(w);
      if (lane == 0) out4[q] = w;
    }
  }
}

cudaError_t launch_totals(const Geometry& g, const Physics& ph, const double* y,
                          double* partials, int npart, double* out4, cudaStream_t s) {
  (void)npart;
  double V = 1.0;
  for (int d = 0; d < g.ndim; ++d) V *= g.dx[d];
  totals_pass1<<<kTotBlocks, kTotThreads, 0, s>>>(y, g.ncell, ph.c_over_chat,
                                                   ph.inv_cchat, V, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  totals_pass2<<<1, kTotThreads, 0, s>>>(partials, kTotBlocks, out4);
  return cudaGetLastError();
}

// Input validation: flag |= 1 for any value that is non-finite or violates
// the field's sign rule (rho > 0, Erad > 0, kappa >= 0).
__global__ void check_field_kernel(int field, const double* __restrict__ x, int n,
                                   int* flag) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = x[i];
    bool ok = isfinite(v);
    if (field == RHD_F_RHO || field == RHD_F_ERAD) ok = ok && v > 0.0;
    if (field == RHD_F_KAPPA) ok = ok && v >= 0.0;
    bad |= ok ? 0 : 1;
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_field(int field, const double* x, int n, int* flag,
                               cudaStream_t s) {
  int blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  if (blocks < 1) blocks = 1;
  check_field_kernel<<<blocks, 256, 0, s>>>(field, x, n, flag);
  return cudaGetLastError();
}

}  // namespace rhd

// ---------------------------------------------------------------- diagnostic
namespace {
__global__ void eval_recip_kernel(const double* __restrict__ x, long long n,
                                  double* __restrict__ r, double* __restrict__ q) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i];
  r[i] = rhd::rcp_pos(v);
  q[i] = rhd::rsqrt_pos(v);
}
}  // namespace

extern "C" rhd_status rhd_eval_recip(const double* x, int64_t n, double* rcp, double* rsqrt) {
  if (n < 0 || (n > 0 && (!x || !rcp || !rsqrt))) {
    rhd::set_global_error("rhd_eval_recip: bad arguments");
    return RHD_ERR_ARG;
  }
  if (n == 0) return RHD_OK;
  eval_recip_kernel<<<(unsigned)((n + 255) / 256), 256>>>(x, (long long)n, rcp, rsqrt);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rhd::set_global_error(cudaGetErrorString(e));
    return RHD_ERR_CUDA;
  }
  return RHD_OK;
}
