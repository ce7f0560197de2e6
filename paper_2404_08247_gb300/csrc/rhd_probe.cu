// rhd_probe.cu -- throughput probe of the fused multiply-add pipes, used to
// measure the roofline denominators of the FP64-bound stage kernels (FP64)
// and of the single-precision transport of the mixed form (FP32) on the GPU
// the library runs on.  The paper has no counterpart.
#include <cuda_runtime.h>

#include "rhd.h"
#include "rhd_internal.cuh"

namespace rhd {

constexpr int PROBE_NT = 256;     // threads per block
constexpr int PROBE_CHAINS = 8;   // independent FMA chains per thread

// written only if the chains reach a value they cannot reach, which keeps
// the compiler from removing them
static __device__ double g_probe_sink[2];

template <typename T>
__global__ void __launch_bounds__(PROBE_NT) fma_probe_kernel(T b, T c, int iters) {
  T a[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
  if (s == (T)-1.25e30) g_probe_sink[sizeof(T) == 8 ? 0 : 1] = (double)s;
}

}  // namespace rhd

extern "C" rhd_status rhd_fma_probe(int precision, int nblocks, int iters, void* stream,
                                    double* flops) {
  if (nblocks <= 0 || iters <= 0 || !flops ||
      (precision != RHD_PREC_FP64 && precision != RHD_PREC_MIXED)) {
    rhd::set_global_error("rhd_fma_probe: precision must be FP64 or MIXED, nblocks and "
                          "iters positive, flops non-null");
    return RHD_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a = a b + c with b < 1 converges to c / (1 - b) = 1: no overflow, no
  // subnormals
  if (precision == RHD_PREC_FP64)
    rhd::fma_probe_kernel<double><<<nblocks, rhd::PROBE_NT, 0, s>>>(0.999999, 1e-6, iters);
  else
    rhd::fma_probe_kernel<float><<<nblocks, rhd::PROBE_NT, 0, s>>>(0.999f, 1e-3f, iters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    rhd::set_global_error(cudaGetErrorString(e));
    return RHD_ERR_CUDA;
  }
  *flops = 2.0 * rhd::PROBE_CHAINS * (double)iters * (double)nblocks * rhd::PROBE_NT;
  return RHD_OK;
}
