// rhd_stage.cuh -- the stage kernel of one grid and its launch, shared by
// the PLM unit (rhd_stage.cu) and the PPM unit (rhd_stage_ppm.cu), which
// compile in parallel.
#pragma once

#include <type_traits>

#include "rhd_tile.cuh"

namespace rhd {

#ifndef RHD_STAGE_MINB
#define RHD_STAGE_MINB 2  // resident blocks per SM (128 registers per thread at 256 threads)
#endif
template <int STAGE, int NDIM, typename R, bool GEN, bool PPM>
__global__ void __launch_bounds__(Tile<NDIM>::NT, NDIM == 3 ? RHD_STAGE_MINB : 2)
    stage_kernel(const StageArgs A) {
  using T = std::conditional_t<PPM, TilePPM<NDIM>, Tile<NDIM>>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (A.st->fail_key != ~0ull) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // a previous launch of this batch failed
  TileStats ts;
  stage_tile<STAGE, T, R, GEN>(A, blockIdx.x * T::TX, blockIdx.y * T::TY,
                               blockIdx.z * T::LZ, smem_raw, ts);
  flush_stats<T::NT>(A.st, ts);
}

template <int STAGE, int NDIM, typename R, bool GEN, bool PPM>
static cudaError_t launch_nd(const StageArgs& A, cudaStream_t s) {
  using T = std::conditional_t<PPM, TilePPM<NDIM>, Tile<NDIM>>;
  using S = SmemT<T, R>;
  // opt in to more than 48 KiB of dynamic shared memory (idempotent)
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<STAGE, NDIM, R, GEN, PPM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((A.g.n[0] + T::TX - 1) / T::TX, (A.g.n[1] + T::TY - 1) / T::TY,
            (A.g.n[2] + T::LZ - 1) / T::LZ);
  stage_kernel<STAGE, NDIM, R, GEN, PPM><<<grid, T::TX * T::TY, S::BYTES, s>>>(A);
  return cudaGetLastError();
}

template <int STAGE, typename R, bool GEN, bool PPM>
static cudaError_t launch_prec(const StageArgs& A, cudaStream_t s) {
  switch (A.g.ndim) {
    case 1: return launch_nd<STAGE, 1, R, GEN, PPM>(A, s);
    case 2: return launch_nd<STAGE, 2, R, GEN, PPM>(A, s);
    default: return launch_nd<STAGE, 3, R, GEN, PPM>(A, s);
  }
}

}  // namespace rhd
