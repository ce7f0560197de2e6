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
  const int bx = blockIdx.x + (NDIM == 1 ? A.blk_off : 0);
  const int by = blockIdx.y + (NDIM == 2 ? A.blk_off : 0);
  const int bz = blockIdx.z + (NDIM == 3 ? A.blk_off : 0);
  stage_tile<STAGE, T, R, GEN>(A, bx * T::TX, by * T::TY, bz * T::LZ, smem_raw, ts);
  flush_stats<T::NT>(A.st, ts);
}

// The tile rows [b0, b1) of the slowest axis (b1 < 0: all of them).
template <int STAGE, int NDIM, typename R, bool GEN, bool PPM>
static cudaError_t launch_nd(const StageArgs& A, cudaStream_t s, int b0, int b1) {
  using T = std::conditional_t<PPM, TilePPM<NDIM>, Tile<NDIM>>;
  using S = SmemT<T, R>;
  // opt in to more than 48 KiB of dynamic shared memory (idempotent)
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<STAGE, NDIM, R, GEN, PPM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)S::BYTES);
  if (e != cudaSuccess) return e;
  unsigned nb[3] = {(unsigned)((A.g.n[0] + T::TX - 1) / T::TX),
                    (unsigned)((A.g.n[1] + T::TY - 1) / T::TY),
                    (unsigned)((A.g.n[2] + T::LZ - 1) / T::LZ)};
  const int rows = (int)nb[NDIM - 1];
  if (b1 < 0 || b1 > rows) b1 = rows;
  if (b0 < 0 || b0 >= b1) return cudaErrorInvalidValue;
  nb[NDIM - 1] = (unsigned)(b1 - b0);
  StageArgs a = A;
  a.blk_off = b0;
  stage_kernel<STAGE, NDIM, R, GEN, PPM><<<dim3(nb[0], nb[1], nb[2]), T::TX * T::TY, S::BYTES,
                                           s>>>(a);
  return cudaGetLastError();
}

template <int STAGE, typename R, bool GEN, bool PPM>
static cudaError_t launch_prec(const StageArgs& A, cudaStream_t s, int b0, int b1) {
  switch (A.g.ndim) {
    case 1: return launch_nd<STAGE, 1, R, GEN, PPM>(A, s, b0, b1);
    case 2: return launch_nd<STAGE, 2, R, GEN, PPM>(A, s, b0, b1);
    default: return launch_nd<STAGE, 3, R, GEN, PPM>(A, s, b0, b1);
  }
}

}  // namespace rhd
