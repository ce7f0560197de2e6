// rhd_stage_ppm.cu -- the stage kernels with piecewise parabolic faces
// (Sec. 3.3): the tile body of rhd_tile.cuh with a 3-cell halo and the z
// edges carried along the column, the general physics selected at run time.
#include "rhd_stage.cuh"

namespace rhd {

template <int STAGE>
static cudaError_t launch_ppm_t(int precision, const StageArgs& A, cudaStream_t s, int b0,
                                int b1) {
  if (precision == RHD_PREC_MIXED) return launch_prec<STAGE, float, true, true>(A, s, b0, b1);
  return launch_prec<STAGE, double, true, true>(A, s, b0, b1);
}

cudaError_t launch_stage_ppm(int stage, int precision, const StageArgs& A, cudaStream_t s,
                             int b0, int b1) {
  if (stage == 0) return launch_ppm_t<0>(precision, A, s, b0, b1);
  return stage == 1 ? launch_ppm_t<1>(precision, A, s, b0, b1)
                    : launch_ppm_t<2>(precision, A, s, b0, b1);
}

}  // namespace rhd
