// rhd_adjoint.cuh -- launchers of the adjoint kernels (rhd_adjoint.cu).
#pragma once

#include "rhd_tile.cuh"

namespace rhd {

// face partials per face: d/d(E, Fx, Fy, Fz) of each of the 4 stencil cells,
// then the opacity partials of the low (a) and high (b) cell
constexpr int FP_SLOTS = 18;

struct AdjointStep {
  Geometry g;
  Physics ph;
  double dt;
  int step;                 // step index (for the status block)
  const double* rho;
  const double* kappa;
  const double* yn;         // tape: y(n), y(n+1/2), y(n+1), slot-major NY * ncell each
  const double* yh;
  const double* y1;
  double* ybar;             // NY * ncell: dL/dy(n+1) in, partial dL/dy(n) out
  double* q;                // NY * ncell scratch
  double* fp;               // adjoint_scratch_doubles(g) scratch
  double* kbar;             // ncell, accumulated
  bool pending_fp;          // fp holds face partials still owed to ybar and kbar
  DevStatus* st;
};

long long adjoint_scratch_doubles(const Geometry& g);
cudaError_t launch_adjoint_step(const AdjointStep& S, cudaStream_t s);
cudaError_t launch_adjoint_finish(const AdjointStep& S, cudaStream_t s);

}  // namespace rhd
