// rhd_hydro.cuh -- host launchers of the hydrodynamic subsystem (Sec. 3.1),
// defined in rhd_hydro.cu and driven by rhd_hydro_step / rhd_step_split
// (rhd_api.cu).
#pragma once

#include "rhd_internal.cuh"

namespace rhd {

// Device buffers of one hydrodynamic step of a grid: the state (rho and the
// evolved slots Egas, mx, my, mz of a state buffer), and scratch owned by the
// context: w (5 * ncell: primitives, then the stage-2 result), u1 (5 * ncell:
// the stage-1 state) and per-axis face fluxes f[d] (5 * hydro_faces(g, d)).
struct HydroBufs {
  double* rho;
  double* y;  // slot-major state buffer (slots Y_EGAS, Y_MX.. read and written)
  double* w;
  double* u1;
  double* f[3];
  unsigned long long* dt_bits;  // one word for the CFL reduction
  // RHD_BC_HALO z faces: the neighbouring slabs' primitive planes, per side
  // [5 fields rho, vx, vy, vz, p][HALO_PLANES planes][n0 n1] in z order (as
  // the radiation halo), and the index of cell 0 in the whole grid (for
  // failure reports)
  const double* halo[2] = {nullptr, nullptr};
  long long cell_base = 0;
};

// faces of axis d: (n_d + 1) per grid line
long long hydro_faces(const Geometry& g, int d);

// One RK2-SSP step of dt (Shu & Osher 1988): U1 = U + dt L(U),
// U <- (U + U1 + dt L(U1)) / 2, L the HLLC finite-volume rate of the Euler
// equations with the reconstruction `recon`.  The result is committed to the
// state only if no cell failed; a failure is recorded in st (stage 3 or 4 for
// the hydrodynamic stages 1 and 2, step index `step`) and later launches of
// the same status block skip their work.
cudaError_t launch_hydro_step(const Geometry& g, double gamma, int recon, double dt,
                              const HydroBufs& b, DevStatus* st, int step, cudaStream_t s);

// The same step in five phases, so that z-slabs can exchange primitive
// planes between them and commit only once every slab has its stage 2: 0:
// primitives of U into w; 1: face fluxes of w and U1 = U + dt L into u1; 2:
// primitives of U1 into w; 3: face fluxes of w and the stage-2 combination,
// staged in w; 4: the commit (skipped after a failure).
cudaError_t launch_hydro_phase(int phase, const Geometry& g, double gamma, int recon, double dt,
                               const HydroBufs& b, DevStatus* st, int step, cudaStream_t s);

// max over cells of sum_d (|v_d| + a)/dx_d as the bit pattern of a
// non-negative double in *b.dt_bits (0 first); a nonphysical cell gives +inf.
cudaError_t launch_hydro_speed(const Geometry& g, double gamma, const HydroBufs& b,
                               cudaStream_t s);

}  // namespace rhd
