// rhd_hydro.cu -- the hydrodynamic subsystem of Sec. 3.1 on the GPU: the
// Euler equations (rho, m, E_gas; ideal gas p = (gamma-1)(E_gas - |m|^2/2rho))
// advanced by a method of lines with RK2-SSP, the primitives reconstructed
// with the transport's option (PLM-MC, PPM or PPM with the Colella-Sekora
// limiter) and HLLC fluxes.
//
// One stage is three kinds of launch over the grid:
//   prim:   primitives w = (rho, v, p) of every cell, once (the face kernels
//           would otherwise convert each cell 2 x 3 times);
//   face:   one thread per face of one axis -- reconstruction from 4 (PLM) or
//           6 (PPM) cells along the axis, ghost cells folded in, then HLLC --
//           into a face-flux array (each flux computed once);
//   update: one thread per cell: the flux differences and the stage
//           combination, with a positivity check;
// and after stage 2 a commit copies the result into the state only if no
// cell failed, so a failed step leaves the state as it was.
#include "rhd_hydro.cuh"
#include "rhd_tile.cuh"

namespace rhd {

namespace {

constexpr int kThreads = 256;

struct Cons {
  const double* q[5];  // rho, m_x, m_y, m_z, E_gas
};

__device__ __forceinline__ bool block_skip(const DevStatus* st) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = st->fail_key != ~0ull;
  __syncthreads();
  return s_skip != 0;
}

__device__ __forceinline__ void record_fail(DevStatus* st, long long cell, int step, int stage) {
  atomicMin(&st->fail_key, ((unsigned long long)cell << 8) | (unsigned)RHD_ERR_NONPHYSICAL);
  st->fail_step = step;
  st->fail_stage = stage;
}

__global__ void __launch_bounds__(kThreads) prim_kernel(int n, double gm1, Cons U,
                                                         double* __restrict__ w, DevStatus* st,
                                                         int step, int stage, long long base) {
  if (block_skip(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double r = U.q[0][i];
    const bool rok = pos_finite(r);
    const double ri = rok ? rcp_pos(r) : 0.0;
    const double mx = U.q[1][i], my = U.q[2][i], mz = U.q[3][i];
    const double vx = mx * ri, vy = my * ri, vz = mz * ri;
    const double ke = 0.5 * (mx * vx + my * vy + mz * vz);
    const double p = gm1 * (U.q[4][i] - ke);
    if (!(rok && pos_finite(p) && finite_bits(vx) && finite_bits(vy) && finite_bits(vz)))
      record_fail(st, base + i, step, stage);
    w[i] = r;
    w[n + i] = vx;
    w[2 * n + i] = vy;
    w[3 * n + i] = vz;
    w[4 * n + i] = p;
  }
}

// Euler flux along D of the primitive state W with total energy E
template <int D>
__device__ __forceinline__ void euler_flux(const double W[5], double E, double F[5]) {
  const double u = W[1 + D];
  const double mu = W[0] * u;
  F[0] = mu;
#pragma unroll
  for (int j = 0; j < 3; ++j) F[1 + j] = mu * W[1 + j] + (j == D ? W[4] : 0.0);
  F[4] = (E + W[4]) * u;
}

// HLLC flux (Toro, Spruce & Speares 1994; Toro's book Sec. 10.4) with the
// wave-speed bounds S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L,
// u_R + a_R).  false if a face state is not physical.
template <int D>
__device__ __forceinline__ bool hllc(double g, double g1i, const double L[5], const double R[5],
                                     double F[5]) {
  if (!(pos_finite(L[0]) && pos_finite(L[4]) && pos_finite(R[0]) && pos_finite(R[4]))) {
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] = 0.0;
    return false;
  }
  const double rLi = rcp_pos(L[0]), rRi = rcp_pos(R[0]);
  const double qL = g * L[4] * rLi, qR = g * R[4] * rRi;  // a^2
  const double aL = qL * rsqrt_pos(qL), aR = qR * rsqrt_pos(qR);
  const double uL = L[1 + D], uR = R[1 + D];
  const double SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
  const double EL = L[4] * g1i + 0.5 * L[0] * (L[1] * L[1] + L[2] * L[2] + L[3] * L[3]);
  const double ER = R[4] * g1i + 0.5 * R[0] * (R[1] * R[1] + R[2] * R[2] + R[3] * R[3]);
  if (SL >= 0.0) {
    euler_flux<D>(L, EL, F);
    return true;
  }
  if (SR <= 0.0) {
    euler_flux<D>(R, ER, F);
    return true;
  }
  // contact speed; the denominator is negative (S_L - u_L <= -a_L,
  // S_R - u_R >= a_R)
  const double dL = SL - uL, dR = SR - uR;
  const double num = R[4] - L[4] + L[0] * uL * dL - R[0] * uR * dR;
  const double Ss = -num * rcp_pos(R[0] * dR - L[0] * dL);
  const bool left = Ss >= 0.0;
  const double* K = left ? L : R;
  const double SK = left ? SL : SR, dK = left ? dL : dR, EK = left ? EL : ER;
  const double rKi = left ? rLi : rRi;
  const double uK = K[1 + D];
  double FK[5];
  euler_flux<D>(K, EK, FK);
  // one reciprocal serves 1/(S_K - S*) = d_K r and 1/d_K = (S_K - S*) r,
  // r = 1/(d_K (S_K - S*)) (positive while S* lies between the bounds)
  const double sK = SK - Ss, den = dK * sK;
  const double r = pos_finite(den) ? rcp_pos(den) : 1.0 / den;
  const double fac = K[0] * dK * dK * r;
  const double Es = fac * (EK * rKi + (Ss - uK) * (Ss + K[4] * rKi * sK * r));
  F[0] = FK[0] + SK * (fac - K[0]);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double us = j == D ? Ss : K[1 + j];
    F[1 + j] = FK[1 + j] + SK * (fac * us - K[0] * K[1 + j]);
  }
  F[4] = FK[4] + SK * (Es - EK);
  return true;
}

// one thread per face of axis D: faces between cells c-1 and c along D,
// c in [0, n_D]; nf = hydro_faces(g, D).  RK: the rhd_recon of the faces
template <int D, int RK>
__global__ void __launch_bounds__(kThreads) face_kernel(const Geometry g, double gamma,
                                                         double g1i,
                                                         const double* __restrict__ w,
                                                         double* __restrict__ f, long long nf,
                                                         DevStatus* st, int step, int stage,
                                                         const double* __restrict__ hlo,
                                                         const double* __restrict__ hhi,
                                                         long long base) {
  if (block_skip(st)) return;
  constexpr int H = RK != RHD_RECON_PLM ? 3 : 2, NS = 2 * H;
  const size_t P = (size_t)g.n[0] * g.n[1];
  const int e0 = g.n[0] + (D == 0), e1 = g.n[1] + (D == 1);
  const int N = g.ncell;
  for (long long fi = (long long)blockIdx.x * blockDim.x + threadIdx.x; fi < nf;
       fi += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(fi % e0);
    const long long r = fi / e0;
    c[1] = (int)(r % e1);
    c[2] = (int)(r / e1);
    double u[5][NS];
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      // a ghost plane of a HALO z face: the neighbouring slab's primitives
      const int hs = D == 2 ? halo_side(g, c[2] - H + o) : -1;
      if (hs >= 0) {
        const int z = c[2] - H + o;
        const double* hp = (hs == 0 ? hlo + (size_t)(z + HALO_PLANES) * P
                                    : hhi + (size_t)(z - g.n[2]) * P) +
                           c[0] + (size_t)g.n[0] * c[1];
#pragma unroll
        for (int k = 0; k < 5; ++k) u[k][o] = __ldg(hp + (size_t)k * HALO_PLANES * P);
        continue;
      }
      bool flip;
      int q[3] = {c[0], c[1], c[2]};
      q[D] = fold(c[D] - H + o, g.n[D], g.bc[D][0], g.bc[D][1], flip, H - 1);
      const int idx = q[0] + g.n[0] * (q[1] + g.n[1] * q[2]);
#pragma unroll
      for (int k = 0; k < 5; ++k) u[k][o] = __ldg(w + (size_t)k * N + idx);
      if (flip) u[1 + D][o] = -u[1 + D][o];
    }
    double L[5], R[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if constexpr (RK == RHD_RECON_PPM_CS) {
        ppm_cs_face(u[k], L[k], R[k]);
      } else if constexpr (RK == RHD_RECON_PPM) {
        ppm_face(u[k], L[k], R[k]);
      } else {
        L[k] = u[k][1] + half_slope(u[k][0], u[k][1], u[k][2]);
        R[k] = u[k][2] - half_slope(u[k][1], u[k][2], u[k][3]);
      }
    }
    double F[5];
    if (!hllc<D>(gamma, g1i, L, R, F)) {
      int q[3] = {c[0], c[1], c[2]};
      q[D] = min(q[D], g.n[D] - 1);
      record_fail(st, base + q[0] + g.n[0] * (q[1] + g.n[1] * q[2]), step, stage);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) f[k * nf + fi] = F[k];
  }
}

struct Faces {
  const double* f[3];
  long long nf[3];
};

// STAGE 1: out = U + dt L;  STAGE 2: out = (U + (U1 + dt L)) / 2
template <int STAGE>
__global__ void __launch_bounds__(kThreads) update_kernel(const Geometry g, double dt, double gm1,
                                                           Cons U, const double* __restrict__ u1,
                                                           Faces F, double* __restrict__ out,
                                                           DevStatus* st, int step,
                                                           long long base) {
  if (block_skip(st)) return;
  const int N = g.ncell;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int x = i % g.n[0];
    const int rr = i / g.n[0];
    const int y = rr % g.n[1], z = rr / g.n[1];
    double rate[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= g.ndim) break;
      const int e0 = g.n[0] + (d == 0), e1 = g.n[1] + (d == 1);
      const long long lo = x + (long long)e0 * (y + (long long)e1 * z);
      const long long hi = lo + (d == 0 ? 1 : (d == 1 ? g.n[0] : (long long)g.n[0] * g.n[1]));
      const double* fd = F.f[d];
      const long long nf = F.nf[d];
#pragma unroll
      for (int k = 0; k < 5; ++k)
        rate[k] -= (__ldg(fd + k * nf + hi) - __ldg(fd + k * nf + lo)) * g.inv_dx[d];
    }
    double o[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (STAGE == 1)
        o[k] = U.q[k][i] + dt * rate[k];
      else
        o[k] = 0.5 * (U.q[k][i] + (u1[(size_t)k * N + i] + dt * rate[k]));
    }
    const double ri = pos_finite(o[0]) ? rcp_pos(o[0]) : 0.0;
    const double p = gm1 * (o[4] - 0.5 * ri * (o[1] * o[1] + o[2] * o[2] + o[3] * o[3]));
    if (!(pos_finite(o[0]) && pos_finite(p))) record_fail(st, base + i, step, 2 + STAGE);
#pragma unroll
    for (int k = 0; k < 5; ++k) out[(size_t)k * N + i] = o[k];
  }
}

// the stage-2 result into the state, unless a cell of this step failed
__global__ void __launch_bounds__(kThreads) commit_kernel(int n, const double* __restrict__ w,
                                                           double* __restrict__ rho,
                                                           double* __restrict__ y,
                                                           DevStatus* st) {
  if (block_skip(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    rho[i] = w[i];
    y[(size_t)Y_MX * n + i] = w[(size_t)n + i];
    y[(size_t)Y_MY * n + i] = w[2 * (size_t)n + i];
    y[(size_t)Y_MZ * n + i] = w[3 * (size_t)n + i];
    y[(size_t)Y_EGAS * n + i] = w[4 * (size_t)n + i];
  }
}

// Signal-speed bound of every cell in the oracle's operation order, rounded
// operation by operation (no contraction), so that the step and the number
// of radiation subcycles derived from it agree with the oracle exactly.
__global__ void __launch_bounds__(kThreads) speed_kernel(const Geometry g, double gamma,
                                                          const double* __restrict__ rho,
                                                          const double* __restrict__ y,
                                                          unsigned long long* out) {
  const int N = g.ncell;
  long long best = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double r = rho[i];
    double v[3], ke = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      v[j] = __ddiv_rn(y[(size_t)(Y_MX + j) * N + i], r);
      ke = __dadd_rn(ke, __dmul_rn(__dmul_rn(__dmul_rn(0.5, r), v[j]), v[j]));
    }
    const double p = __dmul_rn(gamma - 1.0, __dsub_rn(y[(size_t)Y_EGAS * N + i], ke));
    double s;
    if (!(r > 0.0) || !(p > 0.0)) {
      s = __longlong_as_double(kInfBits);
    } else {
      const double a = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), r));
      s = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d < g.ndim) s = __dadd_rn(s, __ddiv_rn(__dadd_rn(fabs(v[d]), a), g.dx[d]));
      if (!(s < __longlong_as_double(kInfBits))) s = __longlong_as_double(kInfBits);
    }
    best = max(best, dbits(s));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    best = max(best, (long long)__shfl_down_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)best);
}

int blocks_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <int RK>
cudaError_t launch_faces(const Geometry& g, double gamma, const double* w, const HydroBufs& b,
                         DevStatus* st, int step, int stage, cudaStream_t s) {
  const double g1i = 1.0 / (gamma - 1.0);
  for (int d = 0; d < g.ndim; ++d) {
    const long long nf = hydro_faces(g, d);
    const int nb = blocks_for(nf);
    const double *hl = b.halo[0], *hh = b.halo[1];
    const long long cb = b.cell_base;
    if (d == 0)
      face_kernel<0, RK><<<nb, kThreads, 0, s>>>(g, gamma, g1i, w, b.f[0], nf, st, step, stage,
                                                 hl, hh, cb);
    else if (d == 1)
      face_kernel<1, RK><<<nb, kThreads, 0, s>>>(g, gamma, g1i, w, b.f[1], nf, st, step, stage,
                                                 hl, hh, cb);
    else
      face_kernel<2, RK><<<nb, kThreads, 0, s>>>(g, gamma, g1i, w, b.f[2], nf, st, step, stage,
                                                 hl, hh, cb);
  }
  return cudaGetLastError();
}

}  // namespace

long long hydro_faces(const Geometry& g, int d) {
  return (long long)g.ncell / g.n[d] * (g.n[d] + 1);
}

cudaError_t launch_hydro_phase(int phase, const Geometry& g, double gamma, int recon, double dt,
                               const HydroBufs& b, DevStatus* st, int step, cudaStream_t s) {
  const int N = g.ncell;
  const int nb = blocks_for(N);
  const double gm1 = gamma - 1.0;
  const long long cb = b.cell_base;
  Cons un, c1;
  un.q[0] = b.rho;
  for (int j = 0; j < 3; ++j) un.q[1 + j] = b.y + (size_t)(Y_MX + j) * N;
  un.q[4] = b.y + (size_t)Y_EGAS * N;
  for (int k = 0; k < 5; ++k) c1.q[k] = b.u1 + (size_t)k * N;
  Faces F;
  for (int d = 0; d < 3; ++d) {
    F.f[d] = b.f[d];
    F.nf[d] = d < g.ndim ? hydro_faces(g, d) : 0;
  }
  auto faces = [&](int stage) {
    if (recon == RHD_RECON_PPM_CS)
      return launch_faces<RHD_RECON_PPM_CS>(g, gamma, b.w, b, st, step, stage, s);
    if (recon == RHD_RECON_PPM)
      return launch_faces<RHD_RECON_PPM>(g, gamma, b.w, b, st, step, stage, s);
    return launch_faces<RHD_RECON_PLM>(g, gamma, b.w, b, st, step, stage, s);
  };
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case 0:  // stage 1: U1 = U + dt L(U)
      prim_kernel<<<nb, kThreads, 0, s>>>(N, gm1, un, b.w, st, step, 3, cb);
      break;
    case 1:
      e = faces(3);
      if (e != cudaSuccess) return e;
      update_kernel<1><<<nb, kThreads, 0, s>>>(g, dt, gm1, un, nullptr, F, b.u1, st, step, cb);
      break;
    case 2:  // stage 2: U <- (U + U1 + dt L(U1)) / 2, staged in w, then committed
      prim_kernel<<<nb, kThreads, 0, s>>>(N, gm1, c1, b.w, st, step, 4, cb);
      break;
    case 3:
      e = faces(4);
      if (e != cudaSuccess) return e;
      update_kernel<2><<<nb, kThreads, 0, s>>>(g, dt, gm1, un, b.u1, F, b.w, st, step, cb);
      break;
    default:
      commit_kernel<<<nb, kThreads, 0, s>>>(N, b.w, b.rho, b.y, st);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_hydro_step(const Geometry& g, double gamma, int recon, double dt,
                              const HydroBufs& b, DevStatus* st, int step, cudaStream_t s) {
  for (int phase = 0; phase < 5; ++phase) {
    cudaError_t e = launch_hydro_phase(phase, g, gamma, recon, dt, b, st, step, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_hydro_speed(const Geometry& g, double gamma, const HydroBufs& b,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.dt_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  speed_kernel<<<blocks_for(g.ncell), kThreads, 0, s>>>(g, gamma, b.rho, b.y, b.dt_bits);
  return cudaGetLastError();
}

}  // namespace rhd
