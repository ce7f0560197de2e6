// rhd_noalloc.cu -- one IMEX step without any device allocation.
//
// rhd_step_noalloc runs the same two stage kernels as rhd_step, but on
// caller-owned input and output buffers, with the stage buffer y(n+1/2) and
// the status block in file-scope device arrays instead of memory from
// cudaMalloc.  It is meant for callers that cannot allocate: code whose device
// memory is entirely owned by another allocator (a framework's caching pool),
// or that must not call cudaMalloc/cudaFree because those calls can
// synchronise the whole device.
//
// The arrays exist once per device for the life of the process and every call
// shares them: a call clears the status block before use and overwrites the
// whole stage buffer, but two calls that overlap on the GPU (different
// streams, or different host threads) race on both.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rhd_internal.cuh"

using namespace rhd;

namespace {

// largest grid this entry point accepts: 2^18 cells (16 MiB of stage buffer)
constexpr int kMaxCells = RHD_NOALLOC_MAX_CELLS;

static __device__ __align__(256) double g_stage_scratch[(size_t)kMaxCells * NY];
static __device__ __align__(256) DevStatus g_noalloc_status;

struct DeviceSymbols {
  bool ready = false;
  double* scratch = nullptr;
  DevStatus* status = nullptr;
};

constexpr int kMaxDevices = 64;
DeviceSymbols g_symbols[kMaxDevices];
std::mutex g_symbols_mutex;
rhd_status noalloc_fail(rhd_status s, const char* msg) {
  set_global_error(msg);
  return s;
}

// Device addresses of the file-scope arrays for the current device.  In host
// code the array names are host-side stand-ins, not device addresses, so the
// kernels are given what cudaGetSymbolAddress returns.  Resolved once per
// device, on the first call made with that device current, and kept for the
// life of the process: a cudaDeviceReset of that device invalidates them.
rhd_status resolve_symbols(int dev, DeviceSymbols*& out) {
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(RHD_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_symbols_mutex);
  DeviceSymbols& s = g_symbols[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_stage_scratch);
    if (e != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
    s.scratch = static_cast<double*>(p);
    e = cudaGetSymbolAddress(&p, g_noalloc_status);
    if (e != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
    s.status = static_cast<DevStatus*>(p);
    s.ready = true;
  }
  out = &s;
  return RHD_OK;
}

void fill(const rhd_params* p, Geometry& g, Physics& ph) { rhd::fill_geometry(p, g, ph); }

// ABI field -> evolved slot (the ABI orders rho, m, Egas, E, F, kappa)
const int kSlotField[NY] = {RHD_F_EGAS, RHD_F_MX, RHD_F_MY, RHD_F_MZ,
                            RHD_F_ERAD, RHD_F_FX, RHD_F_FY, RHD_F_FZ};

}  // namespace

extern "C" rhd_status rhd_step_noalloc(const rhd_params* p, const double* state_in,
                                       double* state_out, double dt, void* stream,
                                       rhd_step_info* info) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->fail_cell = -1;
    info->fail_step = -1;
  }
  char msg[200];
  if (rhd_params_validate(p, msg, sizeof(msg)) != RHD_OK)
    return noalloc_fail(RHD_ERR_ARG, msg);
  if (p->bc[2][0] == RHD_BC_HALO || p->bc[2][1] == RHD_BC_HALO)
    return noalloc_fail(RHD_ERR_ARG, "a grid with a HALO face steps through rhd_step_slabs");
  const int64_t ncell64 = p->n[0] * p->n[1] * p->n[2];
  if (ncell64 > kMaxCells) {
    snprintf(msg, sizeof(msg),
             "grid of %lld cells exceeds the no-allocation limit of %d cells",
             (long long)ncell64, kMaxCells);
    return noalloc_fail(RHD_ERR_ARG, msg);
  }
  if (!state_in || !state_out) return noalloc_fail(RHD_ERR_ARG, "state buffer is NULL");
  const int N = (int)ncell64;
  const size_t bytes = sizeof(double) * RHD_NFIELDS * (size_t)N;
  const char* a = reinterpret_cast<const char*>(state_in);
  const char* b = reinterpret_cast<const char*>(state_out);
  if (a < b + bytes && b < a + bytes)
    return noalloc_fail(RHD_ERR_ARG, "state_in and state_out overlap");
  if (!(dt > 0.0)) dt = rhd_default_dt(p);
  if (!std::isfinite(dt)) return noalloc_fail(RHD_ERR_ARG, "dt is not finite");
  if (!(dt > 0.0)) return noalloc_fail(RHD_ERR_ARG, "dt is not positive");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
  DeviceSymbols* sym = nullptr;
  rhd_status rs = resolve_symbols(dev, sym);
  if (rs != RHD_OK) return rs;

  cudaStream_t s = (cudaStream_t)stream;
  StageArgs A;
  A.cell_base = 0;
  fill(p, A.g, A.ph);
  A.dt = dt;
  A.step = 0;
  A.rho = state_in + (size_t)RHD_F_RHO * N;
  A.kappa = state_in + (size_t)RHD_F_KAPPA * N;
  A.st = sym->status;
  for (int d = 0; d < 3; ++d) A.eps[d] = nullptr;  // TAU factors from kappa, rho on the fly
  for (int q = 0; q < 4; ++q) A.rate[q] = nullptr;
  for (int q = 0; q < NY; ++q) {
    A.yt[q] = state_in + (size_t)kSlotField[q] * N;
    A.yn[q] = A.yt[q];
    A.yo[q] = sym->scratch + (size_t)q * N;
  }
  if ((e = launch_status_reset(sym->status, s)) != cudaSuccess)
    return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
  if ((e = launch_stage(1, p->precision, A, s)) != cudaSuccess)
    return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
  for (int q = 0; q < NY; ++q) {
    A.yt[q] = sym->scratch + (size_t)q * N;
    A.yo[q] = state_out + (size_t)kSlotField[q] * N;
  }
  if ((e = launch_stage(2, p->precision, A, s)) != cudaSuccess)
    return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
  const int statics[2] = {RHD_F_RHO, RHD_F_KAPPA};
  for (int f : statics) {
    e = cudaMemcpyAsync(state_out + (size_t)f * N, state_in + (size_t)f * N,
                        sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));
  }
  DevStatus st;
  e = cudaMemcpyAsync(&st, sym->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(RHD_ERR_CUDA, cudaGetErrorString(e));

  rhd_status code = RHD_OK;
  int64_t cell = -1;
  if (st.fail_key != ~0ull) {
    code = (rhd_status)(st.fail_key & 0xffull);
    cell = (int64_t)(st.fail_key >> 8);
  }
  if (info) {
    info->status = code;
    info->steps_done = code == RHD_OK ? 1 : 0;
    info->fail_cell = cell;
    info->fail_step = code == RHD_OK ? -1 : 0;
    info->fail_stage = code == RHD_OK ? 0 : st.fail_stage;
    info->max_newton = st.max_newton;
    info->max_outer = st.max_outer;
    info->sum_newton = (int64_t)st.sum_newton;
    info->n_solves = (int64_t)st.n_solves;
    info->sum_outer = (int64_t)st.sum_outer;
    info->t = code == RHD_OK ? dt : 0.0;
    info->dt = dt;
  }
  if (code != RHD_OK) {
    snprintf(msg, sizeof(msg), "stage %d failed at cell %lld (status %d)", st.fail_stage,
             (long long)cell, (int)code);
    return noalloc_fail(code, msg);
  }
  return RHD_OK;
}
