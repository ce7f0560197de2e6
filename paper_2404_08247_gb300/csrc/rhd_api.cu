// rhd_api.cu -- the C ABI declared in include/rhd.h.
//
// A context owns the device state of one grid: two ping-pong copies of the
// eight evolved fields (y(n) and y(n+1)), the stage buffer y(n+1/2), the static
// rho and kappa, a status block and the totals scratch.  A step enqueues two
// kernels; nothing waits on the host until rhd_sync/rhd_step reads the status
// block once per batch.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rhd_adjoint.cuh"
#include "rhd_hydro.cuh"
#include "rhd_internal.cuh"

using namespace rhd;

namespace {

struct Rec {
  cudaEvent_t a, b;
  int kind;
};

thread_local char g_err[512] = "";

void set_msg(char* buf, const char* fmt, va_list ap) {
  vsnprintf(buf, 512, fmt, ap);
}

}  // namespace

struct rhd_ctx {
  rhd_params p;
  int device = 0;
  int ncell = 0;
  Geometry g;
  Physics ph;
  double* ybuf[2] = {nullptr, nullptr};
  double* yhalf = nullptr;
  double* rho = nullptr;
  double* kappa = nullptr;
  double* eps[3] = {nullptr, nullptr, nullptr};  // TAU-mode face factors
  bool eps_dirty = true;
  // each cell's solve cost in stage 1 and stage 2 of the last step (2 ncell
  // bytes): the order of the next step's solves
  unsigned char* cost = nullptr;
  DevStatus* d_status = nullptr;
  DevStatus* h_status = nullptr;
  double* d_partials = nullptr;
  double* d_tot = nullptr;
  double* h_tot = nullptr;
  int* d_flag = nullptr;
  int* h_flag = nullptr;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  int cur = 0;
  unsigned fields_set = 0;
  double t = 0.0;
  bool pending = false;
  int pending_n = 0;
  double pending_dt = 0.0;
  int pending_cur0 = 0;
  int64_t launches = 0;
  char err[512] = "";
  bool prof = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double* adj_q = nullptr;   // adjoint scratch, allocated by the first rhd_adjoint
  double* adj_fp = nullptr;
  double* hyd_w = nullptr;   // hydrodynamic scratch, allocated by the first hydro call
  double* hyd_u1 = nullptr;
  double* hyd_f[3] = {nullptr, nullptr, nullptr};
  unsigned long long* hyd_bits = nullptr;
  // HALO faces: the neighbours' ghost planes (2 sides x 4 fields x
  // HALO_PLANES planes), plane 0 of the slab above (kappa, rho) and the TAU
  // factors of the low face; allocated by the first rhd_step_slabs
  double* halo = nullptr;
  double* hyd_halo = nullptr;  // the same for the primitives (2 x 5 x HALO_PLANES planes)
  // a slab stepped stage by stage by its own process (rhd_slab_stage): 0 idle,
  // 1 after stage 1, 2 after stage 2, 3 status read; the step's dt; whether
  // the neighbours' material plane (top face) and TAU factors (bottom face)
  // are set for the current rho and kappa
  int slab_phase = 0;
  double slab_dt = 0.0;
  bool slab_mat_above = false;
  bool slab_eps_below = false;
  // rhd_step_host: its two copy streams and six compute streams (priority
  // falling from the first), and its events (timing disabled), created by
  // the first call
  cudaStream_t hs[8] = {};
  std::vector<cudaEvent_t> hev;
};

// a context whose grid is a z-slab of a decomposed grid
static bool has_halo(const rhd_ctx* c) {
  return c->p.bc[2][0] == RHD_BC_HALO || c->p.bc[2][1] == RHD_BC_HALO;
}
static const int kHaloSlots = 2 * 4 * HALO_PLANES + 3;  // planes of n0 n1 doubles
static const char* const kHaloOnly =
    "a context with a HALO face steps through rhd_step_slabs only";

static rhd_status fail(rhd_ctx* c, rhd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  set_msg(c ? c->err : g_err, fmt, ap);
  va_end(ap);
  if (c) memcpy(g_err, c->err, sizeof(g_err));
  return s;
}

void rhd::set_global_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

#define CUDA_TRY(ctx, call)                                                       \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail((ctx), RHD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static const unsigned kAllFields = (1u << RHD_NFIELDS) - 1u;

// evolved-field slot of an ABI field, -1 for the static ones
static int slot_of(int field) {
  switch (field) {
    case RHD_F_EGAS: return Y_EGAS;
    case RHD_F_MX: return Y_MX;
    case RHD_F_MY: return Y_MY;
    case RHD_F_MZ: return Y_MZ;
    case RHD_F_ERAD: return Y_ERAD;
    case RHD_F_FX: return Y_FX;
    case RHD_F_FY: return Y_FY;
    case RHD_F_FZ: return Y_FZ;
    default: return -1;
  }
}

static double* field_ptr(rhd_ctx* c, int field) {
  if (field == RHD_F_RHO) return c->rho;
  if (field == RHD_F_KAPPA) return c->kappa;
  return c->ybuf[c->cur] + (size_t)slot_of(field) * c->ncell;
}

extern "C" {

void rhd_params_default(rhd_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->ndim = 1;
  for (int d = 0; d < 3; ++d) {
    p->n[d] = 1;
    p->dx[d] = 1.0;
    p->bc[d][0] = p->bc[d][1] = RHD_BC_PERIODIC;
  }
  p->gamma = 5.0 / 3.0;
  p->c = 1.0;
  p->chat = 1.0;
  p->a_rad = 1.0;
  p->kB_over_mu = 1.0;
  p->cfl = 0.4;
  p->closure = RHD_CLOSURE_M1;
  p->vc_order = 2;
  p->hll_mode = RHD_HLL_TAU;
  p->precision = RHD_PREC_FP64;
  p->newton_rtol = 1e-13;
  p->outer_rtol = 1e-13;
  p->newton_max_iter = 64;
  p->outer_max_iter = 32;
  p->scheme = RHD_SCHEME_IMEX_PDARS;
  p->kappa_T_exp = 0.0;
  p->kappa_T_ref = 1.0;
  p->kappa_P_ratio = 1.0;
  p->kappa_F_ratio = 1.0;
  p->reconstruction = RHD_RECON_PLM;
  p->cfl_hydro = 0.3;
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      p->bc_state[d][s][0] = 1.0;
      p->bc_state[d][s][1] = p->bc_state[d][s][2] = p->bc_state[d][s][3] = 0.0;
    }
}

static int bad(char* msg, int len, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, (size_t)len, fmt, ap);
    va_end(ap);
  }
  return 1;
}

rhd_status rhd_params_validate(const rhd_params* p, char* msg, int msglen) {
  if (msg && msglen > 0) msg[0] = 0;
  if (!p) return bad(msg, msglen, "params is NULL"), RHD_ERR_ARG;
  if (p->ndim < 1 || p->ndim > 3)
    return bad(msg, msglen, "ndim must be 1, 2 or 3 (got %d)", p->ndim), RHD_ERR_ARG;
  long double cells = 1;
  for (int d = 0; d < 3; ++d) {
    if (d < p->ndim) {
      if (p->n[d] < 1)
        return bad(msg, msglen, "n[%d] must be >= 1", d), RHD_ERR_ARG;
      if (!(p->dx[d] > 0.0) || !std::isfinite(p->dx[d]))
        return bad(msg, msglen, "dx[%d] must be positive and finite", d), RHD_ERR_ARG;
      for (int s = 0; s < 2; ++s) {
        if (p->bc[d][s] != RHD_BC_PERIODIC && p->bc[d][s] != RHD_BC_REFLECT &&
            p->bc[d][s] != RHD_BC_INFLOW && p->bc[d][s] != RHD_BC_HALO)
          return bad(msg, msglen, "bc[%d][%d] is not an rhd_bc", d, s), RHD_ERR_ARG;
        if (p->bc[d][s] == RHD_BC_HALO && (p->ndim != 3 || d != 2))
          return bad(msg, msglen, "HALO faces are z faces of a 3-D grid (bc[%d][%d])", d, s),
                 RHD_ERR_ARG;
        if (p->bc[d][s] == RHD_BC_HALO && p->n[d] < HALO_PLANES)
          return bad(msg, msglen, "a HALO face needs n[2] >= %d", HALO_PLANES), RHD_ERR_ARG;
        if (p->bc[d][s] != RHD_BC_PERIODIC && p->n[d] < 2)
          return bad(msg, msglen, "a reflecting or inflow axis %d needs n >= 2", d),
                 RHD_ERR_ARG;
        if (p->bc[d][s] == RHD_BC_INFLOW) {
          const double* st = p->bc_state[d][s];
          if (!(st[0] > 0.0) || !std::isfinite(st[0]) || !std::isfinite(st[1]) ||
              !std::isfinite(st[2]) || !std::isfinite(st[3]))
            return bad(msg, msglen, "bc_state[%d][%d] needs E > 0 and finite F", d, s),
                   RHD_ERR_ARG;
        }
      }
      if ((p->bc[d][0] == RHD_BC_PERIODIC) != (p->bc[d][1] == RHD_BC_PERIODIC))
        return bad(msg, msglen, "axis %d: periodic must apply to both faces", d),
               RHD_ERR_ARG;
    } else if (p->n[d] != 1) {
      return bad(msg, msglen, "n[%d] must be 1 for ndim = %d", d, p->ndim), RHD_ERR_ARG;
    }
    cells *= (long double)p->n[d];
  }
  if (cells > 2147483647.0L)
    return bad(msg, msglen, "grid has more than 2^31-1 cells"), RHD_ERR_ARG;
  if (!(p->gamma > 1.0) || !std::isfinite(p->gamma))
    return bad(msg, msglen, "gamma must be > 1"), RHD_ERR_ARG;
  if (!(p->c > 0.0) || !std::isfinite(p->c))
    return bad(msg, msglen, "c must be positive and finite"), RHD_ERR_ARG;
  if (!(p->chat > 0.0) || !(p->chat <= p->c))
    return bad(msg, msglen, "chat must satisfy 0 < chat <= c"), RHD_ERR_ARG;
  if (!(p->a_rad > 0.0) || !std::isfinite(p->a_rad))
    return bad(msg, msglen, "a_rad must be positive"), RHD_ERR_ARG;
  if (!(p->kB_over_mu > 0.0) || !std::isfinite(p->kB_over_mu))
    return bad(msg, msglen, "kB_over_mu must be positive"), RHD_ERR_ARG;
  if (!(p->cfl > 0.0) || !std::isfinite(p->cfl))
    return bad(msg, msglen, "cfl must be positive"), RHD_ERR_ARG;
  if (p->closure != RHD_CLOSURE_M1 && p->closure != RHD_CLOSURE_EDDINGTON)
    return bad(msg, msglen, "closure is not an rhd_closure"), RHD_ERR_ARG;
  if (p->vc_order != 1 && p->vc_order != 2)
    return bad(msg, msglen, "vc_order must be 1 or 2"), RHD_ERR_ARG;
  if (p->hll_mode != RHD_HLL_TAU && p->hll_mode != RHD_HLL_NONE)
    return bad(msg, msglen, "hll_mode is not an rhd_hll_mode"), RHD_ERR_ARG;
  if (p->precision != RHD_PREC_FP64 && p->precision != RHD_PREC_MIXED)
    return bad(msg, msglen, "precision is not an rhd_precision"), RHD_ERR_ARG;
  if (!(p->newton_rtol > 0.0) || !(p->outer_rtol >= 0.0))
    return bad(msg, msglen, "tolerances must be positive"), RHD_ERR_ARG;
  if (p->newton_max_iter < 1 || p->outer_max_iter < 1)
    return bad(msg, msglen, "iteration bounds must be >= 1"), RHD_ERR_ARG;
  if (p->scheme != RHD_SCHEME_IMEX_PDARS && p->scheme != RHD_SCHEME_RK2_SSP)
    return bad(msg, msglen, "scheme is not an rhd_scheme"), RHD_ERR_ARG;
  if (!std::isfinite(p->kappa_T_exp) || !(p->kappa_T_ref > 0.0) ||
      !std::isfinite(p->kappa_T_ref))
    return bad(msg, msglen, "kappa_T_exp must be finite and kappa_T_ref > 0"), RHD_ERR_ARG;
  if (!(p->kappa_P_ratio > 0.0) || !std::isfinite(p->kappa_P_ratio) ||
      !(p->kappa_F_ratio > 0.0) || !std::isfinite(p->kappa_F_ratio))
    return bad(msg, msglen, "kappa_P_ratio and kappa_F_ratio must be positive"),
           RHD_ERR_ARG;
  if (!(p->cfl_hydro > 0.0) || !std::isfinite(p->cfl_hydro))
    return bad(msg, msglen, "cfl_hydro must be positive"), RHD_ERR_ARG;
  if (p->reconstruction != RHD_RECON_PLM && p->reconstruction != RHD_RECON_PPM &&
      p->reconstruction != RHD_RECON_PPM_CS)
    return bad(msg, msglen, "reconstruction is not an rhd_recon"), RHD_ERR_ARG;
  if (p->reconstruction != RHD_RECON_PLM)
    for (int d = 0; d < p->ndim; ++d)
      if (p->bc[d][0] != RHD_BC_PERIODIC && p->n[d] < 3)
        return bad(msg, msglen, "PPM on a reflecting or inflow axis %d needs n >= 3", d),
               RHD_ERR_ARG;
  if (p->kappa_T_exp != 0.0 && p->hll_mode != RHD_HLL_NONE)
    return bad(msg, msglen, "a temperature-dependent opacity needs hll_mode NONE"),
           RHD_ERR_ARG;
  return RHD_OK;
}

double rhd_default_dt(const rhd_params* p) {
  if (rhd_params_validate(p, nullptr, 0) != RHD_OK) return -1.0;
  double s = 0.0;
  for (int d = 0; d < p->ndim; ++d) s += 1.0 / p->dx[d];
  return p->cfl / (p->chat * s);
}

}  // extern "C"

// Device-side geometry and physics of validated params (shared by the
// single-grid, batched and no-allocation paths).
void rhd::fill_geometry(const rhd_params* p, Geometry& g, Physics& ph) {
  memset(&g, 0, sizeof(g));
  g.ndim = p->ndim;
  int stride = 1;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = (int)p->n[d];
    g.stride[d] = stride;
    stride *= g.n[d];
    g.dx[d] = p->dx[d];
    g.inv_dx[d] = 1.0 / p->dx[d];
    g.bc[d][0] = p->bc[d][0];
    g.bc[d][1] = p->bc[d][1];
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 4; ++q) g.bc_state[d][s][q] = p->bc_state[d][s][q];
  }
  g.ncell = stride;
  memset(&ph, 0, sizeof(ph));
  ph.c = p->c;
  ph.chat = p->chat;
  ph.a_rad = p->a_rad;
  ph.cv_spec = p->kB_over_mu / (p->gamma - 1.0);
  ph.inv_c = 1.0 / p->c;
  ph.c_over_chat = p->c / p->chat;
  ph.chat_over_c = p->chat / p->c;
  ph.inv_c2 = 1.0 / (p->c * p->c);
  ph.inv_cchat = 1.0 / (p->c * p->chat);
  ph.closure = p->closure;
  ph.vc_order = p->vc_order;
  ph.hll_mode = p->hll_mode;
  ph.newton_rtol = p->newton_rtol;
  ph.outer_rtol = p->outer_rtol;
  ph.newton_max = p->newton_max_iter;
  ph.outer_max = p->outer_max_iter;
  ph.scheme = p->scheme;
  ph.kappa_T_exp = p->kappa_T_exp;
  ph.inv_kappa_T_ref = 1.0 / p->kappa_T_ref;
  ph.kappa_P_ratio = p->kappa_P_ratio;
  ph.kappa_F_ratio = p->kappa_F_ratio;
  ph.reconstruction = p->reconstruction;
}

static void release(rhd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  for (auto e : c->hev) cudaEventDestroy(e);
  for (auto h : c->hs)
    if (h) cudaStreamDestroy(h);
  cudaFree(c->ybuf[0]);
  cudaFree(c->ybuf[1]);
  cudaFree(c->yhalf);
  cudaFree(c->rho);
  cudaFree(c->kappa);
  for (int d = 0; d < 3; ++d) cudaFree(c->eps[d]);
  cudaFree(c->cost);
  cudaFree(c->d_status);
  cudaFree(c->d_partials);
  cudaFree(c->d_tot);
  cudaFree(c->d_flag);
  cudaFree(c->adj_q);
  cudaFree(c->adj_fp);
  cudaFree(c->hyd_w);
  cudaFree(c->hyd_u1);
  for (int d = 0; d < 3; ++d) cudaFree(c->hyd_f[d]);
  cudaFree(c->hyd_bits);
  cudaFree(c->halo);
  cudaFree(c->hyd_halo);
  cudaFreeHost(c->h_status);
  cudaFreeHost(c->h_tot);
  cudaFreeHost(c->h_flag);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

static cudaEvent_t take_event(rhd_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void recycle_records(rhd_ctx* c) {
  for (auto& r : c->recs) {
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
}

extern "C" {

rhd_status rhd_init(const rhd_params* p, rhd_ctx** out) {
  if (!out) return fail(nullptr, RHD_ERR_ARG, "out is NULL");
  *out = nullptr;
  char msg[256];
  if (rhd_params_validate(p, msg, sizeof(msg)) != RHD_OK)
    return fail(nullptr, RHD_ERR_ARG, "invalid params: %s", msg);
  rhd_ctx* c = new rhd_ctx();
  c->p = *p;
  fill_geometry(p, c->g, c->ph);
  c->ncell = c->g.ncell;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    fail(nullptr, RHD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    delete c;
    return RHD_ERR_CUDA;
  }
  const size_t N = (size_t)c->ncell;
  const size_t ybytes = sizeof(double) * NY * N;
  e = cudaMalloc(&c->ybuf[0], ybytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->ybuf[1], ybytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->yhalf, ybytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->rho, sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMalloc(&c->kappa, sizeof(double) * N);
  if (p->hll_mode == RHD_HLL_TAU)
    for (int d = 0; d < p->ndim && e == cudaSuccess; ++d)
      e = cudaMalloc(&c->eps[d], sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMalloc(&c->cost, 2 * N);
  if (e == cudaSuccess) e = cudaMemset(c->cost, 0, 2 * N);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(DevStatus));
  if (e == cudaSuccess)
    e = cudaMalloc(&c->d_partials, sizeof(double) * totals_partials_needed());
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tot, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_tot, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fail(nullptr, RHD_ERR_CUDA, "allocating %zu bytes of device state: %s",
         3 * ybytes + 2 * sizeof(double) * N, cudaGetErrorString(e));
    release(c);
    return RHD_ERR_CUDA;
  }
  c->stream = c->own;
  *out = c;
  return RHD_OK;
}

rhd_status rhd_set_stream(rhd_ctx* c, void* s) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)s;
  return RHD_OK;
}

rhd_status rhd_use_private_stream(rhd_ctx* c) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->stream = c->own;
  return RHD_OK;
}

static rhd_status check_copy_args(rhd_ctx* c, int field, const void* ptr, int64_t count) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->slab_phase != 0) return fail(c, RHD_ERR_STATE, "a slab step is in progress");
  if (field < 0 || field >= RHD_NFIELDS) return fail(c, RHD_ERR_ARG, "bad field %d", field);
  if (!ptr) return fail(c, RHD_ERR_ARG, "buffer is NULL");
  if (count != (int64_t)c->ncell)
    return fail(c, RHD_ERR_ARG, "count %lld != ncell %d", (long long)count, c->ncell);
  return RHD_OK;
}

static rhd_status copy_in(rhd_ctx* c, int field, const double* src, int on_dev) {
  if (field == RHD_F_RHO || field == RHD_F_KAPPA) {
    c->eps_dirty = true;
    c->slab_mat_above = c->slab_eps_below = false;  // the neighbours' planes are stale
  }
  CUDA_TRY(c, cudaMemcpyAsync(field_ptr(c, field), src, sizeof(double) * c->ncell,
                              on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, launch_check_field(field, field_ptr(c, field), c->ncell, c->d_flag, c->stream));
  c->launches += 1;
  return RHD_OK;
}

rhd_status rhd_state_set(rhd_ctx* c, int field, const double* src, int64_t count,
                         int src_on_device) {
  rhd_status s = check_copy_args(c, field, src, count);
  if (s != RHD_OK) return s;
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  s = copy_in(c, field, src, src_on_device);
  if (s != RHD_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (*c->h_flag) {
    c->fields_set &= ~(1u << field);
    return fail(c, RHD_ERR_ARG, "field %d holds a non-finite or out-of-range value", field);
  }
  c->fields_set |= 1u << field;
  return RHD_OK;
}

rhd_status rhd_state_set_all(rhd_ctx* c, const double* src, int64_t count,
                             int src_on_device) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (count != (int64_t)RHD_NFIELDS * c->ncell)
    return fail(c, RHD_ERR_ARG, "count must be RHD_NFIELDS * ncell");
  rhd_status s = check_copy_args(c, 0, src, c->ncell);
  if (s != RHD_OK) return s;
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  for (int f = 0; f < RHD_NFIELDS; ++f) {
    s = copy_in(c, f, src + (size_t)f * c->ncell, src_on_device);
    if (s != RHD_OK) return s;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (*c->h_flag) {
    c->fields_set = 0;
    return fail(c, RHD_ERR_ARG, "state holds a non-finite or out-of-range value");
  }
  c->fields_set = kAllFields;
  return RHD_OK;
}

rhd_status rhd_state_get(rhd_ctx* c, int field, double* dst, int64_t count,
                         int dst_on_device) {
  rhd_status s = check_copy_args(c, field, dst, count);
  if (s != RHD_OK) return s;
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemcpyAsync(dst, field_ptr(c, field), sizeof(double) * c->ncell,
                              dst_on_device ? cudaMemcpyDeviceToDevice
                                            : cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RHD_OK;
}

rhd_status rhd_stage_get(rhd_ctx* c, int field, double* dst, int64_t count,
                         int dst_on_device) {
  rhd_status s = check_copy_args(c, field, dst, count);
  if (s != RHD_OK) return s;
  int slot = slot_of(field);
  if (slot < 0) return fail(c, RHD_ERR_ARG, "the stage buffer holds evolved fields only");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemcpyAsync(dst, c->yhalf + (size_t)slot * c->ncell,
                              sizeof(double) * c->ncell,
                              dst_on_device ? cudaMemcpyDeviceToDevice
                                            : cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RHD_OK;
}

rhd_status rhd_state_get_all(rhd_ctx* c, double* dst, int64_t count, int dst_on_device) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (count != (int64_t)RHD_NFIELDS * c->ncell)
    return fail(c, RHD_ERR_ARG, "count must be RHD_NFIELDS * ncell");
  rhd_status s = check_copy_args(c, 0, dst, c->ncell);
  if (s != RHD_OK) return s;
  CUDA_TRY(c, cudaSetDevice(c->device));
  for (int f = 0; f < RHD_NFIELDS; ++f)
    CUDA_TRY(c, cudaMemcpyAsync(dst + (size_t)f * c->ncell, field_ptr(c, f),
                                sizeof(double) * c->ncell,
                                dst_on_device ? cudaMemcpyDeviceToDevice
                                              : cudaMemcpyDeviceToHost,
                                c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RHD_OK;
}

static cudaError_t launch_recorded(rhd_ctx* c, int kind, int stage, const StageArgs& A) {
  if (!c->prof) return launch_stage(stage, c->p.precision, A, c->stream);
  Rec r;
  r.a = take_event(c);
  r.b = take_event(c);
  r.kind = kind;
  cudaEventRecord(r.a, c->stream);
  cudaError_t e = launch_stage(stage, c->p.precision, A, c->stream);
  cudaEventRecord(r.b, c->stream);
  c->recs.push_back(r);
  return e;
}

rhd_status rhd_step_async(rhd_ctx* c, int nsteps, double dt) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is already pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (has_halo(c)) return fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  if (nsteps < 0) return fail(c, RHD_ERR_ARG, "nsteps < 0");
  if (!(dt > 0.0)) dt = rhd_default_dt(&c->p);
  if (!std::isfinite(dt)) return fail(c, RHD_ERR_ARG, "dt is not finite");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
  c->launches += 1;
  if (c->p.hll_mode == RHD_HLL_TAU && c->eps_dirty) {
    CUDA_TRY(c, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps, c->stream));
    c->launches += 1;
    c->eps_dirty = false;
  }
  StageArgs A;
  A.cell_base = 0;
  for (int d = 0; d < 3; ++d) A.eps[d] = c->eps[d];
  A.g = c->g;
  A.ph = c->ph;
  A.dt = dt;
  A.rho = c->rho;
  A.kappa = c->kappa;
  A.st = c->d_status;
  int cur = c->cur;
  const int N = c->ncell;
  for (int s = 0; s < nsteps; ++s) {
    A.step = s;
    slots_of<const double*>(A.yt, c->ybuf[cur], N);
    slots_of<const double*>(A.yn, c->ybuf[cur], N);
    slots_of<double*>(A.yo, c->yhalf, N);
    A.cost = c->cost;
    CUDA_TRY(c, launch_recorded(c, 0, 1, A));
    slots_of<const double*>(A.yt, c->yhalf, N);
    slots_of<double*>(A.yo, c->ybuf[cur ^ 1], N);
    A.cost = c->cost + N;
    CUDA_TRY(c, launch_recorded(c, 1, 2, A));
    c->launches += 2;
    cur ^= 1;
  }
  c->pending = true;
  c->pending_n = nsteps;
  c->pending_dt = dt;
  c->pending_cur0 = c->cur;
  return RHD_OK;
}

rhd_status rhd_sync(rhd_ctx* c, rhd_step_info* info) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!c->pending) return fail(c, RHD_ERR_STATE, "no step batch is pending");
  CUDA_TRY(c, cudaSetDevice(c->device));
  c->pending = false;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const DevStatus& st = *c->h_status;
  const int n = c->pending_n;
  rhd_status code = RHD_OK;
  int done = n;
  int64_t cell = -1;
  if (st.fail_key != ~0ull) {
    code = (rhd_status)(st.fail_key & 0xffull);
    cell = (int64_t)(st.fail_key >> 8);
    done = st.fail_step;
  }
  c->cur = c->pending_cur0 ^ (done & 1);
  c->t += done * c->pending_dt;
  if (info) {
    info->status = code;
    info->steps_done = done;
    info->fail_cell = cell;
    info->fail_step = code == RHD_OK ? -1 : st.fail_step;
    info->fail_stage = code == RHD_OK ? 0 : st.fail_stage;
    info->max_newton = st.max_newton;
    info->max_outer = st.max_outer;
    info->sum_newton = (int64_t)st.sum_newton;
    info->n_solves = (int64_t)st.n_solves;
    info->sum_outer = (int64_t)st.sum_outer;
    info->t = c->t;
    info->dt = c->pending_dt;
  }
  if (code != RHD_OK)
    return fail(c, code, "step %d stage %d failed at cell %lld (status %d)", st.fail_step,
                st.fail_stage, (long long)cell, (int)code);
  return RHD_OK;
}

rhd_status rhd_step(rhd_ctx* c, int nsteps, double dt, rhd_step_info* info) {
  rhd_status s = rhd_step_async(c, nsteps, dt);
  if (s != RHD_OK) {
    if (info) {
      memset(info, 0, sizeof(*info));
      info->status = s;
      info->fail_cell = -1;
      info->fail_step = -1;
      info->t = c ? c->t : 0.0;
    }
    return s;
  }
  return rhd_sync(c, info);
}

// ------------------------------------------------ a step of a host-held state
// rhd_step_host: the state is copied in and out in chunks of tile rows along
// the slowest axis, so that the copies overlap the stage kernels.  A stage
// launch over rows [r0, r1) reads the cells of those rows and their ghost
// cells, at most 3 deep (the PPM stencil), so with chunks of at least 2 tile
// rows (>= 8 planes) it needs its own chunks' inputs and its two neighbour
// chunks' (cyclically: periodic faces wrap); the TAU factors of a chunk's +d
// faces need its own and the next chunk's rho and kappa.

static rhd_status host_step_fail_info(rhd_ctx* c, rhd_status s, rhd_step_info* info) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = s;
    info->fail_cell = -1;
    info->fail_step = -1;
    info->t = c ? c->t : 0.0;
  }
  return s;
}

static StageArgs host_stage_args(rhd_ctx* c, double dt, int step, int stage) {
  StageArgs A;
  A.cell_base = 0;
  for (int d = 0; d < 3; ++d) A.eps[d] = c->eps[d];
  A.g = c->g;
  A.ph = c->ph;
  A.dt = dt;
  A.rho = c->rho;
  A.kappa = c->kappa;
  A.st = c->d_status;
  A.step = step;
  const int N = c->ncell;
  const int in = c->cur ^ (step & 1);  // y(n) of this step
  if (stage == 1) {
    slots_of<const double*>(A.yt, c->ybuf[in], N);
    slots_of<const double*>(A.yn, c->ybuf[in], N);
    slots_of<double*>(A.yo, c->yhalf, N);
  } else {
    slots_of<const double*>(A.yt, c->yhalf, N);
    slots_of<const double*>(A.yn, c->ybuf[in], N);
    slots_of<double*>(A.yo, c->ybuf[in ^ 1], N);
  }
  A.cost = c->cost + (stage == 1 ? 0 : N);
  return A;
}

// The chunks and launch groups of rhd_step_host for a grid: K chunks of
// tile rows along the slowest axis (at least 2 rows each, at most 16
// chunks), rows r0[k] .. r0[k+1] and cells i0[k] .. i0[k+1]; the stage-1
// groups g1 (chunk 0, chunks 1 .. K/4 - 1, the rest) and the last stage-2
// groups g2 (chunks 1 .. K-4 in up to three, K-3 .. K-2, K-1, then 0).
struct HostPlan {
  int K = 0;
  std::vector<int> r0;
  std::vector<size_t> i0;
  std::vector<std::pair<int, int>> g1, g2;
};

static HostPlan host_step_plan(const Geometry& g) {
  HostPlan P;
  const int rows = stage_rows(g);
  const int K = std::max(1, std::min(16, rows / 2));
  P.K = K;
  P.r0.assign(K + 1, 0);
  P.i0.assign(K + 1, 0);
  for (int k = 0; k <= K; ++k) P.r0[k] = (int)((long long)k * rows / K);
  for (int k = 0; k < K; ++k) {
    size_t n = 0;
    for (int r = P.r0[k]; r < P.r0[k + 1]; ++r) n += (size_t)stage_row_cells(g, r);
    P.i0[k + 1] = P.i0[k] + n;
  }
  if (K >= 3) {
    const int q1 = std::max(2, K / 4);
    P.g1 = {{0, 1}, {1, q1}, {q1, K}};
    if (K >= 5) {
      const int nb = std::min(3, K - 4);  // groups of the body 1 .. K-4
      for (int j = 0; j < nb; ++j)
        P.g2.push_back({1 + j * (K - 4) / nb, 1 + (j + 1) * (K - 4) / nb});
      P.g2.push_back({K - 3, K - 1});
      P.g2.push_back({K - 1, K});
      P.g2.push_back({0, 1});
    } else {
      P.g2 = {{1, K - 1}, {K - 1, K}, {0, 1}};
    }
  } else if (K == 2) {
    P.g1 = {{0, 1}, {1, 2}};
    P.g2 = {{1, 2}, {0, 1}};
  } else {
    P.g1 = {{0, 1}};
    P.g2 = {{0, 1}};
  }
  return P;
}

static rhd_status host_step_enqueue(rhd_ctx* c, const double* src, double* dst, int nsteps,
                                    double dt) {
  if (!c->hs[0]) {
    int least = 0, greatest = 0;  // numerically: greatest priority <= least
    CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    for (int k = 0; k < 8; ++k) {
      const int prio = k < 2 ? least : std::min(least, greatest + (k - 2));
      CUDA_TRY(c, cudaStreamCreateWithPriority(&c->hs[k], cudaStreamNonBlocking, prio));
    }
  }
  const Geometry& g = c->g;
  const size_t N = (size_t)c->ncell;
  const HostPlan P = host_step_plan(g);
  const int K = P.K;
  const std::vector<int>& r0 = P.r0;
  const std::vector<size_t>& i0 = P.i0;
  const std::vector<std::pair<int, int>>& g1 = P.g1;
  const std::vector<std::pair<int, int>>& g2 = P.g2;
  if (i0[K] != N) return fail(c, RHD_ERR_STATE, "chunks cover %zu of %zu cells", i0[K], N);
  const int nev = 5 * K + 10;
  while ((int)c->hev.size() < nev) {
    cudaEvent_t e = nullptr;
    CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->hev.push_back(e);
  }
  cudaEvent_t* in_ev = c->hev.data();  // chunk k copied in, on copy stream 0 and 1
  cudaEvent_t* tau_ev = in_ev + 2 * K; // TAU factors of chunk k's +d faces
  cudaEvent_t* s1 = tau_ev + K;        // stage 1 of launch group q (at most K groups)
  cudaEvent_t* s2 = s1 + K;            // stage 2 (of the last step) of launch group q
  cudaEvent_t* ev = s2 + K;            // start, last stage 1, joins of the six streams
  cudaStream_t cs[2] = {c->hs[0], c->hs[1]};
  cudaStream_t* ks = c->hs + 2;        // compute stream q: launch group q
  const int prec = c->p.precision;
  const bool tau = c->p.hll_mode == RHD_HLL_TAU;
  auto cyc = [K](int k) { return (k % K + K) % K; };

  CUDA_TRY(c, cudaEventRecord(ev[0], c->stream));
  for (int k = 0; k < 8; ++k) CUDA_TRY(c, cudaStreamWaitEvent(c->hs[k], ev[0], 0));
  CUDA_TRY(c, launch_status_reset(c->d_status, cs[0]));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), cs[0]));
  c->launches += 1;
  if (tau) {
    c->eps_dirty = false;
    c->slab_mat_above = c->slab_eps_below = false;
  }

  // copies in, in the order 0, K-1, 1, ..., K-2 (chunk 0 needs K-1 and 1),
  // even fields on copy stream 0 and odd ones on copy stream 1 (two copy
  // engines; a field's copies in and out share a stream, so dst may be src).
  // Only copies go on the copy streams: a kernel there would wait for SMs the
  // stage kernels hold, and every later copy behind it.
  std::vector<int> order(1, 0);
  if (K > 1) order.push_back(K - 1);
  for (int k = 1; k < K - 1; ++k) order.push_back(k);
  for (int x : order) {
    const size_t n = i0[x + 1] - i0[x];
    for (int f = 0; f < RHD_NFIELDS; ++f)
      CUDA_TRY(c, cudaMemcpyAsync(field_ptr(c, f) + i0[x], src + f * N + i0[x],
                                  sizeof(double) * n, cudaMemcpyHostToDevice, cs[f & 1]));
    for (int h = 0; h < 2; ++h) CUDA_TRY(c, cudaEventRecord(in_ev[2 * x + h], cs[h]));
  }

  // Stage launches over groups of chunks [a, b): few launches, small ones
  // where they start or end the pipeline.  Group q runs on compute stream q,
  // whose priority falls with q: launched together, the groups' blocks are
  // dispatched in group order, each group's last wave shared with the next
  // group's first blocks.  Stage 1: chunk 0 as soon as chunks K-1, 0, 1 are in, chunks
  // 1 .. K/4 - 1 (enough work to cover the remaining copies in), then the
  // rest.  The last stage 2: groups each copied out as it finishes while the
  // next ones compute, none larger than a quarter of the grid (so that a slow
  // copy out keeps pace): chunks 1 .. K-4 in up to three groups, then
  // K-3 .. K-2, K-1, and 0 last.  A stage-1 group reads the inputs of chunks a-1 .. b and the
  // TAU factors of chunks a-1 .. b-1 (launched on the stream of the first
  // group that needs them); a stage-2 group the stage-1 outputs of a-1 .. b.
  const StageArgs A1 = host_stage_args(c, dt, 0, 1);
  std::vector<int> grp1(K, -1);          // the stage-1 group of each chunk
  std::vector<int> tau_on(K, -1);        // the stream index that made chunk k's TAU factors
  for (int q = 0; q < (int)g1.size(); ++q) {
    const int a = g1[q].first, b = g1[q].second;
    const int si = q;
    cudaStream_t st = ks[si];
    std::vector<char> waited(K, 0);
    for (int k = a - 1; k <= b; ++k) {
      if (waited[cyc(k)]) continue;
      for (int h = 0; h < 2; ++h)
        CUDA_TRY(c, cudaStreamWaitEvent(st, in_ev[2 * cyc(k) + h], 0));
      waited[cyc(k)] = 1;
    }
    if (tau) {
      for (int k = a - 1; k < b; ++k) {
        const int j = cyc(k);
        if (tau_on[j] < 0) {
          CUDA_TRY(c, launch_tau_eps(g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps, st,
                                     nullptr, nullptr, (long long)i0[j], (long long)i0[j + 1]));
          CUDA_TRY(c, cudaEventRecord(tau_ev[j], st));
          tau_on[j] = si;
          c->launches += 1;
        } else if (tau_on[j] != si) {
          CUDA_TRY(c, cudaStreamWaitEvent(st, tau_ev[j], 0));
        }
      }
    }
    CUDA_TRY(c, launch_stage(1, prec, A1, st, r0[a], r0[b]));
    CUDA_TRY(c, cudaEventRecord(s1[q], st));
    for (int k = a; k < b; ++k) grp1[k] = q;
    c->launches += 1;
  }
  // the input check (as rhd_state_set_all), read after the step: whole
  // fields on the stream of the last stage-1 group, whose wait covers every
  // chunk's copy
  const int nq1 = (int)g1.size();
  for (int f = 0; f < RHD_NFIELDS; ++f)
    CUDA_TRY(c, launch_check_field(f, field_ptr(c, f), c->ncell, c->d_flag, ks[nq1 - 1]));
  c->launches += RHD_NFIELDS;

  // the steps between: whole-grid launches on the first compute stream
  const StageArgs A2 = host_stage_args(c, dt, nsteps - 1, 2);
  if (nsteps > 1) {
    for (int q = 0; q < (int)g1.size(); ++q) CUDA_TRY(c, cudaStreamWaitEvent(ks[0], s1[q], 0));
    CUDA_TRY(c, launch_stage(2, prec, host_stage_args(c, dt, 0, 2), ks[0]));
    for (int s = 1; s < nsteps; ++s) {
      CUDA_TRY(c, launch_stage(1, prec, host_stage_args(c, dt, s, 1), ks[0]));
      if (s < nsteps - 1) CUDA_TRY(c, launch_stage(2, prec, host_stage_args(c, dt, s, 2), ks[0]));
    }
    c->launches += 2 * (nsteps - 1);
    CUDA_TRY(c, cudaEventRecord(ev[1], ks[0]));
    for (int q = 1; q < 6; ++q) CUDA_TRY(c, cudaStreamWaitEvent(ks[q], ev[1], 0));
  }
  for (int q = 0; q < (int)g2.size(); ++q) {
    const int a = g2[q].first, b = g2[q].second;
    cudaStream_t st = ks[q];
    if (nsteps == 1) {
      std::vector<char> seen(g1.size(), 0);
      for (int k = a - 1; k <= b; ++k) {
        const int gq = grp1[(k + K) % K];
        if (!seen[gq]) CUDA_TRY(c, cudaStreamWaitEvent(st, s1[gq], 0));
        seen[gq] = 1;
      }
    }
    CUDA_TRY(c, launch_stage(2, prec, A2, st, r0[a], r0[b]));
    CUDA_TRY(c, cudaEventRecord(s2[q], st));
    c->launches += 1;
  }
  // copies out: rho and kappa (unchanged; not copied back in place) first,
  // then each group's evolved fields after its stage 2, on the stream that
  // copied the field in
  if (dst != src)
    for (int f : {RHD_F_RHO, RHD_F_KAPPA})
      CUDA_TRY(c, cudaMemcpyAsync(dst + f * N, field_ptr(c, f), sizeof(double) * N,
                                  cudaMemcpyDeviceToHost, cs[f & 1]));
  const double* out = c->ybuf[c->cur ^ (nsteps & 1)];
  for (int q = 0; q < (int)g2.size(); ++q) {
    for (int h = 0; h < 2; ++h) CUDA_TRY(c, cudaStreamWaitEvent(cs[h], s2[q], 0));
    const size_t lo = i0[g2[q].first], n = i0[g2[q].second] - lo;
    for (int f = 0; f < RHD_NFIELDS; ++f) {
      const int slot = slot_of(f);
      if (slot < 0) continue;
      CUDA_TRY(c, cudaMemcpyAsync(dst + f * N + lo, out + (size_t)slot * N + lo,
                                  sizeof(double) * n, cudaMemcpyDeviceToHost, cs[f & 1]));
    }
  }
  for (int k = 0; k < 8; ++k) {
    CUDA_TRY(c, cudaEventRecord(ev[2 + k], c->hs[k]));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, ev[2 + k], 0));
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
  return RHD_OK;
}

rhd_status rhd_host_step_plan(const rhd_params* p, int* nchunks, int64_t* cells, int* rows,
                              int* groups, int ngroups[2], int cap) {
  char msg[256];
  if (!p || !nchunks || !cells || !rows || !groups || !ngroups)
    return fail(nullptr, RHD_ERR_ARG, "a pointer argument is NULL");
  if (rhd_params_validate(p, msg, sizeof(msg)) != RHD_OK)
    return fail(nullptr, RHD_ERR_ARG, "invalid params: %s", msg);
  Geometry g;
  Physics ph;
  fill_geometry(p, g, ph);
  const HostPlan P = host_step_plan(g);
  const int ng = (int)(P.g1.size() + P.g2.size());
  if (cap < P.K + 1 || cap < ng)
    return fail(nullptr, RHD_ERR_ARG, "cap %d < %d", cap, std::max(P.K + 1, ng));
  *nchunks = P.K;
  for (int k = 0; k <= P.K; ++k) {
    cells[k] = (int64_t)P.i0[k];
    rows[k] = P.r0[k];
  }
  int j = 0;
  for (const auto& q : P.g1) { groups[2 * j] = q.first; groups[2 * j + 1] = q.second; ++j; }
  for (const auto& q : P.g2) { groups[2 * j] = q.first; groups[2 * j + 1] = q.second; ++j; }
  ngroups[0] = (int)P.g1.size();
  ngroups[1] = (int)P.g2.size();
  return RHD_OK;
}

rhd_status rhd_step_host(rhd_ctx* c, const double* src, double* dst, int64_t count,
                         int nsteps, double dt, rhd_step_info* info) {
  if (!c) return host_step_fail_info(c, fail(nullptr, RHD_ERR_ARG, "ctx is NULL"), info);
  rhd_status s = RHD_OK;
  if (c->pending)
    s = fail(c, RHD_ERR_STATE, "a step batch is pending");
  else if (c->slab_phase != 0)
    s = fail(c, RHD_ERR_STATE, "a slab step is in progress");
  else if (has_halo(c))
    s = fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  else if (!src || !dst)
    s = fail(c, RHD_ERR_ARG, "buffer is NULL");
  else if (count != (int64_t)RHD_NFIELDS * c->ncell)
    s = fail(c, RHD_ERR_ARG, "count must be RHD_NFIELDS * ncell");
  else if (nsteps < 1)
    s = fail(c, RHD_ERR_ARG, "nsteps < 1");
  else if (dst != src && dst < src + count && src < dst + count)
    s = fail(c, RHD_ERR_ARG, "dst overlaps src without being src");
  if (s == RHD_OK) {
    if (!(dt > 0.0)) dt = rhd_default_dt(&c->p);
    if (!std::isfinite(dt)) s = fail(c, RHD_ERR_ARG, "dt is not finite");
  }
  if (s != RHD_OK) return host_step_fail_info(c, s, info);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess)
    return host_step_fail_info(
        c, fail(c, RHD_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e)), info);
  const int cur0 = c->cur;
  const double t0 = c->t;
  *c->h_flag = 0;
  s = host_step_enqueue(c, src, dst, nsteps, dt);
  if (s != RHD_OK) {
    cudaStreamSynchronize(c->stream);
    for (auto h : c->hs)
      if (h) cudaStreamSynchronize(h);
    c->fields_set = 0;  // the copies in may have stopped part way
    return host_step_fail_info(c, s, info);
  }
  c->pending = true;
  c->pending_n = nsteps;
  c->pending_dt = dt;
  c->pending_cur0 = cur0;
  s = rhd_sync(c, info);  // waits for the copies out too
  if (*c->h_flag) {
    c->fields_set = 0;
    c->cur = cur0;
    c->t = t0;
    return host_step_fail_info(
        c, fail(c, RHD_ERR_ARG, "state holds a non-finite or out-of-range value"), info);
  }
  c->fields_set = kAllFields;
  return s;
}

rhd_status rhd_transport(rhd_ctx* c, double* rates, int64_t count, int dst_on_device) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (has_halo(c)) return fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  if (!rates) return fail(c, RHD_ERR_ARG, "rates is NULL");
  if (count != 4 * (int64_t)c->ncell) return fail(c, RHD_ERR_ARG, "count must be 4 * ncell");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const size_t N = (size_t)c->ncell;
  double* out = rates;
  if (!dst_on_device) out = c->ybuf[c->cur ^ 1];  // the idle ping-pong buffer as staging
  CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
  if (c->p.hll_mode == RHD_HLL_TAU && c->eps_dirty) {
    CUDA_TRY(c, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps, c->stream));
    c->launches += 1;
    c->eps_dirty = false;
  }
  StageArgs A;
  A.cell_base = 0;
  A.g = c->g;
  A.ph = c->ph;
  A.dt = 0.0;
  A.step = 0;
  A.rho = c->rho;
  A.kappa = c->kappa;
  A.st = c->d_status;
  for (int d = 0; d < 3; ++d) A.eps[d] = c->eps[d];
  slots_of<const double*>(A.yt, c->ybuf[c->cur], c->ncell);
  slots_of<const double*>(A.yn, c->ybuf[c->cur], c->ncell);
  slots_of<double*>(A.yo, c->yhalf, c->ncell);
  for (int q = 0; q < 4; ++q) A.rate[q] = out + q * N;
  CUDA_TRY(c, launch_stage(0, c->p.precision, A, c->stream));
  c->launches += 2;
  if (!dst_on_device)
    CUDA_TRY(c, cudaMemcpyAsync(rates, out, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost,
                                c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->h_status->fail_key != ~0ull)
    return fail(c, RHD_ERR_NONPHYSICAL, "a face state has E <= 0 near cell %lld",
                (long long)(c->h_status->fail_key >> 8));
  return RHD_OK;
}

rhd_status rhd_totals(rhd_ctx* c, double out[4]) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!out) return fail(c, RHD_ERR_ARG, "out is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (c->prof) {
    Rec r;
    r.a = take_event(c);
    r.b = take_event(c);
    r.kind = 2;
    cudaEventRecord(r.a, c->stream);
    CUDA_TRY(c, launch_totals(c->g, c->ph, c->ybuf[c->cur], c->d_partials,
                              totals_partials_needed(), c->d_tot, c->stream));
    cudaEventRecord(r.b, c->stream);
    c->recs.push_back(r);
  } else {
    CUDA_TRY(c, launch_totals(c->g, c->ph, c->ybuf[c->cur], c->d_partials,
                              totals_partials_needed(), c->d_tot, c->stream));
  }
  c->launches += 2;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_tot, c->d_tot, sizeof(double) * 4,
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int q = 0; q < 4; ++q) out[q] = c->h_tot[q];
  return RHD_OK;
}

rhd_status rhd_profile(rhd_ctx* c, int enable) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (enable) recycle_records(c);
  c->prof = enable != 0;
  return RHD_OK;
}

rhd_status rhd_profile_read(rhd_ctx* c, int64_t launches[3], double ms[3]) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!launches || !ms) return fail(c, RHD_ERR_ARG, "output is NULL");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 3; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  for (auto& r : c->recs) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, r.a, r.b));
    launches[r.kind] += 1;
    ms[r.kind] += (double)t;
  }
  return RHD_OK;
}

// ------------------------------------------------------------ differentiation

static void fill_info_status(rhd_ctx* c, const DevStatus& st, int n, double dt,
                             rhd_step_info* info, rhd_status code, int done, int64_t cell) {
  if (!info) return;
  info->status = code;
  info->steps_done = done;
  info->fail_cell = cell;
  info->fail_step = code == RHD_OK ? -1 : st.fail_step;
  info->fail_stage = code == RHD_OK ? 0 : st.fail_stage;
  info->max_newton = st.max_newton;
  info->max_outer = st.max_outer;
  info->sum_newton = (int64_t)st.sum_newton;
  info->n_solves = (int64_t)st.n_solves;
  info->sum_outer = (int64_t)st.sum_outer;
  info->t = c->t;
  info->dt = dt;
  (void)n;
}

rhd_status rhd_step_record(rhd_ctx* c, int nsteps, double dt, double* tape, int64_t count,
                           rhd_step_info* info) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->fail_cell = -1;
    info->fail_step = -1;
  }
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (has_halo(c)) return fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  if (nsteps < 0) return fail(c, RHD_ERR_ARG, "nsteps < 0");
  if (!tape) return fail(c, RHD_ERR_ARG, "tape is NULL");
  const size_t N = (size_t)c->ncell;
  const size_t S = NY * N;  // doubles per recorded state
  if (count != (int64_t)((2 * (size_t)nsteps + 1) * S))
    return fail(c, RHD_ERR_ARG, "tape count must be (2*nsteps+1)*8*ncell");
  if (!(dt > 0.0)) dt = rhd_default_dt(&c->p);
  if (!std::isfinite(dt)) return fail(c, RHD_ERR_ARG, "dt is not finite");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
  c->launches += 1;
  if (c->p.hll_mode == RHD_HLL_TAU && c->eps_dirty) {
    CUDA_TRY(c, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps, c->stream));
    c->launches += 1;
    c->eps_dirty = false;
  }
  CUDA_TRY(c, cudaMemcpyAsync(tape, c->ybuf[c->cur], sizeof(double) * S,
                              cudaMemcpyDeviceToDevice, c->stream));
  StageArgs A;
  A.cell_base = 0;
  for (int d = 0; d < 3; ++d) A.eps[d] = c->eps[d];
  A.g = c->g;
  A.ph = c->ph;
  A.dt = dt;
  A.rho = c->rho;
  A.kappa = c->kappa;
  A.st = c->d_status;
  const int n = c->ncell;
  for (int s = 0; s < nsteps; ++s) {
    double* yn = tape + (size_t)(2 * s) * S;
    double* yh = yn + S;
    double* y1 = yh + S;
    A.step = s;
    slots_of<const double*>(A.yt, yn, n);
    slots_of<const double*>(A.yn, yn, n);
    slots_of<double*>(A.yo, yh, n);
    CUDA_TRY(c, launch_recorded(c, 0, 1, A));
    slots_of<const double*>(A.yt, yh, n);
    slots_of<double*>(A.yo, y1, n);
    CUDA_TRY(c, launch_recorded(c, 1, 2, A));
    c->launches += 2;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const DevStatus& st = *c->h_status;
  if (st.fail_key != ~0ull) {
    rhd_status code = (rhd_status)(st.fail_key & 0xffull);
    int64_t cell = (int64_t)(st.fail_key >> 8);
    fill_info_status(c, st, nsteps, dt, info, code, st.fail_step, cell);
    return fail(c, code, "recorded step %d stage %d failed at cell %lld (status %d)",
                st.fail_step, st.fail_stage, (long long)cell, (int)code);
  }
  // the context continues from y(nsteps)
  CUDA_TRY(c, cudaMemcpyAsync(c->ybuf[c->cur], tape + (size_t)(2 * nsteps) * S,
                              sizeof(double) * S, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->t += nsteps * dt;
  fill_info_status(c, st, nsteps, dt, info, RHD_OK, nsteps, -1);
  return RHD_OK;
}

rhd_status rhd_adjoint(rhd_ctx* c, const double* tape, int64_t count, int nsteps, double dt,
                       double* ybar, double* kappa_bar) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if ((c->fields_set & ((1u << RHD_F_RHO) | (1u << RHD_F_KAPPA))) !=
      ((1u << RHD_F_RHO) | (1u << RHD_F_KAPPA)))
    return fail(c, RHD_ERR_STATE, "rho and kappa must be set");
  if (has_halo(c)) return fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  if (nsteps < 0) return fail(c, RHD_ERR_ARG, "nsteps < 0");
  if (!tape || !ybar || !kappa_bar) return fail(c, RHD_ERR_ARG, "a buffer is NULL");
  if (c->p.scheme != RHD_SCHEME_IMEX_PDARS || c->p.kappa_T_exp != 0.0 ||
      c->p.kappa_P_ratio != 1.0 || c->p.kappa_F_ratio != 1.0)
    return fail(c, RHD_ERR_ARG,
                "the adjoint covers the IMEX scheme with a grey, temperature-independent "
                "opacity");
  for (int d = 0; d < c->p.ndim; ++d)
    if (c->p.bc[d][0] == RHD_BC_INFLOW || c->p.bc[d][1] == RHD_BC_INFLOW)
      return fail(c, RHD_ERR_ARG, "the adjoint covers periodic and reflecting boundaries");
  if (c->p.reconstruction != RHD_RECON_PLM)
    return fail(c, RHD_ERR_ARG, "the adjoint covers PLM faces");
  const size_t N = (size_t)c->ncell;
  const size_t S = NY * N;
  if (count != (int64_t)((2 * (size_t)nsteps + 1) * S))
    return fail(c, RHD_ERR_ARG, "tape count must be (2*nsteps+1)*8*ncell");
  if (!(dt > 0.0)) dt = rhd_default_dt(&c->p);
  if (!std::isfinite(dt)) return fail(c, RHD_ERR_ARG, "dt is not finite");
  if (nsteps == 0) return RHD_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (!c->adj_q || !c->adj_fp) {
    // both or neither: a failed second allocation releases the first
    cudaFree(c->adj_q);
    c->adj_q = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->adj_q, sizeof(double) * S));
    cudaError_t e = cudaMalloc(&c->adj_fp, sizeof(double) * adjoint_scratch_doubles(c->g));
    if (e != cudaSuccess) {
      cudaGetLastError();  // clear the allocation error for later launch checks
      c->adj_fp = nullptr;
      cudaFree(c->adj_q);
      c->adj_q = nullptr;
      return fail(c, RHD_ERR_CUDA, "adjoint scratch: %s", cudaGetErrorString(e));
    }
  }
  CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
  AdjointStep A;
  A.g = c->g;
  A.ph = c->ph;
  A.dt = dt;
  A.rho = c->rho;
  A.kappa = c->kappa;
  A.ybar = ybar;
  A.q = c->adj_q;
  A.fp = c->adj_fp;
  A.kbar = kappa_bar;
  A.st = c->d_status;
  for (int k = nsteps - 1; k >= 0; --k) {
    A.step = k;
    A.yn = tape + (size_t)(2 * k) * S;
    A.yh = A.yn + S;
    A.y1 = A.yh + S;
    A.pending_fp = k < nsteps - 1;
    CUDA_TRY(c, launch_adjoint_step(A, c->stream));
  }
  CUDA_TRY(c, launch_adjoint_finish(A, c->stream));
  c->launches += 1 + 4 * (int64_t)nsteps + 1;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->h_status->fail_key != ~0ull)
    return fail(c, RHD_ERR_NEWTON,
                "adjoint step %d: singular local-solve Jacobian at cell %lld",
                c->h_status->fail_step, (long long)(c->h_status->fail_key >> 8));
  return RHD_OK;
}

// ------------------------------------------------ hydrodynamics (Sec. 3.1)

static rhd_status hydro_alloc(rhd_ctx* c);

static rhd_status hydro_ready(rhd_ctx* c) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (has_halo(c)) return fail(c, RHD_ERR_STATE, "%s", kHaloOnly);
  for (int d = 0; d < c->p.ndim; ++d)
    if (c->p.bc[d][0] == RHD_BC_INFLOW || c->p.bc[d][1] == RHD_BC_INFLOW)
      return fail(c, RHD_ERR_ARG, "the hydrodynamic step takes periodic and reflecting axes");
  return hydro_alloc(c);
}

// the hydrodynamic scratch of a context, allocated once
static rhd_status hydro_alloc(rhd_ctx* c) {
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (c->hyd_bits) return RHD_OK;  // allocated last: every buffer is there
  const size_t N = (size_t)c->ncell;
  double** bufs[5] = {&c->hyd_w, &c->hyd_u1, &c->hyd_f[0], &c->hyd_f[1], &c->hyd_f[2]};
  size_t bytes[5] = {sizeof(double) * 5 * N, sizeof(double) * 5 * N, 0, 0, 0};
  for (int d = 0; d < c->p.ndim; ++d) bytes[2 + d] = sizeof(double) * 5 * hydro_faces(c->g, d);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 5 && e == cudaSuccess; ++i)
    if (bytes[i] && !*bufs[i]) e = cudaMalloc(bufs[i], bytes[i]);
  if (e == cudaSuccess) e = cudaMalloc(&c->hyd_bits, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the allocation error for later launch checks
    // none or all: release what this call could not complete
    for (int i = 0; i < 5; ++i) {
      cudaFree(*bufs[i]);
      *bufs[i] = nullptr;
    }
    c->hyd_bits = nullptr;
    return fail(c, RHD_ERR_CUDA, "hydrodynamic scratch: %s", cudaGetErrorString(e));
  }
  return RHD_OK;
}

static HydroBufs hydro_bufs(rhd_ctx* c) {
  HydroBufs b;
  b.rho = c->rho;
  b.y = c->ybuf[c->cur];
  b.w = c->hyd_w;
  b.u1 = c->hyd_u1;
  for (int d = 0; d < 3; ++d) b.f[d] = c->hyd_f[d];
  b.dt_bits = c->hyd_bits;
  return b;
}

static rhd_status hydro_dt_of(rhd_ctx* c, double* dt) {
  HydroBufs b = hydro_bufs(c);
  CUDA_TRY(c, launch_hydro_speed(c->g, c->p.gamma, b, c->stream));
  c->launches += 1;
  unsigned long long bits = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bits, c->hyd_bits, sizeof(bits), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double smax;
  memcpy(&smax, &bits, sizeof(smax));
  if (!(smax > 0.0) || !std::isfinite(smax))
    return fail(c, RHD_ERR_NONPHYSICAL, "a cell has rho <= 0 or p <= 0: no hydrodynamic step");
  *dt = c->p.cfl_hydro / smax;
  return RHD_OK;
}

// nsteps hydrodynamic steps of dt (dt <= 0: the CFL step of each state);
// steps_done and the failure go to info; time advances by each step when
// advance_time.
static rhd_status hydro_run(rhd_ctx* c, int nsteps, double dt, rhd_step_info* info,
                            bool advance_time) {
  if (info) {
    memset(info, 0, sizeof(*info));
    info->fail_cell = -1;
    info->fail_step = -1;
  }
  const int launches_per_step = 5 + 2 * c->p.ndim;
  int done = 0;
  double last = dt;
  rhd_status code = RHD_OK;
  while (done < nsteps && code == RHD_OK) {
    // fixed dt: every remaining step in one batch; else one step per CFL bound
    int batch = dt > 0.0 ? nsteps - done : 1;
    double h = dt;
    if (!(h > 0.0)) {
      rhd_status s = hydro_dt_of(c, &h);
      if (s != RHD_OK) {
        code = s;
        break;
      }
    }
    last = h;
    CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
    c->launches += 1;
    HydroBufs b = hydro_bufs(c);
    for (int k = 0; k < batch; ++k) {
      CUDA_TRY(c, launch_hydro_step(c->g, c->p.gamma, c->p.reconstruction, h, b, c->d_status,
                                    k, c->stream));
      c->launches += launches_per_step;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const DevStatus& st = *c->h_status;
    int ok = batch;
    c->eps_dirty = true;  // rho has changed
    c->slab_mat_above = c->slab_eps_below = false;
    if (st.fail_key != ~0ull) {
      code = (rhd_status)(st.fail_key & 0xffull);
      ok = st.fail_step;
      if (info) {
        info->fail_cell = (int64_t)(st.fail_key >> 8);
        info->fail_step = done + st.fail_step;
        info->fail_stage = st.fail_stage;
      }
    }
    done += ok;
    if (advance_time) c->t += ok * h;
  }
  if (info) {
    info->status = code;
    info->steps_done = done;
    info->t = c->t;
    info->dt = last;
  }
  if (code != RHD_OK)
    return fail(c, code, "hydrodynamic step %d failed (status %d)", done, (int)code);
  return RHD_OK;
}

rhd_status rhd_hydro_dt(rhd_ctx* c, double* dt) {
  rhd_status s = hydro_ready(c);
  if (s != RHD_OK) return s;
  if (!dt) return fail(c, RHD_ERR_ARG, "dt is NULL");
  return hydro_dt_of(c, dt);
}

rhd_status rhd_hydro_step(rhd_ctx* c, int nsteps, double dt, rhd_step_info* info) {
  rhd_status s = hydro_ready(c);
  if (s == RHD_OK && nsteps < 0) s = fail(c, RHD_ERR_ARG, "nsteps < 0");
  if (s == RHD_OK && !std::isfinite(dt)) s = fail(c, RHD_ERR_ARG, "dt is not finite");
  if (s != RHD_OK) {
    if (info) {
      memset(info, 0, sizeof(*info));
      info->status = s;
      info->fail_cell = -1;
      info->fail_step = -1;
    }
    return s;
  }
  return hydro_run(c, nsteps, dt, info, true);
}

rhd_status rhd_step_split(rhd_ctx* c, int nsteps, double dt_h, rhd_step_info* info) {
  rhd_status s = hydro_ready(c);
  if (s == RHD_OK && nsteps < 0) s = fail(c, RHD_ERR_ARG, "nsteps < 0");
  if (s == RHD_OK && !std::isfinite(dt_h)) s = fail(c, RHD_ERR_ARG, "dt_h is not finite");
  rhd_step_info total;
  memset(&total, 0, sizeof(total));
  total.fail_cell = -1;
  total.fail_step = -1;
  total.t = c ? c->t : 0.0;
  const double dt_rad = c ? rhd_default_dt(&c->p) : 0.0;
  for (int k = 0; s == RHD_OK && k < nsteps; ++k) {
    rhd_step_info one;
    s = hydro_run(c, 1, dt_h, &one, false);
    const double h = one.dt;
    if (s == RHD_OK) {
      int nsub = (int)std::ceil(h / dt_rad - 1e-12);
      if (nsub < 1) nsub = 1;
      s = rhd_step(c, nsub, h / nsub, &one);
      total.max_newton = std::max(total.max_newton, one.max_newton);
      total.max_outer = std::max(total.max_outer, one.max_outer);
      total.sum_newton += one.sum_newton;
      total.sum_outer += one.sum_outer;
      total.n_solves += one.n_solves;
    }
    total.dt = h;
    if (s != RHD_OK) {
      total.fail_cell = one.fail_cell;
      total.fail_step = k;
      total.fail_stage = one.fail_stage;
    } else {
      total.steps_done = k + 1;
    }
  }
  total.status = s;
  if (c) total.t = c->t;
  if (info) *info = total;
  return s;
}

// ---- z-slabs of one grid on one device

}  // extern "C"

// params of two slabs of one grid: equal but for n[2] and the z faces
static bool same_grid_but_z(const rhd_params& a, const rhd_params& b) {
  if (a.ndim != b.ndim || a.n[0] != b.n[0] || a.n[1] != b.n[1]) return false;
  for (int d = 0; d < 3; ++d) {
    if (a.dx[d] != b.dx[d]) return false;
    for (int s = 0; s < 2; ++s) {
      if (d < 2 && a.bc[d][s] != b.bc[d][s]) return false;
      for (int q = 0; q < 4; ++q)
        if (a.bc_state[d][s][q] != b.bc_state[d][s][q]) return false;
    }
  }
  return a.gamma == b.gamma && a.c == b.c && a.chat == b.chat && a.a_rad == b.a_rad &&
         a.kB_over_mu == b.kB_over_mu && a.cfl == b.cfl && a.closure == b.closure &&
         a.vc_order == b.vc_order && a.hll_mode == b.hll_mode && a.precision == b.precision &&
         a.newton_rtol == b.newton_rtol && a.outer_rtol == b.outer_rtol &&
         a.newton_max_iter == b.newton_max_iter && a.outer_max_iter == b.outer_max_iter &&
         a.scheme == b.scheme && a.kappa_T_exp == b.kappa_T_exp &&
         a.kappa_T_ref == b.kappa_T_ref && a.kappa_P_ratio == b.kappa_P_ratio &&
         a.kappa_F_ratio == b.kappa_F_ratio && a.reconstruction == b.reconstruction &&
         a.cfl_hydro == b.cfl_hydro;
}

// Copy the ghost planes of slab s from its neighbours: depth planes of the
// nfield fields slot[] of the buffers src[] (field f of slab u at
// src[u] + f * ncell(u)) per HALO face into the slab's halo buffer
// [side][field][HALO_PLANES planes][n0 n1], one device-to-device copy per
// field and face.
static cudaError_t exchange(rhd_ctx* const* slabs, int nslab, int s, double* const* src,
                            const int* slot, int nfield, double* halo, int depth,
                            cudaStream_t st) {
  rhd_ctx* c = slabs[s];
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  for (int side = 0; side < 2; ++side) {
    if (c->p.bc[2][side] != RHD_BC_HALO) continue;
    const int nb = side == 0 ? (s + nslab - 1) % nslab : (s + 1) % nslab;
    const rhd_ctx* u = slabs[nb];
    // the low face takes the top depth planes of the slab below (ghost
    // planes -depth..-1), the high face the bottom ones of the slab above
    const size_t z0 = side == 0 ? (size_t)u->g.n[2] - depth : 0;
    const size_t i0 = side == 0 ? HALO_PLANES - depth : 0;
    double* h = halo + (size_t)side * nfield * HALO_PLANES * P;
    for (int q = 0; q < nfield; ++q) {
      cudaError_t e = cudaMemcpyAsync(
          h + ((size_t)q * HALO_PLANES + i0) * P,
          src[nb] + (size_t)slot[q] * u->ncell + z0 * P, sizeof(double) * depth * P,
          cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

static void clear_info(rhd_step_info* info, double t) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  info->fail_cell = -1;
  info->fail_step = -1;
  info->t = t;
}

// The checks every slab call makes: distinct contexts of one grid's z-slabs,
// one device and stream, every field set, HALO faces between neighbours and
// at both ends or at neither.
static rhd_status check_slabs(rhd_ctx* const* slabs, int nslab) {
  if (!slabs || nslab < 1) return fail(nullptr, RHD_ERR_ARG, "slabs is NULL or nslab < 1");
  for (int s = 0; s < nslab; ++s) {
    if (!slabs[s]) return fail(nullptr, RHD_ERR_ARG, "slabs[%d] is NULL", s);
    for (int r = 0; r < s; ++r)
      if (slabs[r] == slabs[s])
        return fail(slabs[s], RHD_ERR_ARG, "slabs[%d] and slabs[%d] are one context", r, s);
  }
  rhd_ctx* c0 = slabs[0];
  const int last = nslab - 1;
  for (int s = 0; s < nslab; ++s) {
    rhd_ctx* c = slabs[s];
    if (c->p.ndim != 3) return fail(c0, RHD_ERR_ARG, "slab %d: slabs are 3-D grids", s);
    if (!same_grid_but_z(c->p, c0->p))
      return fail(c0, RHD_ERR_ARG, "slab %d: params differ from slab 0 beyond n[2] and "
                  "the z faces", s);
    if (c->device != c0->device || c->stream != c0->stream)
      return fail(c0, RHD_ERR_ARG, "slab %d: slabs share one device and one stream", s);
    if (c->pending) return fail(c0, RHD_ERR_STATE, "slab %d: a step batch is pending", s);
    if (c->slab_phase != 0)
      return fail(c0, RHD_ERR_STATE, "slab %d: a stage-by-stage step is in progress", s);
    if (c->fields_set != kAllFields)
      return fail(c0, RHD_ERR_STATE, "slab %d: not every field has been set", s);
    if (s < last && (c->p.bc[2][1] != RHD_BC_HALO || slabs[s + 1]->p.bc[2][0] != RHD_BC_HALO))
      return fail(c0, RHD_ERR_ARG, "the face between slabs %d and %d must be HALO on both "
                  "sides", s, s + 1);
  }
  const bool wrap = c0->p.bc[2][0] == RHD_BC_HALO;
  if (wrap != (slabs[last]->p.bc[2][1] == RHD_BC_HALO))
    return fail(c0, RHD_ERR_ARG, "the bottom face of slab 0 and the top face of slab %d "
                "are both HALO (a periodic grid) or neither", last);
  if (!wrap && c0->p.bc[2][0] == RHD_BC_PERIODIC && nslab > 1)
    return fail(c0, RHD_ERR_ARG, "a periodic z axis of several slabs uses HALO end faces");
  CUDA_TRY(c0, cudaSetDevice(c0->device));
  return RHD_OK;
}

// nsteps radiation steps of dt of checked slabs (rhd_step_slabs)
static rhd_status slab_radiation(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                                 rhd_step_info* info) {
  rhd_ctx* c0 = slabs[0];
  clear_info(info, c0->t);
  const cudaStream_t st = c0->stream;
  const size_t P = (size_t)c0->g.n[0] * c0->g.n[1];
  for (int s = 0; s < nslab; ++s)
    if (!slabs[s]->halo) {
      cudaError_t e = cudaMalloc(&slabs[s]->halo, sizeof(double) * kHaloSlots * P);
      if (e != cudaSuccess) {
        cudaGetLastError();
        slabs[s]->halo = nullptr;
        return fail(c0, RHD_ERR_CUDA, "slab %d: halo buffers: %s", s, cudaGetErrorString(e));
      }
    }
  auto hk = [&](rhd_ctx* c) { return c->halo + (size_t)8 * HALO_PLANES * P; };
  auto hr = [&](rhd_ctx* c) { return hk(c) + P; };
  auto ezlo = [&](rhd_ctx* c) { return hk(c) + 2 * P; };

  // TAU factors: a slab's top face needs plane 0 of the slab above, its
  // bottom face is the top face of the slab below (recomputed every call:
  // a neighbour's rho or kappa may have changed)
  if (c0->p.hll_mode == RHD_HLL_TAU) {
    for (int s = 0; s < nslab; ++s) {
      rhd_ctx* c = slabs[s];
      const bool top = c->p.bc[2][1] == RHD_BC_HALO;
      if (top) {
        const rhd_ctx* u = slabs[(s + 1) % nslab];
        CUDA_TRY(c0, cudaMemcpyAsync(hk(c), u->kappa, sizeof(double) * P,
                                     cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(c0, cudaMemcpyAsync(hr(c), u->rho, sizeof(double) * P,
                                     cudaMemcpyDeviceToDevice, st));
      }
      CUDA_TRY(c0, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps, st,
                                  top ? hk(c) : nullptr, top ? hr(c) : nullptr));
      c->launches += 1;
      c->eps_dirty = false;
    }
    for (int s = 0; s < nslab; ++s) {
      rhd_ctx* c = slabs[s];
      if (c->p.bc[2][0] != RHD_BC_HALO) continue;
      const rhd_ctx* l = slabs[(s + nslab - 1) % nslab];
      CUDA_TRY(c0, cudaMemcpyAsync(ezlo(c), l->eps[2] + (size_t)(l->g.n[2] - 1) * P,
                                   sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
    }
  }

  CUDA_TRY(c0, launch_status_reset(c0->d_status, st));
  c0->launches += 1;
  static const int kRadSlots[4] = {Y_ERAD, Y_FX, Y_FY, Y_FZ};
  const int depth = c0->p.reconstruction == RHD_RECON_PLM ? 2 : 3;
  std::vector<StageArgs> A(nslab);
  std::vector<int> cur(nslab), cur0(nslab);
  long long base = 0;
  for (int s = 0; s < nslab; ++s) {
    rhd_ctx* c = slabs[s];
    StageArgs& a = A[s];
    a.cell_base = base;
    base += c->ncell;
    for (int d = 0; d < 3; ++d) a.eps[d] = c->eps[d];
    a.g = c->g;
    a.ph = c->ph;
    a.dt = dt;
    a.rho = c->rho;
    a.kappa = c->kappa;
    a.st = c0->d_status;  // one status block: a failure anywhere stops every slab
    a.halo[0] = c->halo;
    a.halo[1] = c->halo + (size_t)4 * HALO_PLANES * P;
    a.eps_zlo = ezlo(c);
    cur[s] = cur0[s] = c->cur;
  }
  std::vector<double*> src(nslab);
  for (int k = 0; k < nsteps; ++k) {
    for (int s = 0; s < nslab; ++s) src[s] = slabs[s]->ybuf[cur[s]];
    for (int s = 0; s < nslab; ++s)
      CUDA_TRY(c0, exchange(slabs, nslab, s, src.data(), kRadSlots, 4, slabs[s]->halo, depth,
                            st));
    for (int s = 0; s < nslab; ++s) {
      rhd_ctx* c = slabs[s];
      StageArgs& a = A[s];
      a.step = k;
      slots_of<const double*>(a.yt, c->ybuf[cur[s]], c->ncell);
      slots_of<const double*>(a.yn, c->ybuf[cur[s]], c->ncell);
      slots_of<double*>(a.yo, c->yhalf, c->ncell);
      a.cost = c->cost;
      CUDA_TRY(c0, launch_stage(1, c->p.precision, a, st));
    }
    for (int s = 0; s < nslab; ++s) src[s] = slabs[s]->yhalf;
    for (int s = 0; s < nslab; ++s)
      CUDA_TRY(c0, exchange(slabs, nslab, s, src.data(), kRadSlots, 4, slabs[s]->halo, depth,
                            st));
    for (int s = 0; s < nslab; ++s) {
      rhd_ctx* c = slabs[s];
      StageArgs& a = A[s];
      slots_of<const double*>(a.yt, c->yhalf, c->ncell);
      slots_of<double*>(a.yo, c->ybuf[cur[s] ^ 1], c->ncell);
      a.cost = c->cost + c->ncell;
      CUDA_TRY(c0, launch_stage(2, c->p.precision, a, st));
      c->launches += 2;
      cur[s] ^= 1;
    }
  }
  CUDA_TRY(c0, cudaMemcpyAsync(c0->h_status, c0->d_status, sizeof(DevStatus),
                               cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c0, cudaStreamSynchronize(st));
  const DevStatus& ds = *c0->h_status;
  rhd_status code = RHD_OK;
  int done = nsteps;
  int64_t cell = -1;
  if (ds.fail_key != ~0ull) {
    code = (rhd_status)(ds.fail_key & 0xffull);
    cell = (int64_t)(ds.fail_key >> 8);
    done = ds.fail_step;
  }
  for (int s = 0; s < nslab; ++s) {
    slabs[s]->cur = cur0[s] ^ (done & 1);
    slabs[s]->t += done * dt;
  }
  if (info) {
    info->status = code;
    info->steps_done = done;
    info->fail_cell = cell;
    info->fail_step = code == RHD_OK ? -1 : ds.fail_step;
    info->fail_stage = code == RHD_OK ? 0 : ds.fail_stage;
    info->max_newton = ds.max_newton;
    info->max_outer = ds.max_outer;
    info->sum_newton = (int64_t)ds.sum_newton;
    info->n_solves = (int64_t)ds.n_solves;
    info->sum_outer = (int64_t)ds.sum_outer;
    info->t = c0->t;
    info->dt = dt;
  }
  if (code != RHD_OK)
    return fail(c0, code, "step %d stage %d failed at cell %lld of the slabs (status %d)",
                ds.fail_step, ds.fail_stage, (long long)cell, (int)code);
  return RHD_OK;
}

// the hydrodynamic step's conditions on checked slabs: no inflow face
static rhd_status check_slabs_hydro(rhd_ctx* const* slabs, int nslab) {
  rhd_ctx* c0 = slabs[0];
  for (int d = 0; d < 2; ++d)
    if (c0->p.bc[d][0] == RHD_BC_INFLOW || c0->p.bc[d][1] == RHD_BC_INFLOW)
      return fail(c0, RHD_ERR_ARG, "the hydrodynamic step takes periodic and reflecting axes");
  if (c0->p.bc[2][0] == RHD_BC_INFLOW || slabs[nslab - 1]->p.bc[2][1] == RHD_BC_INFLOW)
    return fail(c0, RHD_ERR_ARG, "the hydrodynamic step takes periodic and reflecting axes");
  for (int s = 0; s < nslab; ++s) {
    rhd_status r = hydro_alloc(slabs[s]);
    if (r != RHD_OK) return fail(c0, r, "slab %d: %s", s, slabs[s]->err);
  }
  const size_t P = (size_t)c0->g.n[0] * c0->g.n[1];
  for (int s = 0; s < nslab; ++s)
    if (!slabs[s]->hyd_halo) {
      cudaError_t e =
          cudaMalloc(&slabs[s]->hyd_halo, sizeof(double) * 2 * 5 * HALO_PLANES * P);
      if (e != cudaSuccess) {
        cudaGetLastError();
        slabs[s]->hyd_halo = nullptr;
        return fail(c0, RHD_ERR_CUDA, "slab %d: halo buffers: %s", s, cudaGetErrorString(e));
      }
    }
  return RHD_OK;
}

// nsteps hydrodynamic steps of dt (dt <= 0: the CFL step of the whole grid
// before each step) of checked slabs, like hydro_run on the whole grid
static rhd_status slab_hydro(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                             rhd_step_info* info, bool advance_time) {
  rhd_ctx* c0 = slabs[0];
  clear_info(info, c0->t);
  const cudaStream_t st = c0->stream;
  const size_t P = (size_t)c0->g.n[0] * c0->g.n[1];
  static const int kPrimSlots[5] = {0, 1, 2, 3, 4};
  const int depth = c0->p.reconstruction == RHD_RECON_PLM ? 2 : 3;
  std::vector<unsigned long long> bits(nslab);
  std::vector<double*> src(nslab);
  for (int s = 0; s < nslab; ++s) src[s] = slabs[s]->hyd_w;
  int done = 0;
  double last = dt;
  rhd_status code = RHD_OK;
  while (done < nsteps && code == RHD_OK) {
    int batch = dt > 0.0 ? nsteps - done : 1;
    double h = dt;
    if (!(h > 0.0)) {
      // the largest signal-speed bound of any slab: the whole grid's
      for (int s = 0; s < nslab; ++s) {
        CUDA_TRY(c0, launch_hydro_speed(slabs[s]->g, c0->p.gamma, hydro_bufs(slabs[s]), st));
        slabs[s]->launches += 1;
        CUDA_TRY(c0, cudaMemcpyAsync(&bits[s], slabs[s]->hyd_bits, sizeof(bits[s]),
                                     cudaMemcpyDeviceToHost, st));
      }
      CUDA_TRY(c0, cudaStreamSynchronize(st));
      unsigned long long mx = 0;
      for (int s = 0; s < nslab; ++s) mx = std::max(mx, bits[s]);
      double smax;
      memcpy(&smax, &mx, sizeof(smax));
      if (!(smax > 0.0) || !std::isfinite(smax)) {
        code = fail(c0, RHD_ERR_NONPHYSICAL,
                    "a cell has rho <= 0 or p <= 0: no hydrodynamic step");
        break;
      }
      h = c0->p.cfl_hydro / smax;
    }
    last = h;
    CUDA_TRY(c0, launch_status_reset(c0->d_status, st));
    c0->launches += 1;
    std::vector<HydroBufs> B(nslab);
    long long base = 0;
    for (int s = 0; s < nslab; ++s) {
      B[s] = hydro_bufs(slabs[s]);
      B[s].halo[0] = slabs[s]->hyd_halo;
      B[s].halo[1] = slabs[s]->hyd_halo + (size_t)5 * HALO_PLANES * P;
      B[s].cell_base = base;
      base += slabs[s]->ncell;
    }
    for (int k = 0; k < batch; ++k) {
      for (int phase = 0; phase < 5; ++phase) {
        // the face phases read the neighbours' primitives of this stage
        if (phase == 1 || phase == 3)
          for (int s = 0; s < nslab; ++s)
            CUDA_TRY(c0, exchange(slabs, nslab, s, src.data(), kPrimSlots, 5,
                                  slabs[s]->hyd_halo, depth, st));
        for (int s = 0; s < nslab; ++s) {
          CUDA_TRY(c0, launch_hydro_phase(phase, slabs[s]->g, c0->p.gamma,
                                          c0->p.reconstruction, h, B[s], c0->d_status, k, st));
          slabs[s]->launches += phase == 1 || phase == 3 ? 1 + c0->p.ndim : 1;
        }
      }
    }
    CUDA_TRY(c0, cudaMemcpyAsync(c0->h_status, c0->d_status, sizeof(DevStatus),
                                 cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c0, cudaStreamSynchronize(st));
    const DevStatus& ds = *c0->h_status;
    int ok = batch;
    for (int s = 0; s < nslab; ++s) slabs[s]->eps_dirty = true;  // rho has changed
    if (ds.fail_key != ~0ull) {
      code = (rhd_status)(ds.fail_key & 0xffull);
      ok = ds.fail_step;
      if (info) {
        info->fail_cell = (int64_t)(ds.fail_key >> 8);
        info->fail_step = done + ds.fail_step;
        info->fail_stage = ds.fail_stage;
      }
    }
    done += ok;
    if (advance_time)
      for (int s = 0; s < nslab; ++s) slabs[s]->t += ok * h;
  }
  if (info) {
    info->status = code;
    info->steps_done = done;
    info->t = c0->t;
    info->dt = last;
  }
  if (code != RHD_OK)
    return fail(c0, code, "hydrodynamic step %d of the slabs failed (status %d)", done,
                (int)code);
  return RHD_OK;
}

extern "C" {

rhd_status rhd_step_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                          rhd_step_info* info) {
  clear_info(info, 0.0);
  rhd_status s = check_slabs(slabs, nslab);
  if (s != RHD_OK) return s;
  if (nsteps < 0) return fail(slabs[0], RHD_ERR_ARG, "nsteps < 0");
  if (!(dt > 0.0)) dt = rhd_default_dt(&slabs[0]->p);
  if (!std::isfinite(dt)) return fail(slabs[0], RHD_ERR_ARG, "dt is not finite");
  return slab_radiation(slabs, nslab, nsteps, dt, info);
}

rhd_status rhd_hydro_step_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt,
                                rhd_step_info* info) {
  clear_info(info, 0.0);
  rhd_status s = check_slabs(slabs, nslab);
  if (s == RHD_OK) s = check_slabs_hydro(slabs, nslab);
  if (s != RHD_OK) return s;
  if (nsteps < 0) return fail(slabs[0], RHD_ERR_ARG, "nsteps < 0");
  if (!std::isfinite(dt)) return fail(slabs[0], RHD_ERR_ARG, "dt is not finite");
  return slab_hydro(slabs, nslab, nsteps, dt, info, true);
}

rhd_status rhd_step_split_slabs(rhd_ctx* const* slabs, int nslab, int nsteps, double dt_h,
                                rhd_step_info* info) {
  clear_info(info, 0.0);
  rhd_status s = check_slabs(slabs, nslab);
  if (s == RHD_OK) s = check_slabs_hydro(slabs, nslab);
  if (s != RHD_OK) return s;
  rhd_ctx* c0 = slabs[0];
  if (nsteps < 0) return fail(c0, RHD_ERR_ARG, "nsteps < 0");
  if (!std::isfinite(dt_h)) return fail(c0, RHD_ERR_ARG, "dt_h is not finite");
  rhd_step_info total;
  clear_info(&total, c0->t);
  const double dt_rad = rhd_default_dt(&c0->p);
  for (int k = 0; s == RHD_OK && k < nsteps; ++k) {
    rhd_step_info one;
    s = slab_hydro(slabs, nslab, 1, dt_h, &one, false);
    const double h = one.dt;
    if (s == RHD_OK) {
      int nsub = (int)std::ceil(h / dt_rad - 1e-12);
      if (nsub < 1) nsub = 1;
      s = slab_radiation(slabs, nslab, nsub, h / nsub, &one);
      total.max_newton = std::max(total.max_newton, one.max_newton);
      total.max_outer = std::max(total.max_outer, one.max_outer);
      total.sum_newton += one.sum_newton;
      total.sum_outer += one.sum_outer;
      total.n_solves += one.n_solves;
    }
    total.dt = h;
    if (s != RHD_OK) {
      total.fail_cell = one.fail_cell;
      total.fail_step = k;
      total.fail_stage = one.fail_stage;
    } else {
      total.steps_done = k + 1;
    }
  }
  total.status = s;
  total.t = c0->t;
  if (info) *info = total;
  return s;
}

int64_t rhd_launch_count(const rhd_ctx* c) { return c ? c->launches : 0; }

double rhd_time(const rhd_ctx* c) { return c ? c->t : 0.0; }

const char* rhd_last_error(const rhd_ctx* c) { return c ? c->err : g_err; }

void rhd_destroy(rhd_ctx* c) { release(c); }

}  // extern "C"

// ------------------------------------------------------------------------
// A z-slab stepped by its own process (the decomposition across processes or
// GPUs, Sec. 3.2: a stage needs the neighbours' ghost planes only).  The
// caller moves the planes between slabs (NCCL, MPI, a file ...); the library
// packs the planes a neighbour needs, stores the planes it receives and runs
// each stage on them, with the same kernels and halo reads as
// rhd_step_slabs, so that the slabs stay bit-identical to the whole grid.

// halo buffer of a slab: [2 sides][4 fields][HALO_PLANES][n0 n1], then the
// kappa and rho planes of the slab above and the TAU factors of the low face
static rhd_status slab_halo(rhd_ctx* c) {
  if (c->halo) return RHD_OK;
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  cudaError_t e = cudaMalloc(&c->halo, sizeof(double) * kHaloSlots * P);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->halo = nullptr;
    return fail(c, RHD_ERR_CUDA, "halo buffer: %s", cudaGetErrorString(e));
  }
  return RHD_OK;
}

// the hydrodynamic scratch and the primitives' halo buffer of a slab
// [2 sides][5 fields rho, vx, vy, vz, p][HALO_PLANES][n0 n1]
static rhd_status slab_hyd_halo(rhd_ctx* c) {
  rhd_status s = hydro_alloc(c);
  if (s != RHD_OK) return s;
  if (c->hyd_halo) return RHD_OK;
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  cudaError_t e = cudaMalloc(&c->hyd_halo, sizeof(double) * 2 * 5 * HALO_PLANES * P);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->hyd_halo = nullptr;
    return fail(c, RHD_ERR_CUDA, "halo buffer: %s", cudaGetErrorString(e));
  }
  return RHD_OK;
}

static int slab_depth(const rhd_ctx* c) {
  return c->p.reconstruction == RHD_RECON_PLM ? 2 : 3;
}

extern "C" {

int64_t rhd_slab_plane_doubles(const rhd_ctx* c, int what) {
  if (!c || c->p.ndim != 3) return -1;
  const int64_t P = (int64_t)c->g.n[0] * c->g.n[1];
  switch (what) {
    case RHD_SLAB_BOUNDARY_LOW:
    case RHD_SLAB_BOUNDARY_HIGH:
    case RHD_SLAB_GHOSTS_LOW:
    case RHD_SLAB_GHOSTS_HIGH: return 4 * slab_depth(c) * P;
    case RHD_SLAB_MATERIAL_LOW:
    case RHD_SLAB_MATERIAL_ABOVE: return 2 * P;
    case RHD_SLAB_EPS_HIGH:
    case RHD_SLAB_EPS_BELOW: return P;
    case RHD_SLAB_PRIM_BOUNDARY_LOW:
    case RHD_SLAB_PRIM_BOUNDARY_HIGH:
    case RHD_SLAB_PRIM_GHOSTS_LOW:
    case RHD_SLAB_PRIM_GHOSTS_HIGH: return 5 * slab_depth(c) * P;
    default: return -1;
  }
}

static rhd_status slab_check(rhd_ctx* c, int what, const void* buf, int64_t count) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!has_halo(c)) return fail(c, RHD_ERR_ARG, "the context has no HALO face");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (!buf) return fail(c, RHD_ERR_ARG, "buffer is NULL");
  const int64_t want = rhd_slab_plane_doubles(c, what);
  if (want < 0) return fail(c, RHD_ERR_ARG, "bad plane kind %d", what);
  if (count != want)
    return fail(c, RHD_ERR_ARG, "count %lld != %lld doubles", (long long)count, (long long)want);
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (what >= RHD_SLAB_PRIM_BOUNDARY_LOW) return slab_hyd_halo(c);
  return slab_halo(c);
}

rhd_status rhd_slab_planes_get(rhd_ctx* c, int what, int stage, double* dst, int64_t count,
                               int dst_on_device) {
  rhd_status s = slab_check(c, what, dst, count);
  if (s != RHD_OK) return s;
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (what == RHD_SLAB_BOUNDARY_LOW || what == RHD_SLAB_BOUNDARY_HIGH) {
    // stage 1 reads y(n), stage 2 y(n+1/2)
    if (stage == 1 && c->slab_phase != 0)
      return fail(c, RHD_ERR_STATE, "stage-1 planes: the slab is within a step");
    if (stage == 2 && c->slab_phase != 1)
      return fail(c, RHD_ERR_STATE, "stage-2 planes: stage 1 has not run");
    if (stage != 1 && stage != 2) return fail(c, RHD_ERR_ARG, "stage must be 1 or 2");
    const double* src = stage == 1 ? c->ybuf[c->cur] : c->yhalf;
    const int depth = slab_depth(c);
    const size_t z0 = what == RHD_SLAB_BOUNDARY_LOW ? 0 : (size_t)c->g.n[2] - depth;
    static const int kSlots[4] = {Y_ERAD, Y_FX, Y_FY, Y_FZ};
    for (int q = 0; q < 4; ++q)
      CUDA_TRY(c, cudaMemcpyAsync(dst + (size_t)q * depth * P,
                                  src + (size_t)kSlots[q] * c->ncell + z0 * P,
                                  sizeof(double) * depth * P, kind, c->stream));
  } else if (what == RHD_SLAB_MATERIAL_LOW) {
    CUDA_TRY(c, cudaMemcpyAsync(dst, c->kappa, sizeof(double) * P, kind, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(dst + P, c->rho, sizeof(double) * P, kind, c->stream));
  } else if (what == RHD_SLAB_EPS_HIGH) {
    if (c->p.hll_mode != RHD_HLL_TAU) return fail(c, RHD_ERR_ARG, "TAU factors: HLL mode NONE");
    const bool top = c->p.bc[2][1] == RHD_BC_HALO;
    if (top && !c->slab_mat_above)
      return fail(c, RHD_ERR_STATE, "TAU factors: the material plane of the slab above is "
                  "not set");
    if (c->eps_dirty) {
      double* hk = c->halo + (size_t)8 * HALO_PLANES * P;
      CUDA_TRY(c, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps,
                                 c->stream, top ? hk : nullptr, top ? hk + P : nullptr));
      c->launches += 1;
      c->eps_dirty = false;
    }
    CUDA_TRY(c, cudaMemcpyAsync(dst, c->eps[2] + (size_t)(c->g.n[2] - 1) * P,
                                sizeof(double) * P, kind, c->stream));
  } else if (what == RHD_SLAB_PRIM_BOUNDARY_LOW || what == RHD_SLAB_PRIM_BOUNDARY_HIGH) {
    // the primitives of the current hydrodynamic stage (after phase 0 or 2)
    if (c->slab_phase != 10 && c->slab_phase != 12)
      return fail(c, RHD_ERR_STATE, "primitive planes: run hydrodynamic phase 0 or 2 first");
    const int depth = slab_depth(c);
    const size_t z0 = what == RHD_SLAB_PRIM_BOUNDARY_LOW ? 0 : (size_t)c->g.n[2] - depth;
    for (int q = 0; q < 5; ++q)
      CUDA_TRY(c, cudaMemcpyAsync(dst + (size_t)q * depth * P,
                                  c->hyd_w + (size_t)q * c->ncell + z0 * P,
                                  sizeof(double) * depth * P, kind, c->stream));
  } else {
    return fail(c, RHD_ERR_ARG, "plane kind %d is set, not read", what);
  }
  if (!dst_on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RHD_OK;
}

rhd_status rhd_slab_planes_set(rhd_ctx* c, int what, const double* src, int64_t count,
                               int src_on_device) {
  rhd_status s = slab_check(c, what, src, count);
  if (s != RHD_OK) return s;
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  double* hk = c->halo + (size_t)8 * HALO_PLANES * P;
  if (what == RHD_SLAB_GHOSTS_LOW || what == RHD_SLAB_GHOSTS_HIGH) {
    const int side = what == RHD_SLAB_GHOSTS_LOW ? 0 : 1;
    if (c->p.bc[2][side] != RHD_BC_HALO)
      return fail(c, RHD_ERR_ARG, "ghost planes for a face that is not HALO");
    const int depth = slab_depth(c);
    // planes in z order: below, z = -depth..-1; above, z = n2..n2+depth-1
    const size_t i0 = side == 0 ? HALO_PLANES - depth : 0;
    double* h = c->halo + (size_t)side * 4 * HALO_PLANES * P;
    for (int q = 0; q < 4; ++q)
      CUDA_TRY(c, cudaMemcpyAsync(h + ((size_t)q * HALO_PLANES + i0) * P,
                                  src + (size_t)q * depth * P, sizeof(double) * depth * P, kind,
                                  c->stream));
  } else if (what == RHD_SLAB_MATERIAL_ABOVE) {
    if (c->p.bc[2][1] != RHD_BC_HALO) return fail(c, RHD_ERR_ARG, "the top face is not HALO");
    CUDA_TRY(c, cudaMemcpyAsync(hk, src, sizeof(double) * 2 * P, kind, c->stream));
    c->slab_mat_above = true;
    c->eps_dirty = true;
  } else if (what == RHD_SLAB_EPS_BELOW) {
    if (c->p.bc[2][0] != RHD_BC_HALO) return fail(c, RHD_ERR_ARG, "the low face is not HALO");
    CUDA_TRY(c, cudaMemcpyAsync(hk + 2 * P, src, sizeof(double) * P, kind, c->stream));
    c->slab_eps_below = true;
  } else if (what == RHD_SLAB_PRIM_GHOSTS_LOW || what == RHD_SLAB_PRIM_GHOSTS_HIGH) {
    const int side = what == RHD_SLAB_PRIM_GHOSTS_LOW ? 0 : 1;
    if (c->p.bc[2][side] != RHD_BC_HALO)
      return fail(c, RHD_ERR_ARG, "ghost planes for a face that is not HALO");
    const int depth = slab_depth(c);
    const size_t i0 = side == 0 ? HALO_PLANES - depth : 0;
    double* h = c->hyd_halo + (size_t)side * 5 * HALO_PLANES * P;
    for (int q = 0; q < 5; ++q)
      CUDA_TRY(c, cudaMemcpyAsync(h + ((size_t)q * HALO_PLANES + i0) * P,
                                  src + (size_t)q * depth * P, sizeof(double) * depth * P, kind,
                                  c->stream));
  } else {
    return fail(c, RHD_ERR_ARG, "plane kind %d is read, not set", what);
  }
  if (!src_on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return RHD_OK;
}

}  // extern "C"

extern "C" {

rhd_status rhd_slab_stage(rhd_ctx* c, int stage, double dt) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!has_halo(c)) return fail(c, RHD_ERR_ARG, "the context has no HALO face");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (stage != 1 && stage != 2) return fail(c, RHD_ERR_ARG, "stage must be 1 or 2");
  if (stage == 1 && c->slab_phase != 0)
    return fail(c, RHD_ERR_STATE, "stage 1: the previous step has not been committed");
  if (stage == 2 && c->slab_phase != 1) return fail(c, RHD_ERR_STATE, "stage 2 before stage 1");
  CUDA_TRY(c, cudaSetDevice(c->device));
  rhd_status s = slab_halo(c);
  if (s != RHD_OK) return s;
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  if (stage == 1) {
    if (!(dt > 0.0)) dt = rhd_default_dt(&c->p);
    if (!std::isfinite(dt)) return fail(c, RHD_ERR_ARG, "dt is not finite");
    if (c->p.hll_mode == RHD_HLL_TAU) {
      const bool top = c->p.bc[2][1] == RHD_BC_HALO, low = c->p.bc[2][0] == RHD_BC_HALO;
      if ((top && !c->slab_mat_above) || (low && !c->slab_eps_below))
        return fail(c, RHD_ERR_STATE, "TAU factors: the neighbours' material and factor "
                    "planes are not set (RHD_SLAB_MATERIAL_ABOVE, RHD_SLAB_EPS_BELOW)");
      if (c->eps_dirty) {
        double* hk = c->halo + (size_t)8 * HALO_PLANES * P;
        CUDA_TRY(c, launch_tau_eps(c->g, c->rho, c->kappa, c->ph.kappa_F_ratio, c->eps,
                                   c->stream, top ? hk : nullptr, top ? hk + P : nullptr));
        c->launches += 1;
        c->eps_dirty = false;
      }
    }
    CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
    c->launches += 1;
    c->slab_dt = dt;
  }
  StageArgs a;
  a.cell_base = 0;
  for (int d = 0; d < 3; ++d) a.eps[d] = c->eps[d];
  a.g = c->g;
  a.ph = c->ph;
  a.dt = c->slab_dt;
  a.step = 0;
  a.rho = c->rho;
  a.kappa = c->kappa;
  a.st = c->d_status;
  a.halo[0] = c->halo;
  a.halo[1] = c->halo + (size_t)4 * HALO_PLANES * P;
  a.eps_zlo = c->halo + (size_t)8 * HALO_PLANES * P + 2 * P;
  const int N = c->ncell;
  if (stage == 1) {
    slots_of<const double*>(a.yt, c->ybuf[c->cur], N);
    slots_of<const double*>(a.yn, c->ybuf[c->cur], N);
    slots_of<double*>(a.yo, c->yhalf, N);
  } else {
    slots_of<const double*>(a.yt, c->yhalf, N);
    slots_of<const double*>(a.yn, c->ybuf[c->cur], N);
    slots_of<double*>(a.yo, c->ybuf[c->cur ^ 1], N);
  }
  a.cost = c->cost + (stage == 1 ? 0 : N);
  CUDA_TRY(c, launch_stage(stage, c->p.precision, a, c->stream));
  c->launches += 1;
  c->slab_phase = stage;
  return RHD_OK;
}

rhd_status rhd_slab_status(rhd_ctx* c, rhd_step_info* info) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->slab_phase != 2 && c->slab_phase != 13)
    return fail(c, RHD_ERR_STATE, "no slab step has run all its stages");
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const DevStatus& st = *c->h_status;
  rhd_status code = RHD_OK;
  int64_t cell = -1;
  if (st.fail_key != ~0ull) {
    code = (rhd_status)(st.fail_key & 0xffull);
    cell = (int64_t)(st.fail_key >> 8);
  }
  if (info) {
    clear_info(info, c->t);
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
    info->dt = c->slab_dt;
  }
  c->slab_phase = c->slab_phase == 2 ? 3 : 14;
  return code;
}

rhd_status rhd_slab_commit(rhd_ctx* c, int commit) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (c->slab_phase != 3 && c->slab_phase != 14)
    return fail(c, RHD_ERR_STATE, "the slab step's status was not read");
  if (c->slab_phase == 14) {
    // hydrodynamic step: phase 4 copies the staged result into the state
    c->slab_phase = 0;
    if (!commit) return RHD_OK;
    CUDA_TRY(c, cudaSetDevice(c->device));
    HydroBufs b = hydro_bufs(c);
    CUDA_TRY(c, launch_hydro_phase(4, c->g, c->p.gamma, c->p.reconstruction, c->slab_dt, b,
                                   c->d_status, 0, c->stream));
    c->launches += 1;
    c->t += c->slab_dt;
    c->eps_dirty = true;  // rho has changed
    c->slab_mat_above = c->slab_eps_below = false;
    return RHD_OK;
  }
  if (commit) {
    c->cur ^= 1;
    c->t += c->slab_dt;
  }
  c->slab_phase = 0;
  return RHD_OK;
}

}  // extern "C"

extern "C" {

rhd_status rhd_slab_hydro_speed(rhd_ctx* c, double* smax) {
  if (!c || !smax) return fail(c, RHD_ERR_ARG, "ctx or smax is NULL");
  if (!has_halo(c)) return fail(c, RHD_ERR_ARG, "the context has no HALO face");
  if (c->pending || c->slab_phase != 0)
    return fail(c, RHD_ERR_STATE, "a step is in progress");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  CUDA_TRY(c, cudaSetDevice(c->device));
  rhd_status s = slab_hyd_halo(c);
  if (s != RHD_OK) return s;
  HydroBufs b = hydro_bufs(c);
  CUDA_TRY(c, launch_hydro_speed(c->g, c->p.gamma, b, c->stream));
  c->launches += 1;
  unsigned long long bits = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bits, c->hyd_bits, sizeof(bits), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  memcpy(smax, &bits, sizeof(*smax));
  return RHD_OK;
}

rhd_status rhd_slab_hydro_phase(rhd_ctx* c, int phase, double dt) {
  if (!c) return fail(nullptr, RHD_ERR_ARG, "ctx is NULL");
  if (!has_halo(c)) return fail(c, RHD_ERR_ARG, "the context has no HALO face");
  if (c->pending) return fail(c, RHD_ERR_STATE, "a step batch is pending");
  if (c->fields_set != kAllFields)
    return fail(c, RHD_ERR_STATE, "not every field has been set (mask 0x%x)", c->fields_set);
  if (phase < 0 || phase > 3) return fail(c, RHD_ERR_ARG, "phase must be 0 .. 3");
  if ((phase == 0 && c->slab_phase != 0) || (phase > 0 && c->slab_phase != 9 + phase))
    return fail(c, RHD_ERR_STATE, "hydrodynamic phase %d out of order", phase);
  for (int d = 0; d < 2; ++d)
    if (c->p.bc[d][0] == RHD_BC_INFLOW || c->p.bc[d][1] == RHD_BC_INFLOW)
      return fail(c, RHD_ERR_ARG, "the hydrodynamic step takes periodic and reflecting axes");
  if (c->p.bc[2][0] == RHD_BC_INFLOW || c->p.bc[2][1] == RHD_BC_INFLOW)
    return fail(c, RHD_ERR_ARG, "the hydrodynamic step takes periodic and reflecting axes");
  CUDA_TRY(c, cudaSetDevice(c->device));
  rhd_status s = slab_hyd_halo(c);
  if (s != RHD_OK) return s;
  if (phase == 0) {
    if (!(dt > 0.0) || !std::isfinite(dt))
      return fail(c, RHD_ERR_ARG, "dt must be positive and finite (rhd_slab_hydro_speed "
                  "gives the CFL bound of the slab)");
    CUDA_TRY(c, launch_status_reset(c->d_status, c->stream));
    c->launches += 1;
    c->slab_dt = dt;
  }
  const size_t P = (size_t)c->g.n[0] * c->g.n[1];
  HydroBufs b = hydro_bufs(c);
  b.halo[0] = c->hyd_halo;
  b.halo[1] = c->hyd_halo + (size_t)5 * HALO_PLANES * P;
  b.cell_base = 0;
  CUDA_TRY(c, launch_hydro_phase(phase, c->g, c->p.gamma, c->p.reconstruction, c->slab_dt, b,
                                 c->d_status, 0, c->stream));
  c->launches += phase == 1 || phase == 3 ? 1 + c->p.ndim : 1;
  c->slab_phase = 10 + phase;
  return RHD_OK;
}

}  // extern "C"
