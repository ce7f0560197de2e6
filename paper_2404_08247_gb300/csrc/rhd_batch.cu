// rhd_batch.cu -- many independent 1-D and 2-D grids advanced together.
//
// All problems' fields live in pooled device arrays (problem p at a cell
// offset).  A step is two launches of one persistent kernel (stage 1, stage
// 2 of eq. imex1/imex2): each block repeatedly takes the next (problem, tile)
// work item from an atomic counter and runs the same tile body as the
// single-grid kernels (stage_tile), with the problem's own geometry, physics
// and time step.  The launch sequence of a batch of steps is captured once
// into a CUDA graph and replayed.  The 2-D tile shape and the number of
// resident blocks per SM are run-time choices (rhd_batch_configure), which
// the Python autotuner sets from timings.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rhd_tile.cuh"

using namespace rhd;

namespace {

struct ProblemDesc {
  Geometry g;
  Physics ph;
  double dt;
  long long offset;
};

struct WorkItem {
  int prob, x0, y0, kind;  // kind 0: a 1-D row tile, 1: a 2-D tile; 2, 3: the same
                           // with PPM faces
};

struct BatchArgs {
  const ProblemDesc* probs;
  const WorkItem* items;
  int nitems;
  int* counter;
  long long ntot;
  const double* yt;  // slot-major pools: slot q at base + q * ntot
  const double* yn;
  double* yo;
  const double* rho;
  const double* kappa;
  const double* eps0;
  const double* eps1;
  DevStatus* st;
  int step;
  unsigned char* cost;  // this stage's per-cell solve costs (pooled), or null
};

using Tile1 = TileT<1, 256, 1, 1>;
using Tile2a = TileT<2, 32, 8, 1>;
using Tile2b = TileT<2, 64, 4, 1>;
using Tile2c = TileT<2, 16, 16, 1>;
// PPM tiles (kinds 2, 3): the single-grid PPM shapes
using Tile1P = TileT<1, 256, 1, 1, true>;
using Tile2P = TileT<2, 32, 8, 1, true>;
constexpr int kBatchThreads = 256;

// PPMX: the batch holds PPM problems (the kernel then carries both tile kinds)
template <int STAGE, class T2, typename R, bool GEN, bool PPMX>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item, s_skip;
  if (threadIdx.x == 0) s_skip = (B.st->fail_key != ~0ull) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // a previous launch of this batch failed
  TileStats ts;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(B.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();  // every thread has read s_item before it is reused
    if (it >= B.nitems) break;
    const WorkItem w = B.items[it];
    const ProblemDesc& P = B.probs[w.prob];
    StageArgs A;
    A.g = P.g;
    A.ph = P.ph;
    A.dt = P.dt;
    A.step = B.step;
    A.st = B.st;
    A.cell_base = P.offset;
    const long long off = P.offset;
#pragma unroll
    for (int q = 0; q < NY; ++q) {
      A.yt[q] = B.yt + q * B.ntot + off;
      A.yn[q] = B.yn + q * B.ntot + off;
      A.yo[q] = B.yo + q * B.ntot + off;
    }
    A.rho = B.rho + off;
    A.kappa = B.kappa + off;
    A.eps[0] = B.eps0 ? B.eps0 + off : nullptr;
    A.eps[1] = B.eps1 ? B.eps1 + off : nullptr;
    A.eps[2] = nullptr;
    A.cost = B.cost ? B.cost + off : nullptr;
#pragma unroll
    for (int q = 0; q < 4; ++q) A.rate[q] = nullptr;
    if (w.kind == 0)
      stage_tile<STAGE, Tile1, R, GEN>(A, w.x0, 0, 0, smem_raw, ts);
    else if (!PPMX || w.kind == 1)
      stage_tile<STAGE, T2, R, GEN>(A, w.x0, w.y0, 0, smem_raw, ts);
    else if constexpr (PPMX) {
      if (w.kind == 2)
        stage_tile<STAGE, Tile1P, R, true>(A, w.x0, 0, 0, smem_raw, ts);
      else
        stage_tile<STAGE, Tile2P, R, true>(A, w.x0, w.y0, 0, smem_raw, ts);
    }
  }
  flush_stats<kBatchThreads>(B.st, ts);
}

template <class T2, typename R, bool PPMX>
size_t batch_smem() {
  size_t a = SmemT<Tile1, R>::BYTES, b = SmemT<T2, R>::BYTES;
  size_t m = a > b ? a : b;
  if (PPMX) {
    size_t c = SmemT<Tile1P, R>::BYTES, d = SmemT<Tile2P, R>::BYTES;
    m = m > c ? m : c;
    m = m > d ? m : d;
  }
  return m;
}

template <int STAGE, class T2, typename R, bool GEN, bool PPMX = false>
cudaError_t launch_batch_t(const BatchArgs& B, int grid, cudaStream_t s) {
  size_t sm = batch_smem<T2, R, PPMX>();
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<STAGE, T2, R, GEN, PPMX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  batch_kernel<STAGE, T2, R, GEN, PPMX><<<grid, kBatchThreads, sm, s>>>(B);
  return cudaGetLastError();
}

template <int STAGE, typename R, bool GEN>
cudaError_t launch_batch_r(int tile2d, const BatchArgs& B, int grid, cudaStream_t s) {
  switch (tile2d) {
    case 1: return launch_batch_t<STAGE, Tile2b, R, GEN>(B, grid, s);
    case 2: return launch_batch_t<STAGE, Tile2c, R, GEN>(B, grid, s);
    default: return launch_batch_t<STAGE, Tile2a, R, GEN>(B, grid, s);
  }
}

template <typename R, bool GEN>
cudaError_t launch_batch_p(int stage, int tile2d, const BatchArgs& B, int grid,
                           cudaStream_t s) {
  return stage == 1 ? launch_batch_r<1, R, GEN>(tile2d, B, grid, s)
                    : launch_batch_r<2, R, GEN>(tile2d, B, grid, s);
}

// general: some problem of the batch needs the general kernels; ppm: some
// problem has PPM faces (general kernels, the default 2-D tile shape)
cudaError_t launch_batch(int stage, int precision, bool general, bool ppm, int tile2d,
                         const BatchArgs& B, int grid, cudaStream_t s) {
  if (ppm) {
    if (precision == RHD_PREC_MIXED)
      return stage == 1 ? launch_batch_t<1, Tile2a, float, true, true>(B, grid, s)
                        : launch_batch_t<2, Tile2a, float, true, true>(B, grid, s);
    return stage == 1 ? launch_batch_t<1, Tile2a, double, true, true>(B, grid, s)
                      : launch_batch_t<2, Tile2a, double, true, true>(B, grid, s);
  }
  if (precision == RHD_PREC_MIXED)
    return general ? launch_batch_p<float, true>(stage, tile2d, B, grid, s)
                   : launch_batch_p<float, false>(stage, tile2d, B, grid, s);
  return general ? launch_batch_p<double, true>(stage, tile2d, B, grid, s)
                 : launch_batch_p<double, false>(stage, tile2d, B, grid, s);
}

const int kTileX[3] = {32, 64, 16};
const int kTileY[3] = {8, 4, 16};

void fill_desc(const rhd_params* p, ProblemDesc& d) {
  memset(&d, 0, sizeof(d));
  rhd::fill_geometry(p, d.g, d.ph);
  d.dt = rhd_default_dt(p);
}

}  // namespace

struct rhd_batch {
  int nprob = 0;
  int device = 0;
  int precision = 0;
  int num_sms = 0;
  std::vector<ProblemDesc> desc;
  std::vector<long long> offsets;
  long long ntot = 0;
  double* ybuf[2] = {nullptr, nullptr};
  double* yhalf = nullptr;
  double* rho = nullptr;
  double* kappa = nullptr;
  double* eps[2] = {nullptr, nullptr};
  unsigned char* cost = nullptr;  // solve costs of stage 1 and 2 (2 ntot bytes)
  ProblemDesc* d_desc = nullptr;
  WorkItem* d_items = nullptr;
  int nitems = 0;
  int* d_counter = nullptr;
  DevStatus* d_status = nullptr;
  DevStatus* h_status = nullptr;
  int* d_flag = nullptr;
  int* h_flag = nullptr;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  int cur = 0;
  std::vector<unsigned> set_mask;
  std::vector<char> eps_dirty;
  int tile2d = 0;
  int blocks_per_sm = 2;
  bool use_graphs = true;  // rhd_batch_use_graphs
  bool general = false;  // some problem needs the general kernels
  bool ppm = false;      // some problem has PPM faces
  int items_tile = -1;  // tile shape the work list was built for
  struct Graph {
    int nsteps, cur0, tile2d, bps;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  double t = 0.0;
  char err[512] = "";
};

static rhd_status bfail(rhd_batch* b, rhd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) memcpy(b->err, buf, sizeof(buf));
  set_global_error(buf);
  return s;
}

#define BTRY(b, call)                                                               \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return bfail((b), RHD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

static void drop_graphs(rhd_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

static void batch_release(rhd_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaFree(b->ybuf[0]);
  cudaFree(b->ybuf[1]);
  cudaFree(b->yhalf);
  cudaFree(b->rho);
  cudaFree(b->kappa);
  cudaFree(b->cost);
  cudaFree(b->eps[0]);
  cudaFree(b->eps[1]);
  cudaFree(b->d_desc);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->d_status);
  cudaFree(b->d_flag);
  cudaFreeHost(b->h_status);
  cudaFreeHost(b->h_flag);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

// (Re)build the work list for the current 2-D tile shape: 2-D tiles first
// (the larger items), then the 1-D rows, so the dynamic schedule ends on
// small items.
static rhd_status build_items(rhd_batch* b) {
  if (b->items_tile == b->tile2d) return RHD_OK;
  std::vector<WorkItem> items;
  // a batch with PPM problems runs the default 2-D tile shape for all
  const int shape = b->ppm ? 0 : b->tile2d;
  const int tx = kTileX[shape], ty = kTileY[shape];
  for (int pass = 0; pass < 2; ++pass)
    for (int p = 0; p < b->nprob; ++p) {
      const Geometry& g = b->desc[p].g;
      const int ppm = b->desc[p].ph.reconstruction != RHD_RECON_PLM ? 2 : 0;
      if (pass == 0 && g.ndim == 2) {
        for (int y0 = 0; y0 < g.n[1]; y0 += ty)
          for (int x0 = 0; x0 < g.n[0]; x0 += tx) items.push_back({p, x0, y0, 1 + ppm});
      } else if (pass == 1 && g.ndim == 1) {
        for (int x0 = 0; x0 < g.n[0]; x0 += 256) items.push_back({p, x0, 0, ppm});
      }
    }
  cudaFree(b->d_items);
  b->d_items = nullptr;
  BTRY(b, cudaMalloc(&b->d_items, sizeof(WorkItem) * items.size()));
  BTRY(b, cudaMemcpy(b->d_items, items.data(), sizeof(WorkItem) * items.size(),
                     cudaMemcpyHostToDevice));
  b->nitems = (int)items.size();
  b->items_tile = b->tile2d;
  return RHD_OK;
}

extern "C" {

rhd_status rhd_batch_init(const rhd_params* probs, int nprob, rhd_batch** out) {
  if (!out) return bfail(nullptr, RHD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || nprob < 1) return bfail(nullptr, RHD_ERR_ARG, "need at least one problem");
  char msg[256];
  for (int p = 0; p < nprob; ++p) {
    if (rhd_params_validate(&probs[p], msg, sizeof(msg)) != RHD_OK)
      return bfail(nullptr, RHD_ERR_ARG, "problem %d: %s", p, msg);
    if (probs[p].ndim > 2)
      return bfail(nullptr, RHD_ERR_ARG, "problem %d: the batch takes 1-D and 2-D grids", p);
    if (probs[p].precision != probs[0].precision)
      return bfail(nullptr, RHD_ERR_ARG, "problem %d: all problems share one precision", p);
  }
  rhd_batch* b = new rhd_batch();
  b->nprob = nprob;
  b->precision = probs[0].precision;
  b->desc.resize(nprob);
  b->offsets.resize(nprob + 1);
  long long off = 0;
  bool any_tau = false;
  for (int p = 0; p < nprob; ++p) {
    fill_desc(&probs[p], b->desc[p]);
    b->general = b->general || needs_general(b->desc[p].g, b->desc[p].ph);
    b->ppm = b->ppm || probs[p].reconstruction != RHD_RECON_PLM;
    b->desc[p].offset = off;
    b->offsets[p] = off;
    off += b->desc[p].g.ncell;
    any_tau = any_tau || probs[p].hll_mode == RHD_HLL_TAU;
  }
  b->offsets[nprob] = off;
  b->ntot = off;
  b->set_mask.assign(nprob, 0u);
  b->eps_dirty.assign(nprob, 1);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  const size_t N = (size_t)b->ntot;
  if (e == cudaSuccess) e = cudaMalloc(&b->ybuf[0], sizeof(double) * NY * N);
  if (e == cudaSuccess) e = cudaMalloc(&b->ybuf[1], sizeof(double) * NY * N);
  if (e == cudaSuccess) e = cudaMalloc(&b->yhalf, sizeof(double) * NY * N);
  if (e == cudaSuccess) e = cudaMalloc(&b->rho, sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMalloc(&b->kappa, sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMalloc(&b->cost, 2 * N);
  if (e == cudaSuccess) e = cudaMemset(b->cost, 0, 2 * N);
  if (any_tau) {
    if (e == cudaSuccess) e = cudaMalloc(&b->eps[0], sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&b->eps[1], sizeof(double) * N);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, sizeof(ProblemDesc) * nprob);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_desc, b->desc.data(), sizeof(ProblemDesc) * nprob,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    bfail(nullptr, RHD_ERR_CUDA, "batch allocation: %s", cudaGetErrorString(e));
    batch_release(b);
    return RHD_ERR_CUDA;
  }
  b->stream = b->own;
  rhd_status s = build_items(b);
  if (s != RHD_OK) {
    batch_release(b);
    return s;
  }
  *out = b;
  return RHD_OK;
}

rhd_status rhd_batch_set_stream(rhd_batch* b, void* stream) {
  if (!b) return bfail(nullptr, RHD_ERR_ARG, "batch is NULL");
  BTRY(b, cudaSetDevice(b->device));
  BTRY(b, cudaStreamSynchronize(b->stream));
  b->stream = (cudaStream_t)stream;
  drop_graphs(b);  // graphs are launched on the stream they were captured for
  return RHD_OK;
}

rhd_status rhd_batch_configure(rhd_batch* b, int tile2d, int blocks_per_sm) {
  if (!b) return bfail(nullptr, RHD_ERR_ARG, "batch is NULL");
  if (tile2d < 0 || tile2d > 2) return bfail(b, RHD_ERR_ARG, "tile2d must be 0, 1 or 2");
  if (blocks_per_sm < 1 || blocks_per_sm > 2)
    return bfail(b, RHD_ERR_ARG, "blocks_per_sm must be 1 or 2");
  BTRY(b, cudaSetDevice(b->device));
  BTRY(b, cudaStreamSynchronize(b->stream));
  b->tile2d = tile2d;
  b->blocks_per_sm = blocks_per_sm;
  return build_items(b);
}

int64_t rhd_batch_cells(const rhd_batch* b, int prob) {
  if (!b) return -1;
  if (prob < 0) return b->ntot;
  if (prob >= b->nprob) return -1;
  return b->offsets[prob + 1] - b->offsets[prob];
}

static rhd_status batch_copy_args(rhd_batch* b, int prob, const void* ptr, int64_t count) {
  if (!b) return bfail(nullptr, RHD_ERR_ARG, "batch is NULL");
  if (prob < 0 || prob >= b->nprob) return bfail(b, RHD_ERR_ARG, "bad problem %d", prob);
  if (!ptr) return bfail(b, RHD_ERR_ARG, "buffer is NULL");
  long long n = b->offsets[prob + 1] - b->offsets[prob];
  if (count != RHD_NFIELDS * n)
    return bfail(b, RHD_ERR_ARG, "count must be RHD_NFIELDS * %lld", n);
  return RHD_OK;
}

static double* batch_field(rhd_batch* b, int prob, int field) {
  const long long off = b->offsets[prob];
  switch (field) {
    case RHD_F_RHO: return b->rho + off;
    case RHD_F_KAPPA: return b->kappa + off;
    case RHD_F_EGAS: return b->ybuf[b->cur] + Y_EGAS * b->ntot + off;
    case RHD_F_MX: return b->ybuf[b->cur] + Y_MX * b->ntot + off;
    case RHD_F_MY: return b->ybuf[b->cur] + Y_MY * b->ntot + off;
    case RHD_F_MZ: return b->ybuf[b->cur] + Y_MZ * b->ntot + off;
    case RHD_F_ERAD: return b->ybuf[b->cur] + Y_ERAD * b->ntot + off;
    case RHD_F_FX: return b->ybuf[b->cur] + Y_FX * b->ntot + off;
    case RHD_F_FY: return b->ybuf[b->cur] + Y_FY * b->ntot + off;
    default: return b->ybuf[b->cur] + Y_FZ * b->ntot + off;
  }
}

rhd_status rhd_batch_state_set(rhd_batch* b, int prob, const double* src, int64_t count,
                               int src_on_device) {
  rhd_status s = batch_copy_args(b, prob, src, count);
  if (s != RHD_OK) return s;
  BTRY(b, cudaSetDevice(b->device));
  const long long n = b->offsets[prob + 1] - b->offsets[prob];
  BTRY(b, cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream));
  for (int f = 0; f < RHD_NFIELDS; ++f) {
    BTRY(b, cudaMemcpyAsync(batch_field(b, prob, f), src + (size_t)f * n,
                            sizeof(double) * n,
                            src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            b->stream));
    BTRY(b, launch_check_field(f, batch_field(b, prob, f), (int)n, b->d_flag, b->stream));
  }
  if (b->desc[prob].ph.hll_mode == RHD_HLL_TAU) {
    double* eps[3] = {b->eps[0] + b->offsets[prob], b->eps[1] + b->offsets[prob], nullptr};
    BTRY(b, launch_tau_eps(b->desc[prob].g, batch_field(b, prob, RHD_F_RHO),
                           batch_field(b, prob, RHD_F_KAPPA), b->desc[prob].ph.kappa_F_ratio,
                           eps, b->stream));
  }
  BTRY(b, cudaMemcpyAsync(b->h_flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                          b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  if (*b->h_flag) {
    b->set_mask[prob] = 0;
    return bfail(b, RHD_ERR_ARG, "problem %d holds a non-finite or out-of-range value", prob);
  }
  b->set_mask[prob] = 1;
  return RHD_OK;
}

rhd_status rhd_batch_state_get(rhd_batch* b, int prob, double* dst, int64_t count,
                               int dst_on_device) {
  rhd_status s = batch_copy_args(b, prob, dst, count);
  if (s != RHD_OK) return s;
  BTRY(b, cudaSetDevice(b->device));
  const long long n = b->offsets[prob + 1] - b->offsets[prob];
  for (int f = 0; f < RHD_NFIELDS; ++f)
    BTRY(b, cudaMemcpyAsync(dst + (size_t)f * n, batch_field(b, prob, f), sizeof(double) * n,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  return RHD_OK;
}

// Enqueue nsteps steps on stream cs (status reset, then per stage a counter
// reset and one persistent launch) starting from ping-pong buffer cur0.
static cudaError_t enqueue_steps(rhd_batch* b, int nsteps, int cur0, cudaStream_t cs) {
  BatchArgs B;
  B.probs = b->d_desc;
  B.items = b->d_items;
  B.nitems = b->nitems;
  B.counter = b->d_counter;
  B.ntot = b->ntot;
  B.rho = b->rho;
  B.kappa = b->kappa;
  B.eps0 = b->eps[0];
  B.eps1 = b->eps[1];
  B.st = b->d_status;
  int grid = b->num_sms * b->blocks_per_sm;
  if (grid > b->nitems) grid = b->nitems;
  cudaError_t e = launch_status_reset(b->d_status, cs);
  int cur = cur0;
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
    B.step = s;
    B.yt = b->ybuf[cur];
    B.yn = b->ybuf[cur];
    B.yo = b->yhalf;
    B.cost = b->cost;
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), cs);
    if (e == cudaSuccess)
      e = launch_batch(1, b->precision, b->general, b->ppm, b->tile2d, B, grid, cs);
    B.yt = b->yhalf;
    B.yo = b->ybuf[cur ^ 1];
    B.cost = b->cost + b->ntot;
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), cs);
    if (e == cudaSuccess)
      e = launch_batch(2, b->precision, b->general, b->ppm, b->tile2d, B, grid, cs);
    cur ^= 1;
  }
  return e;
}

// Capture the launches of enqueue_steps into a graph.
static rhd_status capture(rhd_batch* b, int nsteps, int cur0, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = b->stream ? b->stream : b->own;  // the legacy stream cannot capture
  BTRY(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_steps(b, nsteps, cur0, cs);
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, RHD_ERR_CUDA, "graph capture: %s",
                 cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, RHD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return RHD_OK;
}

rhd_status rhd_batch_step(rhd_batch* b, int nsteps, rhd_step_info* info) {
  if (!b) return bfail(nullptr, RHD_ERR_ARG, "batch is NULL");
  if (nsteps < 1) return bfail(b, RHD_ERR_ARG, "nsteps must be >= 1");
  for (int p = 0; p < b->nprob; ++p)
    if (!b->set_mask[p]) return bfail(b, RHD_ERR_STATE, "problem %d has no state", p);
  BTRY(b, cudaSetDevice(b->device));
  cudaGraphExec_t exec = nullptr;
  if (b->use_graphs) {
    for (auto& g : b->graphs)
      if (g.nsteps == nsteps && g.cur0 == b->cur && g.tile2d == b->tile2d &&
          g.bps == b->blocks_per_sm)
        exec = g.exec;
    if (!exec) {
      rhd_status s = capture(b, nsteps, b->cur, &exec);
      if (s != RHD_OK) return s;
      b->graphs.push_back({nsteps, b->cur, b->tile2d, b->blocks_per_sm, exec});
    }
  }
  // graphs run on the batch stream, or on the private stream (after the
  // legacy stream's earlier work) when the batch stream is the legacy one
  cudaStream_t rs = b->stream ? b->stream : b->own;
  if (!b->stream) BTRY(b, cudaStreamSynchronize(nullptr));
  if (exec)
    BTRY(b, cudaGraphLaunch(exec, rs));
  else
    BTRY(b, enqueue_steps(b, nsteps, b->cur, rs));
  BTRY(b, cudaMemcpyAsync(b->h_status, b->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                          rs));
  BTRY(b, cudaStreamSynchronize(rs));
  const DevStatus& st = *b->h_status;
  rhd_status code = RHD_OK;
  int done = nsteps;
  int64_t cell = -1;
  if (st.fail_key != ~0ull) {
    code = (rhd_status)(st.fail_key & 0xffull);
    cell = (int64_t)(st.fail_key >> 8);
    done = st.fail_step;
  }
  b->cur ^= (done & 1);
  b->t += done;  // counts steps: every problem has its own dt
  if (info) {
    memset(info, 0, sizeof(*info));
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
    info->t = b->t;
    info->dt = 0.0;
  }
  if (code != RHD_OK)
    return bfail(b, code, "step %d stage %d failed at pooled cell %lld (status %d)",
                 st.fail_step, st.fail_stage, (long long)cell, (int)code);
  return RHD_OK;
}

rhd_status rhd_batch_use_graphs(rhd_batch* b, int enable) {
  if (!b) return bfail(nullptr, RHD_ERR_ARG, "batch is NULL");
  b->use_graphs = enable != 0;
  return RHD_OK;
}

rhd_status rhd_batch_locate(const rhd_batch* b, int64_t pooled_cell, int* prob,
                            int64_t* cell) {
  if (!b || !prob || !cell) return RHD_ERR_ARG;
  if (pooled_cell < 0 || pooled_cell >= b->ntot) return RHD_ERR_ARG;
  int lo = 0, hi = b->nprob;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (b->offsets[mid] <= pooled_cell) lo = mid; else hi = mid;
  }
  *prob = lo;
  *cell = pooled_cell - b->offsets[lo];
  return RHD_OK;
}

const char* rhd_batch_last_error(const rhd_batch* b) { return b ? b->err : ""; }

void rhd_batch_destroy(rhd_batch* b) { batch_release(b); }

}  // extern "C"
