// sip_api.cu -- host runtime and C ABI of libsip.so (declared in include/sip.h).
//
// A plan (the paper's redesigned solver module, arXiv:1303.4538 Sec. 4.1: the
// solver owns its coefficient arrays and computes the incomplete factorisation
// once, before the relaxations) holds, for every block, the plane layout
// tables, per-cell records with the reordered coefficients and Stone's
// factors, the work vectors, the face buffers of the sweeps and a
// device-resident control block.  All launches go to the context's stream;
// the only device->host transfers are the control block reads that a call
// needs to return its results.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sip.h"
#include "sip_internal.h"
#include "sip_kernels.h"

using namespace sipk;

struct sip_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  size_t smem_optin = 0;
  std::string err = "no error";
  size_t kernel_static_smem = 0;  // largest static shared memory of any sweep kernel
  // Device memory of the context's plans comes from its own stream-ordered
  // pool (allocated and freed in stream order on `stream`): creating and
  // destroying plans never synchronises the device, so the slots of a server
  // admit and retire requests while other slots' kernels run.  Null: plain
  // cudaMalloc / cudaFree.
  cudaMemPool_t mempool = nullptr;
  // bytes the pool keeps cached across synchronisations: at least kPoolKeep,
  // raised to the largest footprint a plan creation reached unless the
  // context serves a solve server slot (whose requests are budgeted)
  unsigned long long pool_keep = 0;
  bool keep_peak = true;
  // pinned host control blocks of destroyed plans, reused by the next plans
  std::mutex pin_mu;
  std::vector<void *> pinned;
};
constexpr size_t kPinnedBlock = 256;  // 3 Ctl + 2 status words, rounded up
constexpr unsigned long long kPoolKeep = 1ull << 30;  // bytes a context's pool keeps cached

static std::string g_create_error = "no error";

namespace sipk {
void ctx_keep_peak(sip_ctx *ctx, bool on) {
  if (ctx) ctx->keep_peak = on;
}
}  // namespace sipk

namespace {

int fail(sip_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define CU(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SIP_ERR_OOM : SIP_ERR_CUDA,  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                \
    }                                                                                 \
  } while (0)

// Plane layout tables of a block: PO[s] = first cell of plane s, F[m] = number
// of (i, j) with i + j <= m (cells of one (j, k) cross-section diagonal).
void build_tables(int nx, int ny, int nz, std::vector<int> &PO, std::vector<int> &F) {
  const int np = nx + ny + nz - 2, mmax = nx + ny - 2;
  F.assign(mmax + 1, 0);
  long long acc = 0;
  for (int m = 0; m <= mmax; ++m) {
    const int lo = std::max(0, m - (nx - 1)), hi = std::min(ny - 1, m);
    acc += std::max(0, hi - lo + 1);
    F[m] = (int)acc;
  }
  PO.assign(np, 0);
  long long off = 0;
  for (int s = 0; s < np; ++s) {
    PO[s] = (int)off;
    const int klo = std::max(0, s - mmax), khi = std::min(nz - 1, s);
    for (int k = klo; k <= khi; ++k) off += F[s - k] - (s - k > 0 ? F[s - k - 1] : 0);
  }
}

}  // namespace

struct BlockHost {
  sip_block_desc d;
  DevBlock db;
  std::vector<int> PO, F;
  long long n = 0;
};

struct sip_plan {
  sip_ctx *ctx = nullptr;
  sip_options opt;
  int mode = 0;
  bool sym = false;
  bool a32in = false;
  std::vector<BlockHost> blocks;
  long long ncells = 0;
  int ntiles = 0;
  int Q = 2, NW = 8, NT = 256, TK = 16, tab_ints = 0;
  int Rk[K_NKINDS] = {};     // stage depth chosen per kernel kind
  int gridk[K_NKINDS] = {};  // resident CTAs per kernel kind (grid of the ticketed sweeps)
  std::vector<void *> allocs;
  size_t bytes = 0;
  DevBlock *d_blocks = nullptr;
  Tile *d_tiles_f = nullptr, *d_tiles_b = nullptr;
  int *d_tab = nullptr;
  void *recF = nullptr, *recB = nullptr;  // L and U records, FP64 (F64 mode) or FP32
  void *recA = nullptr;                   // A records in the sweep precision
  double *arec64 = nullptr;               // refined mode, FP64 coefficients: FP64 A of the outer residual
  long long nrows = 0;                    // plane rows of all blocks (row-parallel kernels)
  int rowgrid = 1;                        // CTAs of a row-parallel launch (plan constant: fixes the norm's sum order)
  double *b64 = nullptr, *x64 = nullptr, *y64 = nullptr;
  float *r32 = nullptr, *d32 = nullptr, *y32 = nullptr;
  uint64_t *faces = nullptr;
  double *partials = nullptr;  // [rowgrid] per-CTA sums of r^2
  double *bparts = nullptr;
  int nbparts = 1024;
  Ctl *ctl = nullptr;
  double *hist = nullptr;
  int hist_cap = 0;
  int *status = nullptr;
  int *tickets = nullptr;
  Ctl *h_ctl = nullptr;     // pinned [3]: two chunk snapshots, one final
  int *h_status = nullptr;  // pinned [2]
  int last_nhist = 0;
  long long launches = 0;  // kernels launched by this plan
  // kernel timing (sip_profile_*): event pairs per launch, read back lazily
  bool prof = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double prof_ms[K_NKINDS + 1] = {};
  long long prof_n[K_NKINDS + 1] = {};
  // diagnostics: with SIP_TRACE=<file> in the environment every sweep launch
  // records per-tile timestamps; the last launch of each kind is written to
  // <file> when the plan is destroyed
  unsigned long long *trace = nullptr;
  std::string trace_path;
  // multi-block interfaces: lagged coupling terms folded into beff64 (the
  // right-hand side the residual kernels read) before every iteration
  std::vector<sip_interface> ifaces;
  double *beff64 = nullptr;
  float *hsave32 = nullptr;  // refined mode: interface cells' r32 from the outer residual
  HaloEntry *halo = nullptr;
  int nhalo = 0;
  // captured iterations (sip_options.graphs): graph[0] replays one iteration,
  // graph[1] a chunk of kChunk iterations; kernels launched per replay
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long long graph_kernels[2] = {0, 0};
};

// ------------------------------------------------------------------ helpers
namespace {

cudaError_t ctx_alloc(sip_ctx *ctx, void **v, size_t b) {
  if (ctx->mempool) return cudaMallocFromPoolAsync(v, b, ctx->mempool, ctx->stream);
  return cudaMalloc(v, b);
}

void ctx_free(sip_ctx *ctx, void *v) {
  if (ctx->mempool) cudaFreeAsync(v, ctx->stream);
  else cudaFree(v);
}

// After a plan's allocations: keep the pool's peak cached, so that creating
// a plan of the same size again re-maps no memory.
void pool_keep_peak(sip_ctx *ctx) {
  if (!ctx->mempool || !ctx->keep_peak) return;
  unsigned long long hi = 0;
  if (cudaMemPoolGetAttribute(ctx->mempool, cudaMemPoolAttrUsedMemHigh, &hi) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (hi > ctx->pool_keep && cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrReleaseThreshold, &hi) ==
                                 cudaSuccess)
    ctx->pool_keep = hi;
  cudaGetLastError();
}

void *pinned_take(sip_ctx *ctx) {
  {
    std::lock_guard<std::mutex> lk(ctx->pin_mu);
    if (!ctx->pinned.empty()) {
      void *v = ctx->pinned.back();
      ctx->pinned.pop_back();
      return v;
    }
  }
  void *v = nullptr;
  return cudaMallocHost(&v, kPinnedBlock) == cudaSuccess ? v : nullptr;
}

void pinned_give(sip_ctx *ctx, void *v) {
  if (!v) return;
  std::lock_guard<std::mutex> lk(ctx->pin_mu);
  ctx->pinned.push_back(v);
}

template <typename T>
cudaError_t palloc(sip_plan *p, T **ptr, size_t count) {
  void *v = nullptr;
  const size_t b = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = ctx_alloc(p->ctx, &v, b);
  if (e != cudaSuccess) return e;
  p->allocs.push_back(v);
  p->bytes += b;
  *ptr = (T *)v;
  return cudaSuccess;
}

void pfree(sip_plan *p, void *v, size_t bytes) {
  auto it = std::find(p->allocs.begin(), p->allocs.end(), v);
  if (it != p->allocs.end()) {
    p->allocs.erase(it);
    p->bytes -= bytes;
    ctx_free(p->ctx, v);
  }
}

void free_plan_memory(sip_plan *p) {
  for (auto &g : p->graph)
    if (g) cudaGraphExecDestroy(g);
  p->graph[0] = p->graph[1] = nullptr;
  for (auto &r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  p->recs.clear();
  for (auto e : p->pool) cudaEventDestroy(e);
  p->pool.clear();
  for (void *v : p->allocs) ctx_free(p->ctx, v);
  p->allocs.clear();
  pinned_give(p->ctx, p->h_ctl);  // h_status lives in the same block
  p->h_ctl = nullptr;
  p->h_status = nullptr;
}

int max_active(const void *f, int NT, size_t smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, NT, smem) != cudaSuccess) return 0;
  return occ;
}

SweepCommon common(sip_plan *p, bool backward, int ticket, int reset, int slot, int kind) {
  SweepCommon c;
  c.trace = p->trace ? p->trace + (size_t)kind * p->ntiles * kTraceWords : nullptr;
  c.blocks = p->d_blocks;
  c.tiles = backward ? p->d_tiles_b : p->d_tiles_f;
  c.ntiles = p->ntiles;
  c.tab_ints = p->tab_ints;
  c.ticket = p->tickets + ticket;
  c.reset_ticket = reset >= 0 ? p->tickets + reset : nullptr;
  c.ctl = p->ctl;
  c.ep_slot = slot;
  c.stall = p->opt.debug_stall ? 1 : 0;
  c.faces = p->faces;
  c.status = p->status;
  c.max_spin = p->opt.max_spin > 0 ? p->opt.max_spin : (1ll << 22);
  return c;
}

cudaEvent_t take_event(sip_plan *p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Event pair around a launch when profiling; kind K_NKINDS = utility kernels.
struct ProfScope {
  sip_plan *p;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(sip_plan *p_, int k) : p(p_), kind(k) {
    ++p->launches;
    if (p->prof) {
      a = take_event(p);
      cudaEventRecord(a, p->ctx->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = take_event(p);
      cudaEventRecord(b, p->ctx->stream);
      p->recs.push_back({kind, a, b});
    }
  }
};

template <typename Params>
cudaError_t launch(sip_plan *p, int kind, const Params &prm) {
  const int R = p->Rk[kind];
  const size_t smem = kernel_smem(kind, p->Q, R, p->NT, p->tab_ints);
  const int grid = std::max(1, std::min(p->ntiles, p->gridk[kind]));
  void *args[] = {(void *)&prm};
  ProfScope ps(p, kind);
  return cudaLaunchKernel(kernel_ptr(kind, p->Q, R), dim3(grid), dim3(p->NT), args, smem, p->ctx->stream);
}

// utility launches (layout, reductions, control) are counted as kind K_NKINDS
#define UTIL(call)              \
  do {                          \
    ProfScope ps_(p, K_NKINDS); \
    CU(call);                   \
  } while (0)

int check_status(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  int st = 0;
  CU(cudaMemcpyAsync(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (st == DEV_TIMEOUT)
    return fail(ctx, SIP_ERR_DEVICE_TIMEOUT, "a bounded device wait timed out (inter-tile face never arrived)");
  if (st == DEV_BREAKDOWN)
    return fail(ctx, SIP_ERR_BREAKDOWN, "SIP factorisation broke down (zero or non-finite pivot)");
  if (st != DEV_OK) return fail(ctx, SIP_ERR_CUDA, "unknown device status");
  return SIP_OK;
}

// Forward + finalize + backward of one FP64 iteration.
// Interface terms of the coupled residual from the current x (lagged block Jacobi).
int enqueue_halo(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  if (p->nhalo > 0 && p->mode == SIP_MODE_F32)
    UTIL(launch_cast_f32_f64(p->d32, p->x64, p->ncells, ctx->stream));  // the FP32 iterate is the current x
  if (p->nhalo > 0) UTIL(launch_halo(p->halo, p->nhalo, p->b64, p->x64, p->beff64, p->ctl, ctx->stream));
  return SIP_OK;
}

// Residual r = b - A x over the whole plan (row-parallel kernel), with the
// per-CTA r^2 partials when `norm`.
template <typename TA, typename TX, typename TR>
int enqueue_resid(sip_plan *p, int kind, const TA *arec, const TX *b, const TX *x, TR *r, bool norm) {
  sip_ctx *ctx = p->ctx;
  RowParams<TA, TX, TR> prm;
  prm.blocks = p->d_blocks;
  prm.nblocks = (int)p->blocks.size();
  prm.nrows = p->nrows;
  prm.ctl = p->ctl;
  prm.status = p->status;
  prm.arec = arec;
  prm.b = b;
  prm.x = x;
  prm.r = r;
  prm.partials = norm ? p->partials : nullptr;
  ProfScope ps(p, kind);
  CU(launch_resrow(prm, p->sym, p->rowgrid, ctx->stream));
  return SIP_OK;
}

// Forward substitution y = L^-1 r (in place when r == y).
template <typename T>
int enqueue_forward(sip_plan *p, int kind, const T *r, T *y) {
  sip_ctx *ctx = p->ctx;
  FwdParams<T> f;
  f.c = common(p, false, 0, 1, 0, kind);
  f.rec = (const T *)p->recF;
  f.r = r;
  f.y = y;
  CU(launch(p, kind, f));
  return SIP_OK;
}

// Backward substitution d = U^-1 y and the update x <- x + d.
template <typename T>
int enqueue_backward(sip_plan *p, int kind, const T *y, T *x) {
  sip_ctx *ctx = p->ctx;
  BwdParams<T> b;
  b.c = common(p, true, 1, 0, 1, kind);
  b.rec = (const T *)p->recB;
  b.y = y;
  b.x = x;
  CU(launch(p, kind, b));
  return SIP_OK;
}

int enqueue_relres(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  UTIL(launch_finalize(p->partials, p->rowgrid, p->ctl, p->hist, p->hist_cap, p->status, FIN_RELRES, ctx->stream));
  return SIP_OK;
}

// One FP64 SIP iteration (Sec. 1): r = b - A x and its norm (stop rule),
// y = L^-1 r in place, then x <- x + U^-1 y.
int enqueue_iter_f64(sip_plan *p) {
  if (int rc = enqueue_halo(p)) return rc;
  const double *b = p->beff64 ? p->beff64 : p->b64;
  if (int rc = enqueue_resid(p, K_RES64, (const double *)p->recA, b, p->x64, p->y64, true)) return rc;
  if (int rc = enqueue_relres(p)) return rc;
  if (int rc = enqueue_forward(p, K_FWD64, p->y64, p->y64)) return rc;
  return enqueue_backward(p, K_BWD64, p->y64, p->x64);
}

// One FP64 correction of the refinement: FP64 residual (+ stop rule), then
// m FP32 SIP iterations on A d = r from d = 0, then x64 += (double) d.
int enqueue_iter_refined(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  const int m = std::max(1, p->opt.inner_iters);
  if (int rc = enqueue_halo(p)) return rc;
  const double *bres = p->beff64 ? p->beff64 : p->b64;
  int rc = p->arec64 ? enqueue_resid(p, K_RES64R, (const double *)p->arec64, bres, p->x64, p->r32, true)
                     : enqueue_resid(p, K_RES64R, (const float *)p->recA, bres, p->x64, p->r32, true);
  if (rc) return rc;
  if ((rc = enqueue_relres(p))) return rc;
  for (int q = 0; q < m; ++q) {
    const bool first = q == 0;
    if (first) {
      rc = enqueue_forward(p, K_FWD32, (const float *)p->r32, p->y32);  // d = 0: the residual is r
    } else {
      // exchange: the interface terms of the neighbours' current correction
      // (the inner system is the coupled one)
      if (p->nhalo > 0)
        UTIL(launch_halo32(p->halo, p->nhalo, p->r32, p->d32, p->hsave32, q == 1, p->ctl, ctx->stream));
      rc = enqueue_resid(p, K_RES32, (const float *)p->recA, (const float *)p->r32, (const float *)p->d32, p->y32,
                         false);
      if (!rc) rc = enqueue_forward(p, K_FWD32, (const float *)p->y32, p->y32);
    }
    if (rc) return rc;
    if ((rc = enqueue_backward(p, first ? K_BWD32Z : K_BWD32, (const float *)p->y32, p->d32))) return rc;
  }
  {
    ProfScope ps(p, K_UPD64);
    CU(launch_update64(p->d32, p->x64, p->ncells, p->ctl, ctx->stream));
  }
  return SIP_OK;
}

// One single-precision SIP iteration (the paper's FP32 relaxation, Sec. 4.1):
// residual, norm and forward substitution in FP32 on the converted rhs
// (r32) and solution (d32), then the FP32 backward substitution and update.
int enqueue_iter_f32(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  if (int rc = enqueue_halo(p)) return rc;
  if (p->nhalo > 0) UTIL(launch_cast_f64_f32(p->beff64, p->r32, p->ncells, ctx->stream));
  if (int rc = enqueue_resid(p, K_RES32N, (const float *)p->recA, (const float *)p->r32, (const float *)p->d32,
                             p->y32, true))
    return rc;
  if (int rc = enqueue_relres(p)) return rc;
  if (int rc = enqueue_forward(p, K_FWD32, (const float *)p->y32, p->y32)) return rc;
  return enqueue_backward(p, K_BWD32, (const float *)p->y32, p->d32);
}

int enqueue_iter(sip_plan *p) {
  if (p->mode == SIP_MODE_F32_REFINED) return enqueue_iter_refined(p);
  if (p->mode == SIP_MODE_F32) return enqueue_iter_f32(p);
  return enqueue_iter_f64(p);
}

constexpr int kChunk = 16;  // iterations queued per host check of the control block

// Capture `iters` iterations of the plan into an executable graph.  Every
// launch of an iteration has plan-constant arguments (epochs, tickets and the
// stop flag live in device memory), so one capture replays any iteration.
int capture_iters(sip_plan *p, int slot, int iters) {
  sip_ctx *ctx = p->ctx;
  const long long l0 = p->launches;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  int rc = SIP_OK;
  for (int it = 0; it < iters && rc == SIP_OK; ++it) rc = enqueue_iter(p);
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  if (rc != SIP_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, SIP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&p->graph[slot], g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) {
    p->graph[slot] = nullptr;
    return fail(ctx, SIP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
  }
  p->graph_kernels[slot] = p->launches - l0;
  p->launches = l0;
  return SIP_OK;
}

// Queue n iterations: from the captured graphs when the plan uses them (and
// no per-launch profiling is on), else launch by launch.
int enqueue_iters(sip_plan *p, int n) {
  sip_ctx *ctx = p->ctx;
  if (!p->opt.graphs || p->prof || ctx->stream == nullptr) {
    for (int it = 0; it < n; ++it)
      if (int rc = enqueue_iter(p)) return rc;
    return SIP_OK;
  }
  while (n > 0) {
    const int slot = n >= kChunk ? 1 : 0;
    if (!p->graph[slot])
      if (int rc = capture_iters(p, slot, slot ? kChunk : 1)) return rc;
    CU(cudaGraphLaunch(p->graph[slot], ctx->stream));
    p->launches += p->graph_kernels[slot];
    n -= slot ? kChunk : 1;
  }
  return SIP_OK;
}

// Copy b and x of every block into the plan layout, ||b||, control reset.
int begin_sequence(sip_plan *p, double rtol, int max_iters) {
  sip_ctx *ctx = p->ctx;
  CU(cudaMemsetAsync(p->tickets, 0, 4 * sizeof(int), ctx->stream));
  UTIL(launch_set_ctl(p->ctl, rtol, max_iters, ctx->stream));
  for (auto &bh : p->blocks) {
    UTIL(launch_to_plan_f64(bh.d.b, p->b64, bh.db, ctx->stream));
    UTIL(launch_to_plan_f64(bh.d.x, p->x64, bh.db, ctx->stream));
  }
  if (p->beff64)
    CU(cudaMemcpyAsync(p->beff64, p->b64, (size_t)p->ncells * sizeof(double), cudaMemcpyDeviceToDevice,
                       ctx->stream));
  UTIL(launch_sumsq_partials(p->b64, p->ncells, p->bparts, p->nbparts, ctx->stream));
  if (p->mode == SIP_MODE_F32) {  // rhs and solution converted to single precision
    UTIL(launch_cast_f64_f32(p->b64, p->r32, p->ncells, ctx->stream));
    UTIL(launch_cast_f64_f32(p->x64, p->d32, p->ncells, ctx->stream));
  }
  UTIL(launch_finalize(p->bparts, p->nbparts, p->ctl, p->hist, p->hist_cap, p->status, FIN_BNORM, ctx->stream));
  return SIP_OK;
}

int end_sequence(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  if (p->mode == SIP_MODE_F32) UTIL(launch_cast_f32_f64(p->d32, p->x64, p->ncells, ctx->stream));
  for (auto &bh : p->blocks) UTIL(launch_from_plan_f64(p->x64, bh.d.x, bh.db, ctx->stream));
  CU(cudaMemcpyAsync(&p->h_ctl[2], p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = check_status(p);  // synchronises
  if (rc != SIP_OK) return rc;
  p->last_nhist = p->h_ctl[2].nhist;
  return SIP_OK;
}

// sweep kernels a plan of the given mode launches
std::vector<int> plan_kinds(int mode) {
  if (mode == SIP_MODE_F64) return {K_FACTOR, K_FWD64, K_BWD64};
  if (mode == SIP_MODE_F32) return {K_FACTOR32, K_FWD32, K_BWD32};
  return {K_FACTOR32, K_FWD32, K_BWD32, K_BWD32Z};
}

// Tile shape: rows per thread Q and warps NW (tile = 32 x Q*NW), stage depth
// R.  Shapes are ranked by the launch model of sip_shape.cu (the tile
// wavefront replayed with a fitted per-step cost that grows with the warps
// sharing an SM).  Automatic choices take one or two rows per thread (four
// measured 1.45x the step of two) with an even number of warps for one row
// (a balanced split over the four sub-partitions), up to 16 warps with one
// row and 12 with two (16 x 2 measured slower than modelled at 384^3); R = 3
// unless forced (deeper rings measured slower on GB300: 3 beat 4 by up to
// 11 %, 6 is slower still, and the start slack of a tile grows with R).
struct ShapeChoice {
  int Q = 0, NW = 0, ntiles = 0;
  int R[K_NKINDS] = {}, cap[K_NKINDS] = {};
  double score = 1e300;
};

std::vector<ShapeChoice> shape_candidates(sip_ctx *ctx, const std::vector<BlockHost> &blocks,
                                          const std::vector<int> &kinds, int tab_ints, int forceTK, int forceR,
                                          int forceQ, bool fp64) {
  std::vector<int> dims;
  for (auto &bh : blocks) dims.insert(dims.end(), {bh.d.nx, bh.d.ny, bh.d.nz});
  std::vector<ShapeChoice> all;
  for (int Q : kQs)
    for (int NW = 1; NW <= 16; ++NW) {
      const int TK = Q * NW, NT = 32 * NW;
      if (forceTK > 0 && TK != forceTK) continue;
      if (forceQ > 0 && Q != forceQ) continue;
      if (forceQ == 0 && forceTK == 0) {
        if (Q == 4) continue;
        if (Q == 1 && NW % 2) continue;
        if (Q == 2 && NW > 12) continue;
      }
      ShapeChoice c;
      c.Q = Q;
      c.NW = NW;
      int capmin = INT_MAX;
      bool ok = true;
      for (int kind : kinds) {
        const bool fac = kind == K_FACTOR || kind == K_FACTOR32;
        int bR = 0, bcap = 0;
        for (int R : {3, 4, 6, 2}) {
          // the one-off factorisation may drop to a 2-stage ring when its
          // 64-byte input records do not fit a wide tile
          if (R == 2 ? !fac : (forceR > 0 && R != forceR)) continue;
          if (R == 2 && bcap > 0) break;
          const size_t smem = kernel_smem(kind, Q, R, NT, tab_ints);
          if (smem + ctx->kernel_static_smem > ctx->smem_optin) continue;
          const int capk = ctx->nsm * max_active(kernel_ptr(kind, Q, R), NT, smem);
          if (capk > bcap) { bR = R; bcap = capk; }
          if (forceR == 0 && capk > 0 && R == 3) break;  // R = 3 when it fits
        }
        if (bcap < 1) { ok = false; break; }
        c.R[kind] = bR;
        c.cap[kind] = bcap;
        capmin = std::min(capmin, bcap);
      }
      if (!ok) continue;
      for (auto &bh : blocks) c.ntiles += ((bh.d.ny + kTJ - 1) / kTJ) * ((bh.d.nz + TK - 1) / TK);
      c.score = sweep_model_cycles(dims.data(), (int)blocks.size(), Q, NW, capmin, ctx->nsm, fp64);
      // deeper rings lengthen the start slack of every tile
      const int R = c.R[kinds[1]];
      if (R > 3) c.score *= 1.0 + 0.03 * (R - 3);
      all.push_back(c);
    }
  std::stable_sort(all.begin(), all.end(), [](const ShapeChoice &a, const ShapeChoice &b) { return a.score < b.score; });
  return all;
}

ShapeChoice choose_shape(sip_ctx *ctx, const std::vector<BlockHost> &blocks, const std::vector<int> &kinds,
                         int tab_ints, int forceTK, int forceR, int forceQ, bool fp64) {
  const std::vector<ShapeChoice> c = shape_candidates(ctx, blocks, kinds, tab_ints, forceTK, forceR, forceQ, fp64);
  return c.empty() ? ShapeChoice() : c.front();
}

// ------------------------------------------------------------ autotuner
// sip_options.autotune: the cost model's best few shapes are built as plans
// and their forward + backward sweeps timed on the plan's own buffers; the
// fastest plan is kept.  With SIP_AUTOTUNE_CACHE naming a file, results are
// read from and appended to it, one line per problem signature:
//   <signature> <rows_per_thread> <tile_k> <stages> <ms per sweep pair>
constexpr int kTuneCandidates = 4;
constexpr int kTuneReps = 3;
std::mutex g_tune_mu;

std::string tune_signature(const sip_ctx *ctx, const sip_block_desc *blocks, int nblocks, const sip_options &o) {
  std::string dims;
  for (int b = 0; b < nblocks; ++b)
    dims += std::to_string(blocks[b].nx) + "x" + std::to_string(blocks[b].ny) + "x" + std::to_string(blocks[b].nz) + ",";
  if (nblocks > 4) {  // long lists: FNV-1a of the dims
    unsigned long long h = 1469598103934665603ull;
    for (unsigned char ch : dims) h = (h ^ ch) * 1099511628211ull;
    char buf[32];
    std::snprintf(buf, sizeof(buf), "h%016llx", h);
    dims = buf;
  }
  return "sm" + std::to_string(ctx->nsm) + "/m" + std::to_string(o.mode) + "/s" + std::to_string(blocks[0].symmetric) +
         "/c" + std::to_string(blocks[0].coef_dtype) + "/b" + std::to_string(nblocks) + "/" + dims;
}

bool tune_lookup(const std::string &sig, int &Q, int &TK, int &R) {
  const char *path = getenv("SIP_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[4096];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {  // the last entry of a signature wins
    char key[4096];
    int q = 0, tk = 0, r = 0;
    double ms = 0;
    if (line[0] == '#' || sscanf(line, "%4095s %d %d %d %lf", key, &q, &tk, &r, &ms) < 4) continue;
    if (sig == key) {
      Q = q;
      TK = tk;
      R = r;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_store(const std::string &sig, int Q, int TK, int R, double ms) {
  const char *path = getenv("SIP_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %.4f\n", sig.c_str(), Q, TK, R, ms);
  fclose(f);
}

// ms per forward + backward sweep pair of a built plan, on its own work
// vectors (zeroed first; the caller's x is not touched).
double time_sweeps(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  cudaStream_t st = ctx->stream;
  const bool f64 = p->mode == SIP_MODE_F64;
  if (f64) {
    if (cudaMemsetAsync(p->y64, 0, (size_t)p->ncells * 8, st) != cudaSuccess) return -1;
  } else if (cudaMemsetAsync(p->y32, 0, (size_t)p->ncells * 4, st) != cudaSuccess ||
             cudaMemsetAsync(p->d32, 0, (size_t)p->ncells * 4, st) != cudaSuccess) {
    return -1;
  }
  if (cudaMemsetAsync(p->x64, 0, (size_t)p->ncells * 8, st) != cudaSuccess) return -1;
  if (cudaMemsetAsync(p->tickets, 0, 4 * sizeof(int), st) != cudaSuccess) return -1;
  if (launch_set_ctl(p->ctl, -1.0, 0, st) != cudaSuccess) return -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double ms = -1;
  bool ok = true;
  for (int r = 0; r <= kTuneReps && ok; ++r) {  // the first pair warms up
    if (r == 1) cudaEventRecord(e0, st);
    if (f64) {
      ok = enqueue_forward(p, K_FWD64, (const double *)p->y64, p->y64) == SIP_OK &&
           enqueue_backward(p, K_BWD64, (const double *)p->y64, p->x64) == SIP_OK;
    } else {
      ok = enqueue_forward(p, K_FWD32, (const float *)p->y32, p->y32) == SIP_OK &&
           enqueue_backward(p, K_BWD32, (const float *)p->y32, p->d32) == SIP_OK;
    }
  }
  cudaEventRecord(e1, st);
  float t = 0.f;
  if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
    ms = t / kTuneReps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (check_status(p) != SIP_OK) ms = -1;
  return ms;
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

void sip_default_options(sip_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->alpha = 0.92;
  opt->mode = SIP_MODE_F64;
  opt->inner_iters = 4;
  opt->max_spin = 0;
}

int sip_create(sip_ctx **out, int device, void *stream) {
  if (!out) return SIP_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    g_create_error = "no CUDA device";
    return SIP_ERR_NO_DEVICE;
  }
  if (device < 0 || device >= ndev) return SIP_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return SIP_ERR_NO_DEVICE;
  sip_ctx *ctx = new sip_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return SIP_ERR_NO_DEVICE;
  }
  ctx->nsm = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  {
    // the context's stream-ordered pool (falls back to cudaMalloc if the
    // device or the CUDA driver has none); keeps at least kPoolKeep bytes, and the
    // largest plan footprint reached, cached between plans instead of
    // returning them at every synchronisation
    int pools = 0;
    cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, device);
    if (pools) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      if (cudaMemPoolCreate(&ctx->mempool, &props) == cudaSuccess) {
        unsigned long long keep = kPoolKeep;
        cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
        ctx->pool_keep = keep;
      } else {
        ctx->mempool = nullptr;
        cudaGetLastError();
      }
    }
  }
  for (int kind = 0; kind < K_NKINDS; ++kind)
    for (int Q : {1, 2, 4})  // Q = 1: the factorisation's own decomposition
      for (int R : kRs) {
        const void *f = kernel_ptr(kind, Q, R);
        if (!f) continue;
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(ctx->smem_optin - fa.sharedSizeBytes));
        if (e != cudaSuccess) {
          g_create_error = std::string("kernel attribute setup: ") + cudaGetErrorString(e);
          if (ctx->mempool) cudaMemPoolDestroy(ctx->mempool);
          delete ctx;
          return SIP_ERR_CUDA;
        }
        ctx->kernel_static_smem = std::max(ctx->kernel_static_smem, (size_t)fa.sharedSizeBytes);
      }
  *out = ctx;
  return SIP_OK;
}

int sip_destroy(sip_ctx *ctx) {
  if (!ctx) return SIP_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (void *v : ctx->pinned) cudaFreeHost(v);
  if (ctx->mempool) cudaMemPoolDestroy(ctx->mempool);
  delete ctx;
  return SIP_OK;
}

int sip_trim(sip_ctx *ctx) {
  if (!ctx) return SIP_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess && ctx->mempool) {
    unsigned long long keep = kPoolKeep, zero = 0;
    e = cudaMemPoolTrimTo(ctx->mempool, 0);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) ctx->pool_keep = keep;
    // restart the peak from what live plans hold, so the next plan creation
    // raises the cache limit to its own peak only (best effort: without the
    // reset the limit returns to the earlier peak)
    if (e == cudaSuccess && cudaMemPoolSetAttribute(ctx->mempool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess)
      cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(ctx, SIP_ERR_CUDA, std::string("trim: ") + cudaGetErrorString(e));
  return SIP_OK;
}

const char *sip_last_error(sip_ctx *ctx) {
  static thread_local std::string copy;
  copy = ctx ? ctx->err : g_create_error;
  return copy.c_str();
}

int sip_factor(sip_ctx *ctx, const sip_block_desc *blocks, int nblocks, const sip_interface *ifaces,
               int nifaces, const sip_options *opt_in, sip_plan **out) {
  if (!ctx || !out) return SIP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!blocks || nblocks < 1) return fail(ctx, SIP_ERR_INVALID_ARG, "need at least one block");
  if (nifaces < 0 || (nifaces > 0 && !ifaces)) return fail(ctx, SIP_ERR_INVALID_ARG, "bad interface list");
  sip_options opt;
  if (opt_in) opt = *opt_in;
  else sip_default_options(&opt);
  if (!(opt.alpha >= 0.0 && opt.alpha <= 1.0)) return fail(ctx, SIP_ERR_INVALID_ARG, "alpha must lie in [0, 1]");
  if (opt.mode != SIP_MODE_F64 && opt.mode != SIP_MODE_F32_REFINED && opt.mode != SIP_MODE_F32)
    return fail(ctx, SIP_ERR_INVALID_ARG, "unsupported mode");
  if (opt.mode == SIP_MODE_F32_REFINED && opt.inner_iters < 1)
    return fail(ctx, SIP_ERR_INVALID_ARG, "inner_iters must be >= 1");
  const bool sym = blocks[0].symmetric != 0;
  long long ncells = 0;
  for (int b = 0; b < nblocks; ++b) {
    const sip_block_desc &d = blocks[b];
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(ctx, SIP_ERR_INVALID_ARG, "block dims must be >= 1");
    const long long n = (long long)d.nx * d.ny * d.nz;
    if (n >= (1ll << 31) || (long long)d.nx + d.ny + d.nz > (1 << 20))
      return fail(ctx, SIP_ERR_INVALID_ARG, "block too large (nx*ny*nz must be < 2^31)");
    if (d.coef_dtype != 0 && d.coef_dtype != 1) return fail(ctx, SIP_ERR_INVALID_ARG, "coef_dtype must be 0 or 1");
    if (!d.ap || !d.ae || !d.an || !d.at || !d.b || !d.x)
      return fail(ctx, SIP_ERR_INVALID_ARG, "null coefficient, rhs or solution pointer");
    if ((d.symmetric != 0) != sym) return fail(ctx, SIP_ERR_INVALID_ARG, "all blocks of a plan must share `symmetric`");
    if (!sym && (!d.aw || !d.as || !d.ab))
      return fail(ctx, SIP_ERR_INVALID_ARG, "aw/as/ab may be NULL only for symmetric blocks");
    if (d.coef_dtype != blocks[0].coef_dtype)
      return fail(ctx, SIP_ERR_INVALID_ARG, "all blocks of a plan must share coef_dtype");
    ncells += n;
  }
  if (ncells >= (1ll << 31)) return fail(ctx, SIP_ERR_INVALID_ARG, "plan too large (total cells must be < 2^31)");
  {
    std::vector<int> east(nblocks, 0), west(nblocks, 0);
    for (int q = 0; q < nifaces; ++q) {
      const sip_interface &f = ifaces[q];
      const std::string tag = "interface " + std::to_string(q) + ": ";
      if (f.blk_lo < 0 || f.blk_lo >= nblocks || f.blk_hi < 0 || f.blk_hi >= nblocks || f.blk_lo == f.blk_hi)
        return fail(ctx, SIP_ERR_INVALID_ARG, tag + "block indices out of range or equal");
      const sip_block_desc &L = blocks[f.blk_lo], &H = blocks[f.blk_hi];
      if (f.nj < 1 || f.nk < 1 || f.nj > std::min(L.ny, H.ny) || f.nk > std::min(L.nz, H.nz))
        return fail(ctx, SIP_ERR_INVALID_ARG, tag + "overlap rectangle must lie inside both x faces");
      if (east[f.blk_lo]++ || west[f.blk_hi]++)
        return fail(ctx, SIP_ERR_INVALID_ARG, tag + "a block face carries at most one interface");
    }
  }
  if (opt.tile_j != 0 && opt.tile_j != kTJ) return fail(ctx, SIP_ERR_INVALID_ARG, "tile_j must be 0 or 32");
  if (opt.tile_k < 0 || opt.tile_k > 64 || (opt.tile_k > 0 && opt.tile_k % 2 != 0))
    return fail(ctx, SIP_ERR_INVALID_ARG, "tile_k must be 0 (auto) or an even number <= 64");
  if (opt.stages != 0 && opt.stages != 3 && opt.stages != 4 && opt.stages != 6)
    return fail(ctx, SIP_ERR_INVALID_ARG, "stages must be 0 (auto), 3, 4 or 6");
  if (opt.rows_per_thread != 0 && opt.rows_per_thread != 1 && opt.rows_per_thread != 2 && opt.rows_per_thread != 4)
    return fail(ctx, SIP_ERR_INVALID_ARG, "rows_per_thread must be 0 (auto), 1, 2 or 4");
  if (opt.autotune != 0 && opt.autotune != 1) return fail(ctx, SIP_ERR_INVALID_ARG, "autotune must be 0 or 1");
  if (opt.autotune && opt.tile_k == 0 && opt.rows_per_thread == 0 && opt.stages == 0) {
    const std::string sig = tune_signature(ctx, blocks, nblocks, opt);
    sip_options o = opt;
    o.autotune = 0;
    o.tile_j = kTJ;
    if (tune_lookup(sig, o.rows_per_thread, o.tile_k, o.stages)) {
      const int rc = sip_factor(ctx, blocks, nblocks, ifaces, nifaces, &o, out);
      if (rc == SIP_OK) return rc;  // a stale entry (another build's shapes) falls through to tuning
    }
    // candidates from the cost model
    std::vector<BlockHost> bh(nblocks);
    int tab_ints = 0;
    for (int b = 0; b < nblocks; ++b) {
      bh[b].d = blocks[b];
      tab_ints = std::max(tab_ints, (blocks[b].nx + blocks[b].ny + blocks[b].nz - 2) + (blocks[b].nx + blocks[b].ny - 1));
    }
    const std::vector<ShapeChoice> cand =
        shape_candidates(ctx, bh, plan_kinds(opt.mode), tab_ints, 0, 0, 0, opt.mode == SIP_MODE_F64);
    sip_plan *best = nullptr;
    double best_ms = 0;
    int tried = 0, last_rc = SIP_OK;  // candidates built and timed
    for (const ShapeChoice &c : cand) {
      if (tried == kTuneCandidates) break;
      o.rows_per_thread = c.Q;
      o.tile_k = c.Q * c.NW;
      o.stages = c.R[plan_kinds(opt.mode)[1]];
      sip_plan *tp = nullptr;
      last_rc = sip_factor(ctx, blocks, nblocks, ifaces, nifaces, &o, &tp);
      if (last_rc != SIP_OK) {
        if (best) break;  // e.g. no room for a second plan next to the best one: keep the best
        return last_rc;   // breakdown or invalid input: no shape changes that
      }
      ++tried;
      const double ms = time_sweeps(tp);
      if (ms > 0 && (!best || ms < best_ms)) {
        if (best) sip_plan_destroy(best);
        best = tp;
        best_ms = ms;
      } else {
        sip_plan_destroy(tp);
      }
    }
    if (!best) return fail(ctx, SIP_ERR_CUDA, "autotune: no candidate shape could be timed");
    tune_store(sig, best->Q, best->TK, best->Rk[plan_kinds(opt.mode)[1]], best_ms);
    best->opt.autotune = 1;
    *out = best;
    return SIP_OK;
  }

  sip_plan *p = new sip_plan();
  p->ctx = ctx;
  p->opt = opt;
  p->mode = opt.mode;
  p->sym = sym;
  p->a32in = blocks[0].coef_dtype == 1;
  p->ncells = ncells;
  p->blocks.resize(nblocks);
  p->ifaces.assign(ifaces, ifaces + nifaces);
  for (int b = 0; b < nblocks; ++b) {
    BlockHost &bh = p->blocks[b];
    bh.d = blocks[b];
    build_tables(bh.d.nx, bh.d.ny, bh.d.nz, bh.PO, bh.F);
    bh.n = (long long)bh.d.nx * bh.d.ny * bh.d.nz;
    p->tab_ints = std::max(p->tab_ints, (int)(bh.PO.size() + bh.F.size()));
  }
  const std::vector<int> kinds = plan_kinds(p->mode);
  const ShapeChoice sc = choose_shape(ctx, p->blocks, kinds, p->tab_ints, opt.tile_k, opt.stages, opt.rows_per_thread,
                                      p->mode == SIP_MODE_F64);
  if (sc.Q == 0) {
    delete p;
    return fail(ctx, SIP_ERR_INVALID_ARG, "no tile shape fits on an SM");
  }
  p->Q = sc.Q;
  p->NW = sc.NW;
  p->NT = 32 * sc.NW;
  p->TK = sc.Q * sc.NW;
  for (int k : kinds) {
    p->Rk[k] = sc.R[k];
    p->gridk[k] = sc.cap[k];
  }

  // per-block layout and tiles; claim order: anti-diagonal waves (cj + ck), blocks interleaved
  std::vector<DevBlock> hdb;
  std::vector<Tile> tiles;
  long long cell0 = 0, face0 = 0;
  size_t tab_total = 0;
  for (int b = 0; b < nblocks; ++b) {
    BlockHost &bh = p->blocks[b];
    DevBlock &db = bh.db;
    db.nx = bh.d.nx; db.ny = bh.d.ny; db.nz = bh.d.nz;
    db.nplanes = db.nx + db.ny + db.nz - 2;
    db.TK = p->TK;
    db.nTJ = (db.ny + kTJ - 1) / kTJ;
    db.nTK = (db.nz + p->TK - 1) / p->TK;
    db.mmax = db.nx + db.ny - 2;
    db.tile0 = p->ntiles;
    db.nsteps_max = db.nx + kTJ + p->TK - 2;
    db.cell0 = cell0;
    db.PO = db.F = nullptr;
    db.face0 = face0;
    db.face_tile_words = (long long)db.nsteps_max * (kTJ + p->TK) * kFaceWordsMax;
    db.lo_blk = db.hi_blk = -1;
    db.lo_nj = db.lo_nk = db.hi_nj = db.hi_nk = 0;
    db.row0 = p->nrows;
    p->nrows += (long long)db.nz * (db.nx + db.ny - 1);
    const int nt = db.nTJ * db.nTK;
    p->ntiles += nt;
    face0 += (long long)nt * db.face_tile_words;
    cell0 += bh.n;
    tab_total += bh.PO.size() + bh.F.size();
  }
  {
    int maxwave = 0;
    for (auto &bh : p->blocks) maxwave = std::max(maxwave, bh.db.nTJ + bh.db.nTK - 2);
    for (int w = 0; w <= maxwave; ++w)
      for (int b = 0; b < nblocks; ++b) {
        const DevBlock &db = p->blocks[b].db;
        for (int ck = 0; ck < db.nTK; ++ck) {
          const int cj = w - ck;
          if (cj < 0 || cj >= db.nTJ) continue;
          tiles.push_back(Tile{b, cj, ck, db.tile0 + ck * db.nTJ + cj});
        }
      }
  }
  std::vector<Tile> tiles_b(tiles.rbegin(), tiles.rend());
  // The factorisation's own decomposition: 32 x kFacTK tiles, one row per
  // warp.  Its steps are bound by the FP64 pipe of the SM sub-partitions (one
  // warp instruction per 64 cycles each), so a step costs in proportion to
  // the rows a sub-partition holds; one row per warp and 4 warps per tile
  // keep that at one row and shorten the wavefront's chain, while several
  // tiles share an SM where the wavefront is wide.
  constexpr int kFacTK = 4;
  std::vector<DevBlock> fdb;
  std::vector<Tile> ftiles;
  int fntiles = 0;
  long long fface0 = 0;
  for (int b = 0; b < nblocks; ++b) {
    DevBlock d = p->blocks[b].db;
    d.TK = kFacTK;
    d.nTK = (d.nz + kFacTK - 1) / kFacTK;
    d.tile0 = fntiles;
    d.nsteps_max = d.nx + kTJ + kFacTK - 2;
    d.face0 = fface0;
    d.face_tile_words = (long long)d.nsteps_max * (kTJ + kFacTK) * kFaceWordsMax;
    const int nt = d.nTJ * d.nTK;
    fntiles += nt;
    fface0 += (long long)nt * d.face_tile_words;
    fdb.push_back(d);
  }
  {
    int maxwave = 0;
    for (const DevBlock &d : fdb) maxwave = std::max(maxwave, d.nTJ + d.nTK - 2);
    for (int w = 0; w <= maxwave; ++w)
      for (int b = 0; b < nblocks; ++b) {
        const DevBlock &d = fdb[b];
        for (int ck = 0; ck < d.nTK; ++ck) {
          const int cj = w - ck;
          if (cj < 0 || cj >= d.nTJ) continue;
          ftiles.push_back(Tile{b, cj, ck, d.tile0 + ck * d.nTJ + cj});
        }
      }
  }
  const long long face_words = std::max(face0, fface0);

  auto bail = [&](cudaError_t e, const char *what) {
    free_plan_memory(p);
    delete p;
    return fail(ctx, e == cudaErrorMemoryAllocation ? SIP_ERR_OOM : SIP_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
#define PA(ptr, count)                                   \
  do {                                                   \
    cudaError_t e_ = palloc(p, &(ptr), (size_t)(count)); \
    if (e_ != cudaSuccess) return bail(e_, #ptr);        \
  } while (0)
  const long long N = ncells;
  const bool f64 = p->mode == SIP_MODE_F64;
  {
    // row-parallel launches: every SM filled with the plan's most demanding
    // residual variant, no more CTAs than 8-row groups
    int occ = 0;
    if (f64) {
      occ = resrow_max_active<double, double, double>(sym, true);
    } else {
      occ = resrow_max_active<float, float, float>(sym, p->mode == SIP_MODE_F32);
      if (p->mode == SIP_MODE_F32_REFINED)
        occ = std::min(occ, p->a32in ? resrow_max_active<float, double, float>(sym, true)
                                     : resrow_max_active<double, double, float>(sym, true));
    }
    const int wpc = row_threads() / 32;
    const long long groups = (p->nrows + wpc - 1) / wpc;
    p->rowgrid = (int)std::max(1ll, std::min<long long>((long long)ctx->nsm * std::max(occ, 1), groups));
  }
  PA(p->d_tab, tab_total);
  PA(p->d_blocks, nblocks);
  PA(p->d_tiles_f, p->ntiles);
  PA(p->d_tiles_b, p->ntiles);
  PA(p->faces, face_words);
  DevBlock *d_fblocks = nullptr;
  Tile *d_ftiles = nullptr;
  PA(d_fblocks, nblocks);
  PA(d_ftiles, fntiles);
  PA(p->partials, p->rowgrid);
  PA(p->bparts, p->nbparts);
  PA(p->ctl, 1);
  p->hist_cap = 1 << 20;
  PA(p->hist, p->hist_cap);
  PA(p->status, 1);
  PA(p->tickets, 4);
  if (const char *tp = getenv("SIP_TRACE")) {
    p->trace_path = tp;
    PA(p->trace, (size_t)K_NKINDS * p->ntiles * kTraceWords);
    cudaMemsetAsync(p->trace, 0, (size_t)K_NKINDS * p->ntiles * kTraceWords * 8, ctx->stream);
  }
  PA(p->b64, N);
  PA(p->x64, N);
  double *a7 = nullptr;
  PA(a7, N * 8);
  const int na = a_rec_values(sym);
  if (f64) {
    double *rf = nullptr, *rb = nullptr, *ra = nullptr;
    PA(rf, N * 4);
    PA(rb, N * 4);
    PA(ra, N * na);
    p->recF = rf;
    p->recB = rb;
    p->recA = ra;
    PA(p->y64, N);
  } else {
    float *rf = nullptr, *rb = nullptr, *ra = nullptr;
    PA(rf, N * 4);
    PA(rb, N * 4);
    PA(ra, N * na);
    p->recF = rf;
    p->recB = rb;
    p->recA = ra;
    PA(p->r32, N);
    PA(p->d32, N);
    PA(p->y32, N);
    if (!p->a32in && p->mode == SIP_MODE_F32_REFINED) PA(p->arec64, N * na);
  }
  pool_keep_peak(ctx);
  {
    static_assert(3 * sizeof(Ctl) + 2 * sizeof(int) <= kPinnedBlock, "pinned control block");
    void *blk = pinned_take(ctx);
    if (!blk) return bail(cudaErrorMemoryAllocation, "pinned control block");
    p->h_ctl = static_cast<Ctl *>(blk);
    p->h_status = reinterpret_cast<int *>(static_cast<unsigned char *>(blk) + 3 * sizeof(Ctl));
  }
  cudaStream_t st = ctx->stream;
  std::vector<HaloEntry> hents;
  std::vector<HaloSrc> hsrcs;
  if (nifaces > 0) {
    // one entry per interface face cell, couplings in interface order (lo side first)
    std::vector<int> at_cell;  // entry of a plan cell, -1 if none
    at_cell.assign((size_t)ncells, -1);
    auto cell_of = [&](int b, int i, int j, int k) {
      const BlockHost &bh = p->blocks[b];
      return p->blocks[b].db.cell0 +
             plane_row_base(bh.PO.data(), bh.F.data(), bh.d.nx + bh.d.ny - 2, bh.d.nx, i + j + k, k) + j;
    };
    auto add = [&](long long cell, long long nb, const void *src, long long pn) {
      int &e = at_cell[(size_t)cell];
      if (e < 0) {
        e = (int)hents.size();
        hents.push_back(HaloEntry{cell, {-1, -1}, {0.0, 0.0}});
      }
      const int slot = hents[e].nb[0] < 0 ? 0 : 1;
      hents[e].nb[slot] = nb;
      hsrcs.push_back(HaloSrc{e, slot, src, pn});
    };
    for (const sip_interface &f : p->ifaces) {
      const sip_block_desc &L = blocks[f.blk_lo], &H = blocks[f.blk_hi];
      for (int k = 0; k < f.nk; ++k)
        for (int j = 0; j < f.nj; ++j) {
          const long long cl = cell_of(f.blk_lo, L.nx - 1, j, k), ch = cell_of(f.blk_hi, 0, j, k);
          const long long pl = (long long)(L.nx - 1) + (long long)L.nx * (j + (long long)L.ny * k);
          const long long ph = (long long)H.nx * (j + (long long)H.ny * k);
          add(cl, ch, L.ae, pl);
          if (sym) add(ch, cl, L.ae, pl);  // symmetric: the entry of hi equals lo's AE
          else add(ch, cl, H.aw, ph);
        }
    }
    p->nhalo = (int)hents.size();
    HaloSrc *dsrc = nullptr;
    PA(p->beff64, N);
    PA(p->halo, p->nhalo);
    PA(p->hsave32, p->nhalo);
    PA(dsrc, hsrcs.size());
    cudaError_t e = cudaMemcpyAsync(p->halo, hents.data(), hents.size() * sizeof(HaloEntry),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dsrc, hsrcs.data(), hsrcs.size() * sizeof(HaloSrc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_halo_coefs(dsrc, (int)hsrcs.size(), p->halo, p->a32in ? 1 : 0, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pfree(p, dsrc, hsrcs.size() * sizeof(HaloSrc));
    if (e != cudaSuccess) return bail(e, "interfaces");
  }
  {
    std::vector<int> tab;
    tab.reserve(tab_total);
    for (auto &bh : p->blocks) {
      bh.db.PO = p->d_tab + tab.size();
      tab.insert(tab.end(), bh.PO.begin(), bh.PO.end());
      bh.db.F = p->d_tab + tab.size();
      tab.insert(tab.end(), bh.F.begin(), bh.F.end());
      hdb.push_back(bh.db);
    }
    for (int b = 0; b < nblocks; ++b) {
      fdb[b].PO = p->blocks[b].db.PO;
      fdb[b].F = p->blocks[b].db.F;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_tab, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_blocks, hdb.data(), hdb.size() * sizeof(DevBlock), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_tiles_f, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_tiles_b, tiles_b.data(), tiles_b.size() * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_fblocks, fdb.data(), fdb.size() * sizeof(DevBlock), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_ftiles, ftiles.data(), ftiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->faces, 0, (size_t)face_words * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->tickets, 0, 4 * sizeof(int), st);
    const size_t es = f64 ? 8 : 4;
    if (e == cudaSuccess) e = cudaMemsetAsync(p->recF, 0, (size_t)N * 4 * es, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->recB, 0, (size_t)N * 4 * es, st);
    // host vectors must outlive the async copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(e, "plan upload");
  }
  // A into the plan: the factorisation input (all seven entries, FP64), the
  // A records of the residual in the sweep precision and, in the refined
  // mode with FP64 coefficients, the FP64 A of the outer residual (one pass
  // per block; coefficients that point out of their block are zeroed).
  for (auto &bh : p->blocks) {
    PackSrc ps;
    const void *src[7] = {bh.d.ap, bh.d.aw, bh.d.ae, bh.d.as, bh.d.an, bh.d.ab, bh.d.at};
    for (int q = 0; q < 7; ++q) ps.a[q] = src[q];
    ps.f32 = bh.d.coef_dtype;
    ps.sym = sym ? 1 : 0;
    cudaError_t e = launch_pack_records(ps, bh.db, a7, p->recA, f64 ? 0 : 1, p->arec64, st);
    if (e != cudaSuccess) return bail(e, "reorder A");
  }
  // Stone's factorisation (one wavefront sweep)
  {
    cudaError_t e = launch_set_ctl(p->ctl, -1.0, 0, st);
    if (e != cudaSuccess) return bail(e, "control");
    // on the factorisation's own decomposition (one row per warp, kFacTK rows per tile)
    auto run_factor = [&](int kind, auto &fp) -> cudaError_t {
      fp.c = common(p, false, 2, 0, 0, kind);
      fp.c.blocks = d_fblocks;
      fp.c.tiles = d_ftiles;
      fp.c.ntiles = fntiles;
      fp.c.trace = nullptr;  // the trace buffer is sized for the sweeps' tiles
      const int NTf = 32 * kFacTK;
      int Rf = 3;
      size_t smem = kernel_smem(kind, 1, Rf, NTf, p->tab_ints);
      if (smem + ctx->kernel_static_smem > ctx->smem_optin) {
        Rf = 2;
        smem = kernel_smem(kind, 1, Rf, NTf, p->tab_ints);
      }
      const void *f = kernel_ptr(kind, 1, Rf);
      const int cap = ctx->nsm * max_active(f, NTf, smem);
      if (!f || cap < 1) return cudaErrorInvalidConfiguration;
      const int grid = std::max(1, std::min(fntiles, cap));
      void *args[] = {(void *)&fp};
      ProfScope ps(p, kind);
      return cudaLaunchKernel(f, dim3(grid), dim3(NTf), args, smem, st);
    };
    if (f64) {
      FacParams<double> fp;
      fp.a7 = a7;
      fp.recF = (double *)p->recF;
      fp.recB = (double *)p->recB;
      fp.alpha = opt.alpha;
      e = run_factor(K_FACTOR, fp);
    } else {
      FacParams<float> fp;
      fp.a7 = a7;
      fp.recF = (float *)p->recF;
      fp.recB = (float *)p->recB;
      fp.alpha = opt.alpha;
      e = run_factor(K_FACTOR32, fp);
    }
    if (e != cudaSuccess) return bail(e, "factor launch");
    int rc = check_status(p);
    if (rc != SIP_OK) {
      std::string msg = ctx->err;
      free_plan_memory(p);
      delete p;
      return fail(ctx, rc, msg);
    }
    pfree(p, a7, (size_t)N * 8 * sizeof(double));
    pfree(p, d_ftiles, (size_t)std::max(fntiles, 1) * sizeof(Tile));
    pfree(p, d_fblocks, (size_t)nblocks * sizeof(DevBlock));
  }
  *out = p;
  return SIP_OK;
}

int sip_iterate(sip_plan *p, int niters, double *relres_out) {
  if (!p) return SIP_ERR_INVALID_ARG;
  sip_ctx *ctx = p->ctx;
  if (niters < 0) return fail(ctx, SIP_ERR_INVALID_ARG, "niters must be >= 0");
  int rc = begin_sequence(p, -1.0, niters);
  if (rc) return rc;
  rc = enqueue_iters(p, niters);
  if (rc) return rc;
  rc = end_sequence(p);
  if (rc) return rc;
  if (relres_out) *relres_out = p->h_ctl[2].relres;
  return SIP_OK;
}

int sip_solve(sip_plan *p, double rtol, int max_iters, int *iters_out, double *relres_out) {
  if (!p) return SIP_ERR_INVALID_ARG;
  sip_ctx *ctx = p->ctx;
  if (max_iters < 0 || !(rtol >= 0.0)) return fail(ctx, SIP_ERR_INVALID_ARG, "bad rtol or max_iters");
  int rc = begin_sequence(p, rtol, max_iters);
  if (rc) return rc;
  // Chunks of iterations; the stop rule runs on the device (kernels after the
  // deciding residual do nothing).  The host reads the control block once per
  // chunk, one chunk behind, so the next chunk is always queued.
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // every exit after this point destroys the events and closes the sequence
  // (x copied back, status checked); the first error is the one reported
  auto finish = [&](int first_rc) {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    const int end_rc = end_sequence(p);
    return first_rc != SIP_OK ? first_rc : end_rc;
  };
  auto cuda_fail = [&](cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? SIP_ERR_OOM : SIP_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  if (e != cudaSuccess) return finish(cuda_fail(e, "event create"));
  const int chunk = kChunk;
  int issued = 0;      // iterations queued (each starts with one residual + stop check)
  int nq = 0, nc = 0;  // chunks queued / checked
  bool more = true;
  for (;;) {
    if (more) {
      const int n = std::min(chunk, max_iters + 1 - issued);
      rc = enqueue_iters(p, n);
      if (rc) return finish(rc);
      issued += n;
      const int sl = nq & 1;
      e = cudaMemcpyAsync(&p->h_ctl[sl], p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&p->h_status[sl], p->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaEventRecord(ev[sl], ctx->stream);
      if (e != cudaSuccess) return finish(cuda_fail(e, "control block read"));
      ++nq;
      more = issued < max_iters + 1;
    }
    if (nq - nc >= 2 || (!more && nc < nq)) {
      const int sl = nc & 1;
      e = cudaEventSynchronize(ev[sl]);
      if (e != cudaSuccess) return finish(cuda_fail(e, "event wait"));
      ++nc;
      if (p->h_ctl[sl].done || p->h_status[sl] != DEV_OK) break;
      if (!more && nc == nq) break;
    }
  }
  rc = finish(SIP_OK);
  if (rc) return rc;
  const Ctl *hc = &p->h_ctl[2];
  if (iters_out) *iters_out = hc->iter;
  if (relres_out) *relres_out = hc->relres;
  return hc->relres <= rtol ? SIP_OK : SIP_NOT_CONVERGED;
}

int sip_get_history(sip_plan *p, double *host_out, int cap, int *n_out) {
  if (!p) return SIP_ERR_INVALID_ARG;
  sip_ctx *ctx = p->ctx;
  const int n = std::min(p->last_nhist, p->hist_cap);
  if (n_out) *n_out = n;
  if (host_out && cap > 0 && n > 0) {
    CU(cudaMemcpyAsync(host_out, p->hist, sizeof(double) * std::min(n, cap), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  return SIP_OK;
}

int sip_export_factors(sip_plan *p, int blk, double *const out[7]) {
  if (!p || !out || blk < 0 || blk >= (int)p->blocks.size()) return SIP_ERR_INVALID_ARG;
  sip_ctx *ctx = p->ctx;
  for (int q = 0; q < 7; ++q)
    if (!out[q]) return fail(ctx, SIP_ERR_INVALID_ARG, "null output");
  CU(launch_export_factors(p->recF, p->recB, p->mode == SIP_MODE_F64 ? 0 : 1, out, p->blocks[blk].db,
                           ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return SIP_OK;
}

int sip_plane_layout(int nx, int ny, int nz, int32_t *rbT) {
  if (nx < 1 || ny < 1 || nz < 1 || !rbT || (long long)nx * ny * nz >= (1ll << 31)) return SIP_ERR_INVALID_ARG;
  std::vector<int> PO, F;
  build_tables(nx, ny, nz, PO, F);
  const int np = nx + ny + nz - 2, mmax = nx + ny - 2;
  for (int k = 0; k < nz; ++k)
    for (int s = 0; s < np; ++s) {
      const int m = s - k;
      const bool row = m >= 0 && m <= mmax && std::max(0, m - (nx - 1)) <= std::min(ny - 1, m);
      rbT[(size_t)k * np + s] = row ? plane_row_base(PO.data(), F.data(), mmax, nx, s, k) : INT32_MIN;
    }
  return SIP_OK;
}

int sip_tile_model(const int32_t *dims, int nblocks, int rows_per_thread, int warps, int ctas, int nsm, int fp64,
                   double *cycles_out) {
  if (!dims || !cycles_out || nblocks < 1 || warps < 1 || warps > 16 || ctas < 1 || nsm < 1) return SIP_ERR_INVALID_ARG;
  if (rows_per_thread != 1 && rows_per_thread != 2 && rows_per_thread != 4) return SIP_ERR_INVALID_ARG;
  const double c = sweep_model_cycles(dims, nblocks, rows_per_thread, warps, ctas, nsm, fp64 != 0);
  if (c < 0) return SIP_ERR_INVALID_ARG;
  *cycles_out = c;
  return SIP_OK;
}

// Natural-layout view of a block descriptor for the residual norm; "" or the
// reason the descriptor is unusable.
static std::string natblock_from_desc(const sip_block_desc *d, NatBlock *nb) {
  if (!d) return "null block descriptor";
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return "block dims must be >= 1";
  if ((long long)d->nx * d->ny * d->nz >= (1ll << 31)) return "block too large (nx*ny*nz must be < 2^31)";
  if (d->coef_dtype != 0 && d->coef_dtype != 1) return "coef_dtype must be 0 or 1";
  if (!d->ap || !d->ae || !d->an || !d->at || !d->b || !d->x) return "null coefficient, rhs or solution pointer";
  if (!d->symmetric && (!d->aw || !d->as || !d->ab)) return "aw/as/ab may be NULL only for symmetric blocks";
  nb->nx = d->nx;
  nb->ny = d->ny;
  nb->nz = d->nz;
  nb->coef_f32 = d->coef_dtype;
  nb->symmetric = d->symmetric != 0;
  const void *a[7] = {d->ap, d->aw, d->ae, d->as, d->an, d->ab, d->at};
  for (int q = 0; q < 7; ++q) nb->a[q] = a[q];
  nb->b = d->b;
  nb->x = d->x;
  return "";
}

int sip_assemble_pcorr(sip_ctx *ctx, const sip_pcorr_desc *in, double *ap, double *aw, double *ae, double *as,
                       double *an, double *ab, double *at, double *b) {
  if (!ctx) return SIP_ERR_INVALID_ARG;
  if (!in) return fail(ctx, SIP_ERR_INVALID_ARG, "null descriptor");
  if (in->nx < 1 || in->ny < 1 || in->nz < 1) return fail(ctx, SIP_ERR_INVALID_ARG, "block dimensions must be >= 1");
  // the largest face array ((nx + 1) ny nz and the like) indexes with 64-bit integers;
  // a block must fit the 2^31 - 1 cells of the solver's descriptors
  if ((long long)in->nx * in->ny * in->nz > 2147483647LL)
    return fail(ctx, SIP_ERR_INVALID_ARG, "block larger than 2^31 - 1 cells");
  if (!in->dx || !in->dy || !in->dz || !in->rho || !in->g || !in->ux || !in->uy || !in->uz)
    return fail(ctx, SIP_ERR_INVALID_ARG, "null input array");
  if (!ap || !ae || !an || !at || !b) return fail(ctx, SIP_ERR_INVALID_ARG, "null output array");
  CU(cudaSetDevice(ctx->device));
  PcorrArgs a;
  a.nx = in->nx;
  a.ny = in->ny;
  a.nz = in->nz;
  a.dirichlet_bottom = in->dirichlet_bottom ? 1 : 0;
  a.dx = in->dx;
  a.dy = in->dy;
  a.dz = in->dz;
  a.rho = in->rho;
  a.g = in->g;
  a.ux = in->ux;
  a.uy = in->uy;
  a.uz = in->uz;
  a.ap = ap;
  a.aw = aw;
  a.ae = ae;
  a.as = as;
  a.an = an;
  a.ab = ab;
  a.at = at;
  a.b = b;
  const long long n = (long long)in->nx * in->ny * in->nz;
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  // enough CTAs of 256 threads to fill every SM (8 resident each), fewer for small blocks
  const int grid = (int)std::min<long long>((n + 255) / 256, (long long)sms * 8);
  CU(launch_assemble_pcorr(a, grid, ctx->stream));
  return SIP_OK;
}

int sip_residual_norm(sip_ctx *ctx, const sip_block_desc *blk, double *rnorm_out, double *bnorm_out) {
  if (!ctx) return SIP_ERR_INVALID_ARG;
  NatBlock nb;
  const std::string why = natblock_from_desc(blk, &nb);
  if (!why.empty()) return fail(ctx, SIP_ERR_INVALID_ARG, why);
  CU(cudaSetDevice(ctx->device));
  const long long np = resnorm_parts(nb);
  double *scratch = nullptr;
  CU(ctx_alloc(ctx, (void **)&scratch, (size_t)(2 * np + 2) * sizeof(double)));
  double out[2] = {0.0, 0.0};
  cudaError_t e = launch_resnorm(nb, scratch, scratch + 2 * np, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + 2 * np, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream);
  ctx_free(ctx, scratch);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, SIP_ERR_CUDA, std::string("residual norm: ") + cudaGetErrorString(e));
  if (rnorm_out) *rnorm_out = out[0];
  if (bnorm_out) *bnorm_out = out[1];
  return SIP_OK;
}

int sip_residual_norm_noalloc(sip_ctx *ctx, const sip_block_desc *blk, double *norms_dev) {
  if (!ctx) return SIP_ERR_INVALID_ARG;
  if (!norms_dev) return fail(ctx, SIP_ERR_INVALID_ARG, "null output pointer");
  if (reinterpret_cast<uintptr_t>(norms_dev) % alignof(double) != 0)
    return fail(ctx, SIP_ERR_INVALID_ARG, "norms_dev must be 8-byte aligned");
  {
    // the output must be device (or managed) memory of the context's device:
    // a host pointer or another device's memory would fault in the kernel
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, norms_dev) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SIP_ERR_INVALID_ARG, "norms_dev is not a CUDA pointer");
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        (pa.type == cudaMemoryTypeDevice && pa.device != ctx->device))
      return fail(ctx, SIP_ERR_INVALID_ARG, "norms_dev must be device memory of the context's device");
  }
  NatBlock nb;
  const std::string why = natblock_from_desc(blk, &nb);
  if (!why.empty()) return fail(ctx, SIP_ERR_INVALID_ARG, why);
  const long long np = resnorm_parts(nb);
  if (np > kNoallocParts)
    return fail(ctx, SIP_ERR_INVALID_ARG,
                "block has " + std::to_string((long long)nb.nx * nb.ny * nb.nz) +
                    " cells; sip_residual_norm_noalloc handles at most " +
                    std::to_string((long long)kNoallocParts * kResChunk) + " (SIP_NOALLOC_MAX_CELLS)");
  CU(cudaSetDevice(ctx->device));
  double *scratch = nullptr;
  CU(noalloc_scratch(ctx->device, &scratch));
  const cudaError_t e = launch_resnorm(nb, scratch, norms_dev, ctx->stream);
  if (e != cudaSuccess) {
    noalloc_forget(ctx->device);  // the next call looks the address up again
    return fail(ctx, SIP_ERR_CUDA, std::string("residual norm: ") + cudaGetErrorString(e));
  }
  return SIP_OK;
}

int sip_profile_enable(sip_plan *p, int enable) {
  if (!p) return SIP_ERR_INVALID_ARG;
  p->prof = enable != 0;
  return SIP_OK;
}

int sip_profile_read(sip_plan *p, int nkinds, double *ms, int64_t *counts, int reset) {
  if (!p || nkinds < 0) return SIP_ERR_INVALID_ARG;
  sip_ctx *ctx = p->ctx;
  CU(cudaStreamSynchronize(ctx->stream));
  for (auto &r : p->recs) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, r.a, r.b));
    p->prof_ms[r.kind] += t;
    p->prof_n[r.kind] += 1;
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->recs.clear();
  for (int k = 0; k < nkinds && k <= K_NKINDS; ++k) {
    if (ms) ms[k] = p->prof_ms[k];
    if (counts) counts[k] = p->prof_n[k];
  }
  if (reset) {
    for (int k = 0; k <= K_NKINDS; ++k) {
      p->prof_ms[k] = 0;
      p->prof_n[k] = 0;
    }
  }
  return SIP_OK;
}

int sip_launch_count(sip_plan *p, int64_t *count_out) {
  if (!p || !count_out) return SIP_ERR_INVALID_ARG;
  *count_out = p->launches;
  return SIP_OK;
}

const char *sip_kernel_name(int kind) {
  static const char *names[] = {"factor", "fwd64",        "bwd64",       "factor32", "fwd32",  "bwd32", "bwd32_x0",
                                "resid64", "resid32", "resid32_norm", "resid64_r32", "update64", "utility"};
  static_assert(sizeof(names) / sizeof(names[0]) == K_NKINDS + 1, "kernel names");
  if (kind < 0 || kind > K_NKINDS) return nullptr;
  return names[kind];
}

int sip_plan_shape(sip_plan *p, int *rows_per_thread, int *tile_k, int *stages) {
  if (!p) return SIP_ERR_INVALID_ARG;
  if (rows_per_thread) *rows_per_thread = p->Q;
  if (tile_k) *tile_k = p->TK;
  if (stages) *stages = p->Rk[plan_kinds(p->mode)[1]];
  return SIP_OK;
}

int sip_plan_bytes(sip_plan *p, size_t *bytes_out) {
  if (!p || !bytes_out) return SIP_ERR_INVALID_ARG;
  *bytes_out = p->bytes;
  return SIP_OK;
}

int sip_plan_destroy(sip_plan *p) {
  if (!p) return SIP_OK;
  cudaStreamSynchronize(p->ctx->stream);
  if (p->trace && !p->trace_path.empty()) {
    std::vector<unsigned long long> h((size_t)K_NKINDS * p->ntiles * kTraceWords);
    if (cudaMemcpy(h.data(), p->trace, h.size() * 8, cudaMemcpyDeviceToHost) == cudaSuccess) {
      FILE *fo = fopen(p->trace_path.c_str(), "a");
      if (fo) {
        fprintf(fo, "# plan ntiles=%d Q=%d NW=%d TK=%d\n", p->ntiles, p->Q, p->NW, p->TK);
        for (int k = 0; k < K_NKINDS; ++k)
          for (const auto &bh : p->blocks)
            for (int ck = 0; ck < bh.db.nTK; ++ck)
              for (int cj = 0; cj < bh.db.nTJ; ++cj) {
                const int gt = bh.db.tile0 + ck * bh.db.nTJ + cj;
                const unsigned long long *r = &h[((size_t)k * p->ntiles + gt) * kTraceWords];
                if (!r[0]) continue;
                fprintf(fo, "%s %d %d %d %llu %llu %llu %llu %llu %llu\n", sip_kernel_name(k), gt, cj, ck, r[0], r[1],
                        r[2], r[3], r[4], r[5]);
              }
        fclose(fo);
      }
    }
  }
  free_plan_memory(p);
  delete p;
  return SIP_OK;
}

}  // extern "C"
