// sip_api.cu -- host runtime and C ABI of libsip.so (declared in include/sip.h).
//
// A plan (the paper's redesigned solver module, arXiv:1303.4538 Sec. 4.1: the
// solver owns its coefficient arrays and computes the incomplete factorisation
// once, before the relaxations) holds, for every block, the plane layout
// tables, reordered copies of A, Stone's factors, the work vectors, the face
// buffers of the sweeps and a device-resident control block.  All launches go
// to the context's stream; the only device->host transfers are the control
// block reads that a call needs to return its results.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
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
  bool attrs_set = false;
  size_t kernel_static_smem = 0;  // largest static shared memory of any sweep kernel
};

static std::string g_create_error = "no error";

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

struct TileShape {
  int TJ = 32, TK = 8, R = 6;
};

}  // namespace

struct BlockHost {
  sip_block_desc d;
  DevBlock db;  // with device rbT
  std::vector<int> rbT;
  long long n = 0;
};

struct sip_plan {
  sip_ctx *ctx = nullptr;
  sip_options opt;
  int mode = 0;
  bool sym = false;
  std::vector<BlockHost> blocks;
  std::vector<sip_interface> ifaces;
  long long ncells = 0;
  int ntiles = 0;
  int NT = 256, EC = 0, FS = 0;
  int Rk[K_NKINDS] = {};     // stage depth chosen per kernel kind
  int gridk[K_NKINDS] = {};  // resident CTAs per kernel kind (grid of the ticketed sweeps)
  std::vector<void *> allocs;
  size_t bytes = 0;
  DevBlock *d_blocks = nullptr;
  Tile *d_tiles_f = nullptr, *d_tiles_b = nullptr;
  int *d_rb = nullptr;
  double *A64[7] = {};
  float *A32[7] = {};
  double *F64[7] = {};
  float *F32[7] = {};
  double *b64 = nullptr, *x64 = nullptr, *y64 = nullptr;
  float *r32 = nullptr, *d32 = nullptr, *y32 = nullptr;
  uint64_t *faces = nullptr;
  double *partials = nullptr;
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
};

// ------------------------------------------------------------------ helpers
namespace {

template <typename T>
cudaError_t palloc(sip_plan *p, T **ptr, size_t count) {
  void *v = nullptr;
  const size_t b = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&v, b);
  if (e != cudaSuccess) return e;
  p->allocs.push_back(v);
  p->bytes += b;
  *ptr = (T *)v;
  return cudaSuccess;
}

void free_plan_memory(sip_plan *p) {
  for (auto &r : p->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  p->recs.clear();
  for (auto e : p->pool) cudaEventDestroy(e);
  p->pool.clear();
  for (void *v : p->allocs) cudaFree(v);
  p->allocs.clear();
  if (p->h_ctl) cudaFreeHost(p->h_ctl);
  if (p->h_status) cudaFreeHost(p->h_status);
  p->h_ctl = nullptr;
  p->h_status = nullptr;
}

// Plane layout of a block: plane s = i+j+k, rows k ascending, cells j
// ascending; rbT[k*nplanes + s] + j is the cell's offset in the block.
void build_rowbase(int nx, int ny, int nz, std::vector<int> &rbT) {
  const int np = nx + ny + nz - 2;
  rbT.assign((size_t)np * nz, INT_MIN);
  long long off = 0;
  for (int s = 0; s < np; ++s) {
    const int klo = std::max(0, s - (nx - 1) - (ny - 1)), khi = std::min(nz - 1, s);
    for (int k = klo; k <= khi; ++k) {
      const int jlo = std::max(0, s - k - (nx - 1)), jhi = std::min(ny - 1, s - k);
      if (jlo > jhi) continue;
      rbT[(size_t)k * np + s] = (int)(off - jlo);
      off += jhi - jlo + 1;
    }
  }
}

int tile_count(int ny, int nz, int TJ, int TK) { return ((ny + TJ - 1) / TJ) * ((nz + TK - 1) / TK); }

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
  for (int kind = 0; kind < K_NKINDS; ++kind)
    for (int R : {3, 6}) {
      const void *f = kernel_ptr(kind, R);
      if (!f) continue;
      cudaFuncAttributes fa;
      cudaError_t e = cudaFuncGetAttributes(&fa, f);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ctx->smem_optin - fa.sharedSizeBytes));
      if (e != cudaSuccess) {
        g_create_error = std::string("kernel attribute setup: ") + cudaGetErrorString(e);
        delete ctx;
        return SIP_ERR_CUDA;
      }
      ctx->kernel_static_smem = std::max(ctx->kernel_static_smem, (size_t)fa.sharedSizeBytes);
    }
  ctx->attrs_set = true;
  *out = ctx;
  return SIP_OK;
}

int sip_destroy(sip_ctx *ctx) {
  delete ctx;
  return SIP_OK;
}

const char *sip_last_error(sip_ctx *ctx) {
  static thread_local std::string copy;
  copy = ctx ? ctx->err : g_create_error;
  return copy.c_str();
}

}  // extern "C"

// ------------------------------------------------------------------ launches
namespace {

int max_active(sip_plan *p, int kind, int R, size_t smem) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_ptr(kind, R), p->NT, smem);
  return occ;
}

SweepCommon common(sip_plan *p, bool backward, int ticket, int reset, int slot) {
  SweepCommon c;
  c.blocks = p->d_blocks;
  c.tiles = backward ? p->d_tiles_b : p->d_tiles_f;
  c.ntiles = p->ntiles;
  c.exch_cells = p->EC;
  c.face_slots = p->FS;
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
  const size_t smem = kernel_smem(kind, R, p->NT, p->EC, p->FS);
  const int grid = std::max(1, std::min(p->ntiles, p->gridk[kind]));
  void *args[] = {(void *)&prm};
  ProfScope ps(p, kind);
  return cudaLaunchKernel(kernel_ptr(kind, R), dim3(grid), dim3(p->NT), args, smem, p->ctx->stream);
}

// utility launches (layout, reductions, control) are counted as kind K_NKINDS
#define UTIL(call) \
  do {             \
    ProfScope ps_(p, K_NKINDS); \
    CU(call);      \
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
int enqueue_iter_f64(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  FwdParams<double> f;
  f.c = common(p, false, 0, 1, 0);
  f.ap = p->A64[0]; f.aw = p->A64[1]; f.ae = p->A64[2]; f.as = p->A64[3];
  f.an = p->A64[4]; f.ab = p->A64[5]; f.at = p->A64[6];
  f.lb = p->F64[0]; f.lw = p->F64[1]; f.ls = p->F64[2]; f.rlp = p->F64[3];
  f.b = p->b64; f.x = p->x64; f.y = p->y64; f.partials = p->partials;
  CU(launch(p, p->sym ? K_FWD64S : K_FWD64, f));
  UTIL(launch_finalize(p->partials, p->ntiles, p->ctl, p->hist, p->hist_cap, p->status, FIN_RELRES, ctx->stream));
  BwdParams<double> b;
  b.c = common(p, true, 1, 0, 1);
  b.ue = p->F64[5]; b.un = p->F64[4]; b.ut = p->F64[6];
  b.y = p->y64; b.x = p->x64; b.x64 = nullptr;
  CU(launch(p, K_BWD64, b));
  return SIP_OK;
}

// One FP64 correction of the refinement: FP64 residual (+ stop rule), then
// m FP32 SIP iterations on A d = r from d = 0, the last adding d to x.
int enqueue_iter_refined(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  const int m = std::max(1, p->opt.inner_iters);
  const bool a32 = (p->A64[0] == nullptr);
  if (a32) {
    ResParams<float> r;
    r.blocks = p->d_blocks; r.tiles = p->d_tiles_f; r.ntiles = p->ntiles; r.exch_cells = p->EC;
    r.ctl = p->ctl; r.status = p->status;
    r.ap = p->A32[0]; r.aw = p->A32[1]; r.ae = p->A32[2]; r.as = p->A32[3];
    r.an = p->A32[4]; r.ab = p->A32[5]; r.at = p->A32[6];
    r.b = p->b64; r.x = p->x64; r.r32 = p->r32; r.partials = p->partials;
    CU(launch(p, p->sym ? K_RES32AS : K_RES32A, r));
  } else {
    ResParams<double> r;
    r.blocks = p->d_blocks; r.tiles = p->d_tiles_f; r.ntiles = p->ntiles; r.exch_cells = p->EC;
    r.ctl = p->ctl; r.status = p->status;
    r.ap = p->A64[0]; r.aw = p->A64[1]; r.ae = p->A64[2]; r.as = p->A64[3];
    r.an = p->A64[4]; r.ab = p->A64[5]; r.at = p->A64[6];
    r.b = p->b64; r.x = p->x64; r.r32 = p->r32; r.partials = p->partials;
    CU(launch(p, p->sym ? K_RES64S : K_RES64, r));
  }
  UTIL(launch_finalize(p->partials, p->ntiles, p->ctl, p->hist, p->hist_cap, p->status, FIN_RELRES, ctx->stream));
  for (int q = 0; q < m; ++q) {
    const bool first = q == 0, lastq = q == m - 1;
    FwdParams<float> f;
    f.c = common(p, false, 0, 1, 0);
    f.ap = p->A32[0]; f.aw = p->A32[1]; f.ae = p->A32[2]; f.as = p->A32[3];
    f.an = p->A32[4]; f.ab = p->A32[5]; f.at = p->A32[6];
    f.lb = p->F32[0]; f.lw = p->F32[1]; f.ls = p->F32[2]; f.rlp = p->F32[3];
    f.b = p->r32; f.x = p->d32; f.y = p->y32; f.partials = nullptr;
    const int fk = first ? K_FWD32Z : (p->sym ? K_FWD32S : K_FWD32);
    CU(launch(p, fk, f));
    BwdParams<float> b;
    b.c = common(p, true, 1, 0, 1);
    b.ue = p->F32[5]; b.un = p->F32[4]; b.ut = p->F32[6];
    b.y = p->y32; b.x = p->d32; b.x64 = lastq ? p->x64 : nullptr;
    const int bk = first ? (lastq ? K_BWD32ZU : K_BWD32Z) : (lastq ? K_BWD32U : K_BWD32);
    CU(launch(p, bk, b));
  }
  return SIP_OK;
}

int enqueue_iter(sip_plan *p) {
  return p->mode == SIP_MODE_F32_REFINED ? enqueue_iter_refined(p) : enqueue_iter_f64(p);
}

// Copy b and x of every block into the plan layout, ||b||, control reset.
int begin_sequence(sip_plan *p, double rtol, int max_iters) {
  sip_ctx *ctx = p->ctx;
  CU(cudaMemsetAsync(p->tickets, 0, 4 * sizeof(int), ctx->stream));
  UTIL(launch_set_ctl(p->ctl, rtol, max_iters, ctx->stream));
  for (auto &bh : p->blocks) {
    UTIL(launch_to_plan_f64(bh.d.b, 0, p->b64, bh.db, 0, 0, ctx->stream));
    UTIL(launch_to_plan_f64(bh.d.x, 0, p->x64, bh.db, 0, 0, ctx->stream));
  }
  UTIL(launch_sumsq_partials(p->b64, p->ncells, p->bparts, p->nbparts, ctx->stream));
  UTIL(launch_finalize(p->bparts, p->nbparts, p->ctl, p->hist, p->hist_cap, p->status, FIN_BNORM, ctx->stream));
  return SIP_OK;
}

int end_sequence(sip_plan *p) {
  sip_ctx *ctx = p->ctx;
  for (auto &bh : p->blocks) UTIL(launch_from_plan_f64(p->x64, bh.d.x, bh.db, ctx->stream));
  CU(cudaMemcpyAsync(&p->h_ctl[2], p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = check_status(p);  // synchronises
  if (rc != SIP_OK) return rc;
  p->last_nhist = p->h_ctl[2].nhist;
  return SIP_OK;
}

}  // namespace

extern "C" {

int sip_factor(sip_ctx *ctx, const sip_block_desc *blocks, int nblocks, const sip_interface *ifaces,
               int nifaces, const sip_options *opt_in, sip_plan **out) {
  if (!ctx || !out) return SIP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!blocks || nblocks < 1) return fail(ctx, SIP_ERR_INVALID_ARG, "need at least one block");
  if (nifaces < 0 || (nifaces > 0 && !ifaces)) return fail(ctx, SIP_ERR_INVALID_ARG, "bad interface list");
  if (nifaces > 0) return fail(ctx, SIP_ERR_INVALID_ARG, "interfaces are not supported by this build yet");
  sip_options opt;
  if (opt_in) opt = *opt_in;
  else sip_default_options(&opt);
  if (!(opt.alpha >= 0.0 && opt.alpha <= 1.0))
    return fail(ctx, SIP_ERR_INVALID_ARG, "alpha must lie in [0, 1]");
  if (opt.mode != SIP_MODE_F64 && opt.mode != SIP_MODE_F32_REFINED)
    return fail(ctx, SIP_ERR_INVALID_ARG, "unsupported mode");
  if (opt.mode == SIP_MODE_F32_REFINED && opt.inner_iters < 1)
    return fail(ctx, SIP_ERR_INVALID_ARG, "inner_iters must be >= 1");
  const bool sym = blocks[0].symmetric != 0;
  long long ncells = 0;
  for (int b = 0; b < nblocks; ++b) {
    const sip_block_desc &d = blocks[b];
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(ctx, SIP_ERR_INVALID_ARG, "block dims must be >= 1");
    const long long n = (long long)d.nx * d.ny * d.nz;
    if (n >= (1ll << 31) || (long long)d.nx + d.ny + d.nz > (1 << 24))
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

  sip_plan *p = new sip_plan();
  p->ctx = ctx;
  p->opt = opt;
  p->mode = opt.mode;
  p->sym = sym;
  p->ncells = ncells;

  // tile shape: threads per CTA and stage depth shared by every block
  TileShape ts;
  {
    const int NT = 256;
    int TJ = opt.tile_j, TK = opt.tile_k;
    if (TJ <= 0 || TK <= 0) {
      int maxny = 0;
      for (int b = 0; b < nblocks; ++b) maxny = std::max(maxny, blocks[b].ny);
      TJ = maxny >= 24 ? 32 : (maxny >= 12 ? 16 : 8);
      TK = NT / TJ;
    }
    if (!(TJ == 8 || TJ == 16 || TJ == 32) || TK < 2 || TJ * TK > 512 || (TJ * TK) % 32 != 0) {
      delete p;
      return fail(ctx, SIP_ERR_INVALID_ARG, "tile_j must be 8, 16 or 32; tile_k >= 2; tile_j*tile_k a multiple of 32, <= 512");
    }
    ts.TJ = TJ;
    ts.TK = TK;
  }
  p->NT = ts.TJ * ts.TK;
  p->EC = (ts.TJ + 2) * (ts.TK + 2);
  p->FS = ts.TJ + ts.TK;

  // per-block layout tables and tile lists
  std::vector<DevBlock> hdb;
  std::vector<Tile> tiles;
  long long cell0 = 0, face0 = 0;
  size_t rb_total = 0;
  p->blocks.resize(nblocks);
  for (int b = 0; b < nblocks; ++b) {
    BlockHost &bh = p->blocks[b];
    bh.d = blocks[b];
    const int nx = bh.d.nx, ny = bh.d.ny, nz = bh.d.nz;
    build_rowbase(nx, ny, nz, bh.rbT);
    bh.n = (long long)nx * ny * nz;
    DevBlock &db = bh.db;
    db.nx = nx; db.ny = ny; db.nz = nz; db.nplanes = nx + ny + nz - 2;
    db.TJ = ts.TJ; db.TK = ts.TK;
    db.nTJ = (ny + ts.TJ - 1) / ts.TJ;
    db.nTK = (nz + ts.TK - 1) / ts.TK;
    db.tile0 = p->ntiles;
    db.nsteps_max = nx + ts.TJ + ts.TK - 2;
    db.cell0 = cell0;
    db.rbT = nullptr;
    db.face0 = face0;
    db.face_tile_words = (long long)db.nsteps_max * (ts.TJ + ts.TK) * kFaceWordsMax;
    db.lo_blk = db.hi_blk = -1;
    db.lo_nj = db.lo_nk = db.hi_nj = db.hi_nk = 0;
    const int nt = db.nTJ * db.nTK;
    p->ntiles += nt;
    face0 += (long long)nt * db.face_tile_words;
    cell0 += bh.n;
    rb_total += bh.rbT.size();
  }
  // claim order: anti-diagonal waves (cj + ck), blocks interleaved
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

  // device allocations
  auto bail = [&](cudaError_t e, const char *what) {
    free_plan_memory(p);
    delete p;
    return fail(ctx, e == cudaErrorMemoryAllocation ? SIP_ERR_OOM : SIP_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
#define PA(ptr, count)                                     \
  do {                                                     \
    cudaError_t e_ = palloc(p, &(ptr), (size_t)(count));   \
    if (e_ != cudaSuccess) return bail(e_, #ptr);          \
  } while (0)
  const long long N = ncells;
  PA(p->d_rb, rb_total);
  PA(p->d_blocks, nblocks);
  PA(p->d_tiles_f, p->ntiles);
  PA(p->d_tiles_b, p->ntiles);
  PA(p->faces, face0);
  PA(p->partials, p->ntiles);
  PA(p->bparts, p->nbparts);
  PA(p->ctl, 1);
  p->hist_cap = 1 << 20;
  PA(p->hist, p->hist_cap);
  PA(p->status, 1);
  PA(p->tickets, 4);
  PA(p->b64, N);
  PA(p->x64, N);
  const bool a32in = blocks[0].coef_dtype == 1;
  const int nA = 7;
  // FP64 copy of A: sweeps of the FP64 mode, factorisation input always
  double *A64tmp[7] = {};
  for (int q = 0; q < nA; ++q) PA(A64tmp[q], N);
  for (int q = 0; q < 7; ++q) PA(p->F64[q], N);
  if (p->mode == SIP_MODE_F64) {
    PA(p->y64, N);
    for (int q = 0; q < 7; ++q) p->A64[q] = A64tmp[q];
  } else {
    PA(p->r32, N);
    PA(p->d32, N);
    PA(p->y32, N);
    for (int q = 0; q < 7; ++q) PA(p->A32[q], N);
    for (int q = 0; q < 7; ++q) PA(p->F32[q], N);
    if (!a32in)
      for (int q = 0; q < 7; ++q) p->A64[q] = A64tmp[q];
  }
  {
    cudaError_t e = cudaMallocHost(&p->h_ctl, 3 * sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_status, 2 * sizeof(int));
    if (e != cudaSuccess) return bail(e, "pinned control block");
  }
  cudaStream_t st = ctx->stream;
  // tables
  {
    size_t off = 0;
    for (auto &bh : p->blocks) {
      cudaError_t e = cudaMemcpyAsync(p->d_rb + off, bh.rbT.data(), bh.rbT.size() * sizeof(int),
                                      cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return bail(e, "row tables");
      bh.db.rbT = p->d_rb + off;
      off += bh.rbT.size();
      hdb.push_back(bh.db);
    }
    cudaError_t e = cudaMemcpyAsync(p->d_blocks, hdb.data(), hdb.size() * sizeof(DevBlock), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_tiles_f, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_tiles_b, tiles_b.data(), tiles_b.size() * sizeof(Tile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->faces, 0, (size_t)face0 * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->tickets, 0, 4 * sizeof(int), st);
    // host vectors must outlive the async copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(e, "plan upload");
  }
  // Stage depth per kernel kind: the deepest ring (6, else 3) with which every
  // tile of the plan is resident at once (one wave), else the one that keeps
  // the most tiles resident.  The ticketed sweeps launch that many CTAs.
  {
    for (int kind = 0; kind < K_NKINDS; ++kind) {
      int bestR = 0, bestCap = -1;
      for (int R : {6, 3}) {
        const size_t smem = kernel_smem(kind, R, p->NT, p->EC, p->FS);
        if (smem + ctx->kernel_static_smem > ctx->smem_optin) continue;
        const int cap = ctx->nsm * max_active(p, kind, R, smem);
        if (cap >= p->ntiles) { bestR = R; bestCap = cap; break; }
        if (cap > bestCap) { bestR = R; bestCap = cap; }
      }
      if (bestCap < 1) {
        free_plan_memory(p);
        delete p;
        return fail(ctx, SIP_ERR_INVALID_ARG, "tile shape does not fit on an SM");
      }
      p->Rk[kind] = bestR;
      p->gridk[kind] = bestCap;
    }
  }
  // A into the plan layout; coefficients that point out of their block are zeroed
  {
    static const int zface[7] = {0, 1, 2, 3, 4, 5, 6};  // ap aw ae as an ab at
    static const int shift_src[7] = {-1, 2, -1, 4, -1, 6, -1};  // symmetric: aw<-ae, as<-an, ab<-at
    static const int shift_axis[7] = {0, 1, 0, 2, 0, 3, 0};
    for (auto &bh : p->blocks) {
      const void *src[7] = {bh.d.ap, bh.d.aw, bh.d.ae, bh.d.as, bh.d.an, bh.d.ab, bh.d.at};
      for (int q = 0; q < 7; ++q) {
        const void *s = src[q];
        int sh = 0;
        if (sym && (q == 1 || q == 3 || q == 5)) {
          s = src[shift_src[q]];
          sh = shift_axis[q];
        }
        cudaError_t e = launch_to_plan_f64(s, bh.d.coef_dtype, A64tmp[q], bh.db, sh ? 0 : zface[q], sh, st);
        if (e == cudaSuccess && p->A32[0])
          e = launch_to_plan_f32(s, bh.d.coef_dtype, p->A32[q], bh.db, sh ? 0 : zface[q], sh, st);
        if (e != cudaSuccess) return bail(e, "reorder A");
      }
    }
  }
  // Stone's factorisation (one wavefront sweep)
  {
    cudaError_t e = launch_set_ctl(p->ctl, -1.0, 0, st);
    if (e != cudaSuccess) return bail(e, "control");
    FacParams fp;
    fp.c = common(p, false, 2, 0, 0);
    for (int q = 0; q < 7; ++q) {
      fp.a[q] = A64tmp[q];
      fp.f[q] = p->F64[q];
      fp.f32[q] = p->F32[q];
    }
    fp.alpha = opt.alpha;
    e = launch(p, K_FACTOR, fp);
    if (e != cudaSuccess) return bail(e, "factor launch");
    int rc = check_status(p);
    if (rc != SIP_OK) {
      std::string msg = ctx->err;
      free_plan_memory(p);
      delete p;
      return fail(ctx, rc, msg);
    }
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
  for (int it = 0; it < niters; ++it) {
    rc = enqueue_iter(p);
    if (rc) return rc;
  }
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
  const int chunk = 16;
  cudaEvent_t ev[2];
  CU(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
  int issued = 0;  // iterations queued (each starts with one residual + stop check)
  int nq = 0, nc = 0;  // chunks queued / checked
  bool more = true;
  for (;;) {
    if (more) {
      const int n = std::min(chunk, max_iters + 1 - issued);
      for (int it = 0; it < n; ++it) {
        rc = enqueue_iter(p);
        if (rc) return rc;
      }
      issued += n;
      const int sl = nq & 1;
      CU(cudaMemcpyAsync(&p->h_ctl[sl], p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaMemcpyAsync(&p->h_status[sl], p->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaEventRecord(ev[sl], ctx->stream));
      ++nq;
      more = issued < max_iters + 1;
    }
    if (nq - nc >= 2 || (!more && nc < nq)) {
      const int sl = nc & 1;
      CU(cudaEventSynchronize(ev[sl]));
      ++nc;
      if (p->h_ctl[sl].done || p->h_status[sl] != DEV_OK) break;
      if (!more && nc == nq) break;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  Ctl *hc = &p->h_ctl[2];
  rc = end_sequence(p);
  if (rc) return rc;
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
  const double *f[7];
  for (int q = 0; q < 7; ++q) f[q] = p->F64[q];
  CU(launch_plan_to_natural_factors(f, out, p->blocks[blk].db, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return SIP_OK;
}

int sip_plane_layout(int nx, int ny, int nz, int32_t *rbT) {
  if (nx < 1 || ny < 1 || nz < 1 || !rbT || (long long)nx * ny * nz >= (1ll << 31)) return SIP_ERR_INVALID_ARG;
  std::vector<int> t;
  build_rowbase(nx, ny, nz, t);
  std::memcpy(rbT, t.data(), t.size() * sizeof(int));
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
  static const char *names[] = {"factor", "fwd64", "fwd64_sym", "bwd64", "fwd32", "fwd32_sym", "fwd32_x0",
                                "fwd32_norm", "fwd32_sym_norm", "bwd32", "bwd32_x0", "bwd32_upd64",
                                "bwd32_x0_upd64", "resid64", "resid64_sym", "resid64_a32", "resid64_a32_sym",
                                "utility"};
  static_assert(sizeof(names) / sizeof(names[0]) == K_NKINDS + 1, "kernel names");
  if (kind < 0 || kind > K_NKINDS) return nullptr;
  return names[kind];
}

int sip_plan_bytes(sip_plan *p, size_t *bytes_out) {
  if (!p || !bytes_out) return SIP_ERR_INVALID_ARG;
  *bytes_out = p->bytes;
  return SIP_OK;
}

int sip_plan_destroy(sip_plan *p) {
  if (!p) return SIP_OK;
  cudaStreamSynchronize(p->ctx->stream);
  free_plan_memory(p);
  delete p;
  return SIP_OK;
}

}  // extern "C"
