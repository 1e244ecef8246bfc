// sip_internal.h -- structures shared by the host runtime and the sm_103a
// kernels of libsip.so (not part of the public C ABI in include/sip.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct sip_ctx;  // include/sip.h

namespace sipk {

// device status word values (host maps them to SIP_ERR_*)
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_BREAKDOWN = 2;

constexpr int kTJ = 32;           // j extent of a column tile = one warp's lanes
constexpr int kFaceWordsMax = 6;  // 3 FP64 values (the factorisation's UN, UE, UT)

// Per-cell records of a plan (arrays of structs, 16-byte aligned):
//   L record [LB LW LS 1/LP]   (forward substitution)
//   U record [UE UN UT 0]      (backward substitution)
//   A record [AP AE AN AT] (symmetric) or [AP AW AE AS AN AB AT 0] (general),
//            in the sweep precision, plus an FP64 copy for the outer residual
//            of the refinement when the coefficients are FP64
//   A7 record (factorisation input, FP64) [AP AW AE AS AN AB AT 0]
constexpr int REC_LB = 0, REC_LW = 1, REC_LS = 2, REC_RLP = 3;
constexpr int RECB_UE = 0, RECB_UN = 1, RECB_UT = 2;
__host__ __device__ constexpr int a_rec_values(bool sym) { return sym ? 4 : 8; }

// Plane layout of one block.  Plane s = i + j + k holds the cells with that
// index sum; inside a plane the rows k ascend and inside a row the cells j
// ascend.  With f(m) the number of (i, j) with i + j = m and F(m) = sum of
// f(0..m), cell (i, j, k) of plane s sits at
//   cell0 + PO[s] + F[min(s, mmax)] - F[s - k] + j - max(0, s - k - (nx - 1)).
// Sweeps tile the (j, k) cross-section into 32 x TK column tiles; a CTA owns
// one tile and walks it along i (a warp owns Q rows k of the tile).
struct DevBlock {
  int nx, ny, nz, nplanes;
  int TK, nTJ, nTK, mmax;
  int tile0;            // global index of the block's tile (0, 0)
  int nsteps_max;       // nx + 32 + TK - 2
  long long cell0;      // first plan cell of the block
  const int *PO;        // [nplanes] first cell of each plane
  const int *F;         // [mmax + 1] prefix sums of the 2-D diagonal lengths
  long long face0;      // first face word of the block's tiles
  long long face_tile_words;  // face words per tile (nsteps_max * (32 + TK) * kFaceWordsMax)
  // x-chain interfaces of a multi-block mesh: neighbour block across the -x
  // face (lo) and the +x face (hi), or -1; overlap rectangle j < nj, k < nk
  int lo_blk, hi_blk;
  int lo_nj, lo_nk, hi_nj, hi_nk;
  // rows of the row-parallel kernels: the block's plane rows (s, k) are
  // numbered row0 + k (nx + ny - 1) + (s - k)
  long long row0;
};

__host__ __device__ inline int plane_row_base(const int *PO, const int *F, int mmax, int nx, int s, int k) {
  const int m = s - k;
  return PO[s] + F[s < mmax ? s : mmax] - F[m] - (m - nx + 1 > 0 ? m - nx + 1 : 0);
}

// Steps a substitution sweep's tile lets its upstream tiles run ahead before
// it starts (the start slack), by value size.  A tile's first prefetched
// faces may then be stale and are re-read, which costs less than the longer
// pipeline fill of a larger slack (measured on GB300: 2 steps 6 % faster than
// 5 at 256^3, 13 % at 128^3; with the 3-stage ring 1 step is best for FP32,
// 2 for FP64, within 4 % of each other).
__host__ __device__ constexpr int sweep_lead(int esize) { return esize == 4 ? 1 : 2; }

struct Tile {
  int blk;    // block index
  int cj, ck; // tile coordinates in the block
  int gtile;  // global tile index = blocks[blk].tile0 + ck * nTJ + cj
};

// Device-resident control of an iterate/solve sequence.
struct Ctl {
  int iter;       // updates applied so far
  int done;       // the stop rule fired: later kernels of the sequence do nothing
  int max_iters;  // stop when iter reaches it
  int nhist;      // entries written to hist
  double rtol;    // stop when relres <= rtol (negative: never)
  double bnorm;   // ||b||_2 of the sequence's right-hand side
  double relres;  // last relres
  unsigned epochs[2];  // face tags: a kernel reads epochs[slot] and sets epochs[slot ^ 1]
  int pad[2];
};

struct SweepCommon {
  const DevBlock *blocks;
  const Tile *tiles;   // tiles in claim order
  int ntiles;
  int tab_ints;        // shared-memory capacity for one block's PO + F tables
  int *ticket;         // claim counter, zero at launch
  int *reset_ticket;   // counter this launch zeroes for the next launch (nullable)
  Ctl *ctl;            // epochs, done flag
  int ep_slot;
  int stall;           // test hook: consumers expect a tag that is never written
  uint64_t *faces;
  int *status;
  long long max_spin;
  // diagnostics (nullable): per tile [claim, gate passed, end, slow face waits,
  // ns in slow waits, SM id]; globaltimer nanoseconds
  unsigned long long *trace;
};
constexpr int kTraceWords = 6;

template <typename T>
struct FwdParams {
  SweepCommon c;
  const T *rec;  // L records
  const T *r;    // right-hand side of the substitution (the residual)
  T *y;          // may alias r
};

template <typename T>
struct BwdParams {
  SweepCommon c;
  const T *rec;  // backward records
  const T *y;
  T *x;          // correction accumulated in place (x <- x + d)
};

template <typename TF>
struct FacParams {
  SweepCommon c;
  const double *a7;  // A7 records
  TF *recF;          // L records
  TF *recB;          // U records
  double alpha;
};

// Residual r = b - A x of every plan cell, one warp per plane row
// (sip_resrow.cu).  Arithmetic in TX (the iterate's type), A widened from TA.
template <typename TA, typename TX, typename TR>
struct RowParams {
  const DevBlock *blocks;
  int nblocks;
  long long nrows;    // rows of all blocks
  const Ctl *ctl;     // done: the kernel does nothing
  const int *status;  // not DEV_OK: the kernel does nothing
  const TA *arec;     // A records: [AP AE AN AT] (symmetric) or [AP AW AE AS AN AB AT 0] per cell
  const TX *b, *x;
  TR *r;
  double *partials;  // per CTA sum of r^2 (nullptr: no norm)
};
int row_threads();
template <typename TA, typename TX, typename TR>
cudaError_t launch_resrow(const RowParams<TA, TX, TR> &prm, bool sym, int grid, cudaStream_t st);
template <typename TA, typename TX, typename TR>
int resrow_max_active(bool sym, bool norm);

// context pool policy (sip_api.cu): whether plan creations raise the
// pool's cached bytes to their peak footprint (default on)
void ctx_keep_peak(sip_ctx *ctx, bool on);

// utilities (sip_util.cu)
// the seven coefficient arrays of a block (natural layout, FP32 or FP64;
// symmetric: aw, as, ab are taken from the neighbours' ae, an, at)
struct PackSrc {
  const void *a[7];  // ap aw ae as an ab at
  int f32, sym;
};
cudaError_t launch_pack_records(const PackSrc &S, const DevBlock &hb, double *a7, void *recA, int recA_f32,
                                double *arec64, cudaStream_t st);
cudaError_t launch_to_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st);
cudaError_t launch_from_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st);
cudaError_t launch_sumsq_partials(const double *v, long long n, double *partials, int nparts,
                                  cudaStream_t st);
cudaError_t launch_finalize(const double *partials, int n, Ctl *ctl, double *hist, int hist_cap,
                            const int *status, int mode, cudaStream_t st);
cudaError_t launch_set_ctl(Ctl *ctl, double rtol, int max_iters, cudaStream_t st);
cudaError_t launch_cast_f64_f32(const double *src, float *dst, long long n, cudaStream_t st);
cudaError_t launch_cast_f32_f64(const float *src, double *dst, long long n, cudaStream_t st);
// refinement update x64 += (double) d over n plan cells; nothing once ctl->done
cudaError_t launch_update64(const float *d, double *x64, long long n, const Ctl *ctl, cudaStream_t st);
cudaError_t launch_export_factors(const void *recF, const void *recB, int is_f32, double *const out[7],
                                  const DevBlock &hb, cudaStream_t st);

// Natural-layout block for the residual norm (sip_resnorm.cu).  a[] = AP, AW,
// AE, AS, AN, AB, AT (double or float); symmetric: AW/AS/AB are not read.
struct NatBlock {
  int nx, ny, nz;
  int coef_f32;
  int symmetric;
  const void *a[7];
  const double *b, *x;
};
constexpr int kResChunk = 4096;  // cells per partial pair of the residual norm
// number of partial pairs (2 doubles each) the residual norm of nb needs
long long resnorm_parts(const NatBlock &nb);
// ||b - A x||_2, ||b||_2 of nb into out2[0..1] (device); scratch: 2 * resnorm_parts(nb) doubles
cudaError_t launch_resnorm(const NatBlock &nb, double *scratch, double *out2, cudaStream_t st);
// fixed scratch of the allocation-free residual norm (sip_noalloc.cu): room for
// kNoallocParts partial pairs; its device address for `device` (which must be
// current) is resolved once and cached
constexpr int kNoallocParts = 16384;
constexpr int kNoallocMaxDevices = 64;
cudaError_t noalloc_scratch(int device, double **out);
// drops the cached address of `device` (after a failed launch)
void noalloc_forget(int device);

// x-interface coupling of a multi-block plan (lagged block Jacobi): every
// interface face cell `cell` of a block gets beff[cell] = b[cell] -
// c[0] x[nb[0]] - c[1] x[nb[1]] from its neighbours' current x (nb[1] = -1:
// one coupling only).  Plan-global cell indices.
struct HaloEntry {
  long long cell;
  long long nb[2];
  double c[2];
};
// where the coupling coefficient c[slot] of entry e comes from: element p of a
// natural-layout coefficient array of the caller (double or float)
struct HaloSrc {
  int e, slot;
  const void *src;
  long long p;
};
cudaError_t launch_halo_coefs(const HaloSrc *src, int nsrc, HaloEntry *ent, int coef_f32, cudaStream_t st);
cudaError_t launch_halo(const HaloEntry *ent, int nent, const double *b, const double *x, double *beff,
                        const Ctl *ctl, cudaStream_t st);
// the refinement's inner exchange: interface cells of r32 minus the coupling
// terms of the current FP32 correction d (first: save r32's values first)
cudaError_t launch_halo32(const HaloEntry *ent, int nent, float *r32, const float *d, float *save, bool first,
                          const Ctl *ctl, cudaStream_t st);

// pressure-correction assembly (sip_assemble.cu): inputs and outputs of one
// block, device pointers; aw / as / ab may be null (symmetric storage)
struct PcorrArgs {
  int nx, ny, nz, dirichlet_bottom;
  const double *dx, *dy, *dz, *rho, *g, *ux, *uy, *uz;
  double *ap, *aw, *ae, *as, *an, *ab, *at, *b;
};
cudaError_t launch_assemble_pcorr(const PcorrArgs &a, int grid, cudaStream_t st);

// finalize modes
constexpr int FIN_BNORM = 0;   // partials are ||b||^2 pieces: set ctl->bnorm
constexpr int FIN_RELRES = 1;  // partials are ||r||^2 pieces: relres, stop rule, counters

// Modelled duration (SM cycles) of one sweep launch over blocks of dims
// (nx, ny, nz per block) with 32 x (Q NW) tiles, `ctas` resident CTAs on
// `nsm` SMs (sip_shape.cu); -1 on a bad argument.
double sweep_model_cycles(const int *dims, int nblocks, int Q, int NW, int ctas, int nsm, bool fp64);

}  // namespace sipk
