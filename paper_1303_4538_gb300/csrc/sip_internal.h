// sip_internal.h -- structures shared by the host runtime and the sm_103a
// kernels of libsip.so (not part of the public C ABI in include/sip.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sipk {

// device status word values (host maps them to SIP_ERR_*)
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_BREAKDOWN = 2;

// Plane layout of one block.  Plane s = i + j + k holds the cells with that
// index sum; inside a plane the rows k ascend and inside a row the cells j
// ascend, so cell (i, j, k) sits at cell0 + rbT[k * nplanes + s] + j.
// Sweeps tile the (j, k) cross-section into TJ x TK column tiles; a CTA owns
// one tile and walks it along i (one thread per (j, k) column).
struct DevBlock {
  int nx, ny, nz, nplanes;
  int TJ, TK, nTJ, nTK;
  int tile0;            // global index of the block's tile (0, 0)
  int nsteps_max;       // nx + TJ + TK - 2
  long long cell0;      // first plan cell of the block
  const int *rbT;       // row-base table, [nz][nplanes]
  long long face0;      // first face word of the block's tiles
  long long face_tile_words;  // face words per tile (nsteps_max * (TJ + TK) * kFaceWordsMax)
  // x-chain interfaces of a multi-block mesh: neighbour block across the -x
  // face (lo) and the +x face (hi), or -1; overlap rectangle j < nj, k < nk
  int lo_blk, hi_blk;
  int lo_nj, lo_nk, hi_nj, hi_nk;
};

constexpr int kFaceWordsMax = 6;  // 3 FP64 values (the factorisation's UN, UE, UT)

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
  int exch_cells;      // max over blocks of (TJ + 2) * (TK + 2)
  int face_slots;      // max over blocks of TJ + TK (consumer records staged per step)
  int *ticket;         // claim counter, zero at launch
  int *reset_ticket;   // counter this launch zeroes for the next launch (nullable)
  Ctl *ctl;            // epochs, done flag
  int ep_slot;
  int stall;           // test hook: consumers expect a tag that is never written
  uint64_t *faces;
  int *status;
  long long max_spin;
};

template <typename T>
struct FwdParams {
  SweepCommon c;
  const T *ap, *aw, *ae, *as, *an, *ab, *at;  // plan layout (symmetric: aw, as, ab unused)
  const T *lb, *lw, *ls, *rlp;
  const T *b, *x;
  T *y;
  double *partials;  // per global tile: sum of r^2
};

template <typename T>
struct BwdParams {
  SweepCommon c;
  const T *un, *ue, *ut;
  const T *y;
  T *x;          // correction accumulated in place (x <- x + d)
  double *x64;   // refined mode, last inner iteration: x64 += (double) x
};

struct FacParams {
  SweepCommon c;
  const double *a[7];  // ap aw ae as an ab at (plan layout)
  double *f[7];        // lb lw ls rlp un ue ut
  float *f32[7];       // optional single-precision copies (nullable)
  double alpha;
};

template <typename TA>
struct ResParams {  // FP64 residual r = b - A x of the refinement loop (no recurrence)
  const DevBlock *blocks;
  const Tile *tiles;
  int ntiles;
  int exch_cells;
  Ctl *ctl;
  int *status;
  const TA *ap, *aw, *ae, *as, *an, *ab, *at;
  const double *b, *x;
  float *r32;
  double *partials;
};

// utilities (sip_util.cu)
cudaError_t launch_to_plan_f64(const void *src, int src_is_f32, double *dst, const DevBlock &hb,
                               int zero_face, int shift_axis, cudaStream_t st);
cudaError_t launch_to_plan_f32(const void *src, int src_is_f32, float *dst, const DevBlock &hb,
                               int zero_face, int shift_axis, cudaStream_t st);
cudaError_t launch_from_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st);
cudaError_t launch_f64_to_f32(const double *src, float *dst, long long n, cudaStream_t st);
cudaError_t launch_sumsq_partials(const double *v, long long n, double *partials, int nparts,
                                  cudaStream_t st);
cudaError_t launch_finalize(const double *partials, int n, Ctl *ctl, double *hist, int hist_cap,
                            const int *status, int mode, cudaStream_t st);
cudaError_t launch_set_ctl(Ctl *ctl, double rtol, int max_iters, cudaStream_t st);
cudaError_t launch_plan_to_natural_factors(const double *const f[7], double *const out[7],
                                           const DevBlock &hb, cudaStream_t st);

// finalize modes
constexpr int FIN_BNORM = 0;   // partials are ||b||^2 pieces: set ctl->bnorm
constexpr int FIN_RELRES = 1;  // partials are ||r||^2 pieces: relres, stop rule, counters

}  // namespace sipk
