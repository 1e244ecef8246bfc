// sip_resrow.cu -- the residual r = b - A x of a SIP iteration (Sec. 1,
// Eq. 3: the right-hand side of the correction system L U d = r), computed
// outside the wavefront.
//
// The residual has no recurrence, so it does not belong on the critical path
// of the forward substitution: a kernel over the plan's tile layout computes
// it ahead of the sweep, and the forward sweep then runs only the L
// recurrence on r (in place).  In the tile layout (sip_internal.h) the 32
// lanes l = j & 31 of a j block cj and row k sit side by side at each
// position p = i + l of the row, so a position is one 32-element run:
//   element(i, j, k) = row(cj, k) + 32 (i + l) + l,
//   row(cj, k) = sk0 + 32 (k nTJ + cj) Lp.
// Work decomposition: one warp per position of a row, lane l = cell
// (p - l, 32 cj + l, k), so every access of a warp is a contiguous run.  The
// neighbours of element e are W/E: e -+ 32; S: e - 33 (lane 0: lane 31 of
// the j block cj - 1 at position p + 31); N: e + 33 (lane 31: lane 0 of
// cj + 1 at position p - 31); B/T: e -+ 32 nTJ Lp.  Tasks are numbered per
// block row-major (task = row0 + (k nTJ + cj) Lp + p), so a warp's
// neighbour rows are read by nearby warps of the same pass and served from
// L2.  Padding positions (p - l outside [0, nx), or j >= ny) are skipped and
// keep the zero they were allocated with.
//
// For a symmetric matrix (Eq. 2 with AW_P = AE_W, AS_P = AN_S, AB_P = AT_B)
// the lower coefficients come from the W, S and B cells' A records.  The
// seven products are accumulated in the fixed order P, W, E, S, N, B, T
// with fused multiply-adds; neighbours outside the block contribute zero.
// The norm is a per-CTA sum of r^2 over a plan-constant grid, so it is
// deterministic.
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_internal.h"

namespace sipk {

namespace {

__device__ __forceinline__ int ld_status(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kRowThreads = 256;

template <typename TA, typename TX, typename TR, bool SYM, bool NORM>
__global__ void __launch_bounds__(kRowThreads, 4) k_resrow(RowParams<TA, TX, TR> P) {
  using TC = TX;  // arithmetic precision: that of the iterate
  __shared__ double s_red[kRowThreads / 32];
  if (__syncthreads_or(P.ctl->done || ld_status(P.status) != DEV_OK)) return;
  constexpr int NA = SYM ? 4 : 8;  // values per A record
  constexpr int OAE = SYM ? 1 : 2, OAN = SYM ? 2 : 4, OAT = SYM ? 3 : 6;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (kRowThreads / 32);
  int bi = -1;
  int nx = 0, ny = 0, nz = 0, nTJ = 1, Lp = 1;
  long long task0 = 0, taskend = 0, sk0 = 0, kstr = 0;
  double acc = 0.0;
  for (long long task = (long long)blockIdx.x * (kRowThreads / 32) + (threadIdx.x >> 5); task < P.nrows;
       task += nwarps) {
    while (task >= taskend) {  // tasks ascend: the owning block only moves forward
      ++bi;
      const DevBlock &B = P.blocks[bi];
      nx = B.nx; ny = B.ny; nz = B.nz; nTJ = B.nTJ; Lp = B.Lp;
      task0 = B.row0;
      taskend = task0 + (long long)nz * nTJ * Lp;
      sk0 = B.sk0;
      kstr = 32ll * nTJ * Lp;
    }
    const long long lt = task - task0;
    const long long rw = lt / Lp;  // row index k nTJ + cj
    const int ps = (int)(lt - rw * Lp);
    const int k = (int)(rw / nTJ), cj = (int)(rw - (long long)k * nTJ);
    const int j = cj * 32 + lane, i = ps - lane;
    if (j >= ny || (unsigned)i >= (unsigned)nx) continue;
    const long long c = sk0 + (rw * Lp + ps) * 32 + lane;
    const bool hw = i > 0, he = i < nx - 1, hs = j > 0, hn = j < ny - 1, hb = k > 0, ht = k < nz - 1;
    // S / N across a j-block edge: the adjacent block's edge lane, 31 positions away
    const long long cS = !hs ? c : (lane > 0 ? c - 33 : c - 32 * Lp + 31 * 32 + 31);
    const long long cN = !hn ? c : (lane < 31 ? c + 33 : c + 32 * Lp - 31 * 32 - 31);
    const long long cB = hb ? c - kstr : c, cT = ht ? c + kstr : c;
    const TA *a = P.arec + c * NA;
    TC r = (TC)P.b[c];
    const TC x0 = (TC)P.x[c];
    const TC xw = hw ? (TC)P.x[c - 32] : TC(0);
    const TC xe = he ? (TC)P.x[c + 32] : TC(0);
    const TC xs = hs ? (TC)P.x[cS] : TC(0);
    const TC xn = hn ? (TC)P.x[cN] : TC(0);
    const TC xb = hb ? (TC)P.x[cB] : TC(0);
    const TC xt = ht ? (TC)P.x[cT] : TC(0);
    const TC ap = (TC)a[0], ae = (TC)a[OAE], an = (TC)a[OAN], at = (TC)a[OAT];
    TC aw, as, ab;
    if constexpr (SYM) {
      aw = hw ? (TC)P.arec[(c - 32) * NA + OAE] : TC(0);
      as = hs ? (TC)P.arec[cS * NA + OAN] : TC(0);
      ab = hb ? (TC)P.arec[cB * NA + OAT] : TC(0);
    } else {
      aw = (TC)a[1];
      as = (TC)a[3];
      ab = (TC)a[5];
    }
    r = fma(-ap, x0, r);
    r = fma(-aw, xw, r);
    r = fma(-ae, xe, r);
    r = fma(-as, xs, r);
    r = fma(-an, xn, r);
    r = fma(-ab, xb, r);
    r = fma(-at, xt, r);
    P.r[c] = (TR)r;
    if constexpr (NORM) acc = fma((double)r, (double)r, acc);
  }
  if constexpr (NORM) {
    // fixed shuffle tree, then the warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kRowThreads / 32; ++q) t += s_red[q];
      P.partials[blockIdx.x] = t;
    }
  }
}

template <typename TA, typename TX, typename TR>
const void *row_kernel(bool sym, bool norm) {
  if (sym) return norm ? (const void *)k_resrow<TA, TX, TR, true, true> : (const void *)k_resrow<TA, TX, TR, true, false>;
  return norm ? (const void *)k_resrow<TA, TX, TR, false, true> : (const void *)k_resrow<TA, TX, TR, false, false>;
}

}  // namespace

int row_threads() { return kRowThreads; }

template <typename TA, typename TX, typename TR>
cudaError_t launch_resrow(const RowParams<TA, TX, TR> &prm, bool sym, int grid, cudaStream_t st) {
  void *args[] = {(void *)&prm};
  return cudaLaunchKernel(row_kernel<TA, TX, TR>(sym, prm.partials != nullptr), dim3(grid), dim3(kRowThreads), args,
                          0, st);
}

template <typename TA, typename TX, typename TR>
int resrow_max_active(bool sym, bool norm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, row_kernel<TA, TX, TR>(sym, norm), kRowThreads, 0) !=
      cudaSuccess)
    return 0;
  return occ;
}

// the four precision combinations of the solver modes
#define SIP_ROW_INST(TA, TX, TR)                                                                              \
  template cudaError_t launch_resrow<TA, TX, TR>(const RowParams<TA, TX, TR> &, bool, int, cudaStream_t); \
  template int resrow_max_active<TA, TX, TR>(bool, bool);
SIP_ROW_INST(double, double, double)  // FP64 iteration
SIP_ROW_INST(float, float, float)     // FP32 iteration / inner iterations of the refinement
SIP_ROW_INST(double, double, float)   // refinement residual, FP64 coefficients
SIP_ROW_INST(float, double, float)    // refinement residual, FP32 coefficients
#undef SIP_ROW_INST

}  // namespace sipk
