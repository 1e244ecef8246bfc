// sip_resrow.cu -- the residual r = b - A x of a SIP iteration (Sec. 1,
// Eq. 3: the right-hand side of the correction system L U d = r), computed
// outside the wavefront.
//
// The residual has no recurrence, so it does not belong on the critical path
// of the forward substitution: a row-parallel kernel computes it over the
// plane layout ahead of the sweep, and the forward sweep then runs only the
// L recurrence on r (in place).  Work
// decomposition: one warp per plane row (s, k) of a block; lanes walk the
// row's cells j (contiguous in memory).  Cell (i, j, k) of row (s, k),
// m = s - k, sits at rowbase(s, k) + j, and its neighbours are
//   W (i-1): rowbase(s-1, k) + j      S (j-1): rowbase(s-1, k) + j - 1
//   E (i+1): rowbase(s+1, k) + j      N (j+1): rowbase(s+1, k) + j + 1
//   B (k-1): rowbase(s-1, k-1) + j    T (k+1): rowbase(s+1, k+1) + j
// so every access of a warp is a contiguous run.  Rows are numbered per
// block k-major (row = row0 + k (nx + ny - 1) + m), which puts the rows a
// row reads from within one grid-stride pass: they are served from L2.
//
// For a symmetric matrix (Eq. 2 with AW_P = AE_W, AS_P = AN_S, AB_P = AT_B)
// the lower coefficients come from the W, S and B cells' A parts.  The
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

// the first four values of an A record (16-byte aligned: 16 B in FP32, 32 B
// in FP64) with vector loads
__device__ __forceinline__ void ld_rec4(const float *a, float v[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(a);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld_rec4(const double *a, double v[4]) {
  const double2 t0 = reinterpret_cast<const double2 *>(a)[0], t1 = reinterpret_cast<const double2 *>(a)[1];
  v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

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
  int nx = 0, ny = 0, nz = 0, mmax = 0, nm = 1;
  long long row0 = 0, rowend = 0;
  const int *PO = nullptr, *F = nullptr;
  // the current block's arrays (block-local cell offsets fit in 32 bits)
  const TA *__restrict__ Ab = nullptr;
  const TX *__restrict__ Xb = nullptr;
  const TX *__restrict__ Bb = nullptr;
  TR *__restrict__ Rb = nullptr;
  double acc = 0.0;
  for (long long row = (long long)blockIdx.x * (kRowThreads / 32) + (threadIdx.x >> 5); row < P.nrows;
       row += nwarps) {
    while (row >= rowend) {  // rows ascend: the owning block only moves forward
      ++bi;
      const DevBlock &B = P.blocks[bi];
      nx = B.nx; ny = B.ny; nz = B.nz; mmax = B.mmax; nm = nx + ny - 1;
      row0 = B.row0; rowend = row0 + (long long)nz * nm;
      PO = B.PO; F = B.F;
      Ab = P.arec + B.cell0 * NA;
      Xb = P.x + B.cell0;
      Bb = P.b + B.cell0;
      Rb = P.r + B.cell0;
    }
    const int lr = (int)(row - row0);
    const int k = lr / nm, m = lr - k * nm, s = m + k;
    const int fm = F[m];
    const int shift = max(0, m - nx + 1);
    const int bP = PO[s] + F[min(s, mmax)] - fm - shift;
    int bW = 0, bE = 0, bB = 0, bT = 0;
    if (m > 0 || k > 0) {
      const int lo = PO[s - 1] + F[min(s - 1, mmax)];
      if (m > 0) bW = lo - F[m - 1] - max(0, m - nx);
      bB = lo - fm - shift;
    }
    if (m < mmax || k < nz - 1) {
      const int hi = PO[s + 1] + F[min(s + 1, mmax)];
      if (m < mmax) bE = hi - F[m + 1] - max(0, m - nx + 2);
      bT = hi - fm - shift;
    }
    const int jlo = max(0, m - (nx - 1)), jhi = min(ny - 1, m);
    const bool hb = k > 0, ht = k < nz - 1;
    for (int j = jlo + lane; j <= jhi; j += 32) {
      const int i = m - j;
      const int c = bP + j;
      const TA *a = Ab + (size_t)c * NA;
      TC r = (TC)Bb[c];
      const TC x0 = (TC)Xb[c];
      const bool hw = i > 0, he = i < nx - 1, hs = j > 0, hn = j < ny - 1;
      const TC xw = hw ? (TC)Xb[bW + j] : TC(0);
      const TC xe = he ? (TC)Xb[bE + j] : TC(0);
      const TC xs = hs ? (TC)Xb[bW + j - 1] : TC(0);
      const TC xn = hn ? (TC)Xb[bE + j + 1] : TC(0);
      const TC xb = hb ? (TC)Xb[bB + j] : TC(0);
      const TC xt = ht ? (TC)Xb[bT + j] : TC(0);
      TC ap, ae, an, at, aw, as, ab;
      if constexpr (SYM) {
        TA v[4];
        ld_rec4(a, v);  // [AP AE AN AT]
        ap = (TC)v[0]; ae = (TC)v[1]; an = (TC)v[2]; at = (TC)v[3];
        aw = hw ? (TC)Ab[(size_t)(bW + j) * NA + OAE] : TC(0);
        as = hs ? (TC)Ab[(size_t)(bW + j - 1) * NA + OAN] : TC(0);
        ab = hb ? (TC)Ab[(size_t)(bB + j) * NA + OAT] : TC(0);
      } else {
        TA v[8];
        ld_rec4(a, v);  // [AP AW AE AS AN AB AT 0]
        ld_rec4(a + 4, v + 4);
        ap = (TC)v[0]; aw = (TC)v[1]; ae = (TC)v[2]; as = (TC)v[3];
        an = (TC)v[4]; ab = (TC)v[5]; at = (TC)v[6];
      }
      r = fma(-ap, x0, r);
      r = fma(-aw, xw, r);
      r = fma(-ae, xe, r);
      r = fma(-as, xs, r);
      r = fma(-an, xn, r);
      r = fma(-ab, xb, r);
      r = fma(-at, xt, r);
      Rb[c] = (TR)r;
      if constexpr (NORM) acc = fma((double)r, (double)r, acc);
    }
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
