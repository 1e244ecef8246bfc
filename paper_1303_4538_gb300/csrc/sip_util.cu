// sip_util.cu -- layout conversion, deterministic reductions and sequence
// control kernels of libsip.so, plus the kernel registry's size rules.
#include <cmath>
#include <cstdint>

#include "sip_internal.h"
#include "sip_kernels.h"
#include "sip_layout.h"

namespace sipk {

// ------------------------------------------------------------ registry
const void *kernel_ptr(int kind, int Q, int R) {
  const void *p = kernel_ptr_64(kind, Q, R);
  if (!p) p = kernel_ptr_32(kind, Q, R);
  return p;
}

size_t kernel_smem(int kind, int Q, int R, int NT, int tab) {
  switch (kind) {
    case K_FACTOR:
    case K_FACTOR32: return fac_layout(Q, R, NT, tab).total;
    case K_FWD64: return fwd_layout(8, Q, R, NT, tab).total;
    case K_BWD64: return bwd_layout(8, false, Q, R, NT, tab).total;
    case K_FWD32: return fwd_layout(4, Q, R, NT, tab).total;
    case K_BWD32: return bwd_layout(4, false, Q, R, NT, tab).total;
    case K_BWD32Z: return bwd_layout(4, true, Q, R, NT, tab).total;
    default: return 0;
  }
}

// ------------------------------------------------------------ layout
static int util_grid(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

__device__ __forceinline__ long long plan_cell(const DevBlock &hb, int i, int j, int k) {
  return hb.cell0 + plane_row_base(hb.PO, hb.F, hb.mmax, hb.nx, i + j + k, k) + j;
}

// Walk over a block's natural rows (j, k): one warp per row, lanes stepping
// along i, so the natural-layout side of every copy is coalesced and the index
// arithmetic stays in 32 bits (a block has fewer than 2^31 cells).  f(i, j, k,
// p, c) gets the natural index p = i + nx (j + ny k) and the plan cell c.
constexpr int kWalkThreads = 256;

static int walk_grid(const DevBlock &hb) {
  const long long rows = (long long)hb.ny * hb.nz;
  long long g = (rows + kWalkThreads / 32 - 1) / (kWalkThreads / 32);
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename Fn>
__device__ __forceinline__ void walk_rows(const DevBlock &hb, Fn &&f) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nrows = hb.ny * hb.nz;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < nrows; r += gridDim.x * wpb) {
    const int k = r / hb.ny, j = r - k * hb.ny;
    const int p0 = r * hb.nx;
    for (int i = lane; i < hb.nx; i += 32) {
      const long long c = hb.cell0 + plane_row_base(hb.PO, hb.F, hb.mmax, hb.nx, i + j + k, k) + j;
      f(i, j, k, p0 + i, c);
    }
  }
}

// The seven matrix entries of every cell into the plan's records, one pass:
// the factorisation input a7 [AP AW AE AS AN AB AT 0] (FP64), the residual's
// A record in the sweep precision (symmetric [AP AE AN AT], general the a7
// order) and, where given, its FP64 copy.  Entries that point out of the
// block are zeroed; a symmetric matrix takes AW, AS, AB from the lower
// neighbour's AE, AN, AT (0 on the lower faces).  Whole records are written,
// so the destinations need no clearing.
template <typename TR>
__global__ void __launch_bounds__(kWalkThreads) k_pack_records(PackSrc S, DevBlock hb, double *a7, TR *recA,
                                                                double *arec64) {
  const int nxy = hb.nx * hb.ny;
  auto ld = [&](int q, int p) -> double {
    const void *a = S.a[q];
    if (!a) return 0.0;
    return S.f32 ? (double)static_cast<const float *>(a)[p] : static_cast<const double *>(a)[p];
  };
  walk_rows(hb, [&](int i, int j, int k, int p, long long c) {
    double v[7];
    v[0] = ld(0, p);
    v[2] = i < hb.nx - 1 ? ld(2, p) : 0.0;
    v[4] = j < hb.ny - 1 ? ld(4, p) : 0.0;
    v[6] = k < hb.nz - 1 ? ld(6, p) : 0.0;
    if (S.sym) {
      v[1] = i > 0 ? ld(2, p - 1) : 0.0;
      v[3] = j > 0 ? ld(4, p - hb.nx) : 0.0;
      v[5] = k > 0 ? ld(6, p - nxy) : 0.0;
    } else {
      v[1] = i > 0 ? ld(1, p) : 0.0;
      v[3] = j > 0 ? ld(3, p) : 0.0;
      v[5] = k > 0 ? ld(5, p) : 0.0;
    }
    double2 *d7 = reinterpret_cast<double2 *>(a7 + c * 8);
    d7[0] = make_double2(v[0], v[1]);
    d7[1] = make_double2(v[2], v[3]);
    d7[2] = make_double2(v[4], v[5]);
    d7[3] = make_double2(v[6], 0.0);
    if (S.sym) {
      const double r4[4] = {v[0], v[2], v[4], v[6]};
      if constexpr (sizeof(TR) == 4) {
        reinterpret_cast<float4 *>(recA)[c] = make_float4((float)r4[0], (float)r4[1], (float)r4[2], (float)r4[3]);
      } else {
        double2 *d = reinterpret_cast<double2 *>(recA + c * 4);
        d[0] = make_double2(r4[0], r4[1]);
        d[1] = make_double2(r4[2], r4[3]);
      }
      if (arec64) {
        double2 *d = reinterpret_cast<double2 *>(arec64 + c * 4);
        d[0] = make_double2(r4[0], r4[1]);
        d[1] = make_double2(r4[2], r4[3]);
      }
    } else {
      if constexpr (sizeof(TR) == 4) {
        float4 *d = reinterpret_cast<float4 *>(recA + c * 8);
        d[0] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
        d[1] = make_float4((float)v[4], (float)v[5], (float)v[6], 0.0f);
      } else {
        double2 *d = reinterpret_cast<double2 *>(recA + c * 8);
        d[0] = make_double2(v[0], v[1]);
        d[1] = make_double2(v[2], v[3]);
        d[2] = make_double2(v[4], v[5]);
        d[3] = make_double2(v[6], 0.0);
      }
      if (arec64) {
        double2 *d = reinterpret_cast<double2 *>(arec64 + c * 8);
        d[0] = make_double2(v[0], v[1]);
        d[1] = make_double2(v[2], v[3]);
        d[2] = make_double2(v[4], v[5]);
        d[3] = make_double2(v[6], 0.0);
      }
    }
  });
}

cudaError_t launch_pack_records(const PackSrc &S, const DevBlock &hb, double *a7, void *recA, int recA_f32,
                                double *arec64, cudaStream_t st) {
  if (recA_f32)
    k_pack_records<float><<<walk_grid(hb), kWalkThreads, 0, st>>>(S, hb, a7, static_cast<float *>(recA), arec64);
  else
    k_pack_records<double><<<walk_grid(hb), kWalkThreads, 0, st>>>(S, hb, a7, static_cast<double *>(recA), arec64);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kWalkThreads) k_to_plan(const double *src, double *dst, DevBlock hb) {
  walk_rows(hb, [&](int, int, int, int p, long long c) { dst[c] = src[p]; });
}

cudaError_t launch_to_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st) {
  k_to_plan<<<walk_grid(hb), kWalkThreads, 0, st>>>(src, dst, hb);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kWalkThreads) k_from_plan(const double *src, double *dst, DevBlock hb) {
  walk_rows(hb, [&](int, int, int, int p, long long c) { dst[p] = src[c]; });
}

cudaError_t launch_from_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st) {
  k_from_plan<<<walk_grid(hb), kWalkThreads, 0, st>>>(src, dst, hb);
  return cudaGetLastError();
}

struct Out7 { double *o[7]; };
template <typename TF>
__global__ void k_export(const TF *recF, const TF *recB, Out7 O, DevBlock hb) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % hb.nx);
    const int j = (int)((p / hb.nx) % hb.ny);
    const int k = (int)(p / ((long long)hb.nx * hb.ny));
    const long long a = plan_cell(hb, i, j, k);
    const TF *f = recF + a * 4;
    const TF *b = recB + a * 4;
    O.o[0][p] = (double)f[REC_LB];
    O.o[1][p] = (double)f[REC_LW];
    O.o[2][p] = (double)f[REC_LS];
    O.o[3][p] = (double)f[REC_RLP];
    O.o[4][p] = (double)b[RECB_UN];
    O.o[5][p] = (double)b[RECB_UE];
    O.o[6][p] = (double)b[RECB_UT];
  }
}

cudaError_t launch_export_factors(const void *recF, const void *recB, int is_f32, double *const out[7],
                                  const DevBlock &hb, cudaStream_t st) {
  Out7 O;
  for (int q = 0; q < 7; ++q) O.o[q] = out[q];
  const int g = util_grid((long long)hb.nx * hb.ny * hb.nz);
  if (is_f32) k_export<float><<<g, 256, 0, st>>>((const float *)recF, (const float *)recB, O, hb);
  else k_export<double><<<g, 256, 0, st>>>((const double *)recF, (const double *)recB, O, hb);
  return cudaGetLastError();
}

// ------------------------------------------------------------ reductions
// Deterministic sum of squares: block q reduces the contiguous chunk q of v
// in a fixed order (strided per thread, fixed shuffle tree, warps in order).
__global__ void k_sumsq_partials(const double *v, long long n, double *partials) {
  __shared__ double red[32];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) s = fma(v[p], v[p], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partials[blockIdx.x] = t;
  }
}

cudaError_t launch_sumsq_partials(const double *v, long long n, double *partials, int nparts,
                                  cudaStream_t st) {
  k_sumsq_partials<<<nparts, 256, 0, st>>>(v, n, partials);
  return cudaGetLastError();
}

// Sum the partials in a fixed order and apply the sequence's stop rule:
// relres(x_n) = sqrt(sum) / ||b||; stop when relres <= rtol or n == max_iters,
// otherwise count the update that the following kernels apply.
__global__ void k_finalize(const double *partials, int n, Ctl *ctl, double *hist, int hist_cap,
                           const int *status, int mode) {
  __shared__ double red[256];
  if (*status != DEV_OK) return;
  if (mode == FIN_RELRES && ctl->done) return;
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += partials[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tot = red[0];
    if (mode == FIN_BNORM) {
      ctl->bnorm = sqrt(tot);
    } else {
      const double scale = ctl->bnorm > 0.0 ? ctl->bnorm : 1.0;
      const double rel = sqrt(tot) / scale;
      ctl->relres = rel;
      if (ctl->nhist < hist_cap) hist[ctl->nhist] = rel;
      ctl->nhist += 1;
      if (rel <= ctl->rtol || ctl->iter >= ctl->max_iters) ctl->done = 1;
      else ctl->iter += 1;
    }
  }
}

cudaError_t launch_finalize(const double *partials, int n, Ctl *ctl, double *hist, int hist_cap,
                            const int *status, int mode, cudaStream_t st) {
  k_finalize<<<1, 256, 0, st>>>(partials, n, ctl, hist, hist_cap, status, mode);
  return cudaGetLastError();
}

// Start a sequence: counters and flags reset, both epoch slots moved past
// every tag used so far (so no stale face word can match).
// ------------------------------------------------------------ interfaces
__global__ void k_halo_coefs(const HaloSrc *src, int nsrc, HaloEntry *ent, int coef_f32) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nsrc; q += gridDim.x * blockDim.x) {
    const HaloSrc s = src[q];
    ent[s.e].c[s.slot] = coef_f32 ? (double)((const float *)s.src)[s.p] : ((const double *)s.src)[s.p];
  }
}

cudaError_t launch_halo_coefs(const HaloSrc *src, int nsrc, HaloEntry *ent, int coef_f32, cudaStream_t st) {
  k_halo_coefs<<<util_grid(nsrc), 256, 0, st>>>(src, nsrc, ent, coef_f32);
  return cudaGetLastError();
}

// Lagged interface terms of the coupled residual, in interface order:
// beff = b - c0 x_nb0 (- c1 x_nb1).  Skipped once the stop rule has fired.
__global__ void k_halo(const HaloEntry *ent, int nent, const double *b, const double *x, double *beff,
                       const Ctl *ctl) {
  if (ctl->done) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nent; q += gridDim.x * blockDim.x) {
    const HaloEntry e = ent[q];
    double v = b[e.cell] - e.c[0] * x[e.nb[0]];
    if (e.nb[1] >= 0) v -= e.c[1] * x[e.nb[1]];
    beff[e.cell] = v;
  }
}

cudaError_t launch_halo(const HaloEntry *ent, int nent, const double *b, const double *x, double *beff,
                        const Ctl *ctl, cudaStream_t st) {
  k_halo<<<util_grid(nent), 256, 0, st>>>(ent, nent, b, x, beff, ctl);
  return cudaGetLastError();
}

// Interface terms of the refinement's inner correction system (the blocks
// exchange the correction d after every inner iteration): the FP32
// right-hand side of an interface cell becomes
//   r32[cell] = r0 - c0 d[nb0] (- c1 d[nb1]),
// each product and difference rounded to float in that order (c: the
// coupling entries rounded to float; r0: the cell's value from the outer
// FP64 residual, saved by the first call of a correction and restored from
// the copy afterwards).  Skipped once the stop rule has fired.
__global__ void k_halo32(const HaloEntry *ent, int nent, float *r32, const float *d, float *save, int first,
                         const Ctl *ctl) {
  if (ctl->done) return;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nent; q += gridDim.x * blockDim.x) {
    const HaloEntry e = ent[q];
    float r0;
    if (first) {
      r0 = r32[e.cell];
      save[q] = r0;
    } else {
      r0 = save[q];
    }
    float v = __fsub_rn(r0, __fmul_rn((float)e.c[0], d[e.nb[0]]));
    if (e.nb[1] >= 0) v = __fsub_rn(v, __fmul_rn((float)e.c[1], d[e.nb[1]]));
    r32[e.cell] = v;
  }
}

cudaError_t launch_halo32(const HaloEntry *ent, int nent, float *r32, const float *d, float *save, bool first,
                          const Ctl *ctl, cudaStream_t st) {
  k_halo32<<<util_grid(nent), 256, 0, st>>>(ent, nent, r32, d, save, first ? 1 : 0, ctl);
  return cudaGetLastError();
}

__global__ void k_cast_f64_f32(const double *src, float *dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (float)src[q];
}
__global__ void k_cast_f32_f64(const float *src, double *dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (double)src[q];
}
cudaError_t launch_cast_f64_f32(const double *src, float *dst, long long n, cudaStream_t st) {
  k_cast_f64_f32<<<util_grid(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
cudaError_t launch_cast_f32_f64(const float *src, double *dst, long long n, cudaStream_t st) {
  k_cast_f32_f64<<<util_grid(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// The refinement's update x64 += (double) d (d: the FP32 correction of the
// last inner iteration), four cells per thread with 16-byte accesses.
__global__ void k_update64(const float *d, double *x64, long long n, const Ctl *ctl) {
  if (ctl->done) return;
  const long long n4 = n / 4;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
    const float4 dv = reinterpret_cast<const float4 *>(d)[q];
    double2 *xp = reinterpret_cast<double2 *>(x64) + 2 * q;
    double2 a = xp[0], b = xp[1];
    a.x += (double)dv.x;
    a.y += (double)dv.y;
    b.x += (double)dv.z;
    b.y += (double)dv.w;
    xp[0] = a;
    xp[1] = b;
  }
  for (long long q = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += stride)
    x64[q] += (double)d[q];
}
cudaError_t launch_update64(const float *d, double *x64, long long n, const Ctl *ctl, cudaStream_t st) {
  k_update64<<<util_grid((n + 3) / 4), 256, 0, st>>>(d, x64, n, ctl);
  return cudaGetLastError();
}

__global__ void k_set_ctl(Ctl *ctl, double rtol, int max_iters) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->iter = 0;
    ctl->done = 0;
    ctl->nhist = 0;
    ctl->max_iters = max_iters;
    ctl->rtol = rtol;
    ctl->relres = -1.0;
    const unsigned e = (ctl->epochs[0] > ctl->epochs[1] ? ctl->epochs[0] : ctl->epochs[1]) + 2u;
    ctl->epochs[0] = e;
    ctl->epochs[1] = e;
  }
}

cudaError_t launch_set_ctl(Ctl *ctl, double rtol, int max_iters, cudaStream_t st) {
  k_set_ctl<<<1, 32, 0, st>>>(ctl, rtol, max_iters);
  return cudaGetLastError();
}

}  // namespace sipk
