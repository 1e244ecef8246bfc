// sip_util.cu -- layout conversion, deterministic reductions and sequence
// control kernels of libsip.so, plus the kernel registry's size rules.
#include <cmath>
#include <cstdint>

#include "sip_internal.h"
#include "sip_kernels.h"

namespace sipk {

// ------------------------------------------------------------ registry
const void *kernel_ptr(int kind, int stages) {
  const void *p = kernel_ptr_64(kind, stages);
  return p ? p : kernel_ptr_32(kind, stages);
}

bool kernel_is_ticketed(int kind) {
  return !(kind == K_RES64 || kind == K_RES64S || kind == K_RES32A || kind == K_RES32AS);
}

static size_t a16(size_t b) { return (b + 15) & ~(size_t)15; }

// stage ring + exchange buffer (+ face ring), laid out as in sip_sweeps.cuh
static size_t sweep_bytes(size_t r, size_t nv, size_t nt, size_t ne, size_t ec, size_t eb, size_t fs, size_t w) {
  return a16(r * nv * nt * eb + 2 * ne * ec * eb) + r * fs * w * 8;
}

size_t kernel_smem(int kind, int R, int NT, int EC, int FS) {
  const size_t nt = (size_t)NT, ec = (size_t)EC, r = (size_t)R, fs = (size_t)FS;
  switch (kind) {
    case K_FACTOR: return sweep_bytes(r, 7, nt, 3, ec, 8, fs, 6);
    case K_FWD64: return sweep_bytes(r, 15, nt, 3, ec, 8, fs, 2);
    case K_FWD64S: return sweep_bytes(r, 14, nt, 5, ec, 8, fs, 2);
    case K_BWD64: return sweep_bytes(r, 5, nt, 1, ec, 8, fs, 2);
    case K_FWD32:
    case K_FWD32N: return sweep_bytes(r, 15, nt, 3, ec, 4, fs, 2);
    case K_FWD32S:
    case K_FWD32SN: return sweep_bytes(r, 14, nt, 5, ec, 4, fs, 2);
    case K_FWD32Z: return sweep_bytes(r, 5, nt, 1, ec, 4, fs, 2);
    case K_BWD32: return sweep_bytes(r, 5, nt, 1, ec, 4, fs, 2);
    case K_BWD32Z: return sweep_bytes(r, 4, nt, 1, ec, 4, fs, 2);
    case K_BWD32U: return sweep_bytes(r, 7, nt, 1, ec, 4, fs, 2);
    case K_BWD32ZU: return sweep_bytes(r, 6, nt, 1, ec, 4, fs, 2);
    case K_RES64: return r * 4 * nt * 8 + a16(r * 7 * nt * 8) + 2 * 2 * ec * 8;
    case K_RES64S: return r * 4 * nt * 8 + a16(r * 6 * nt * 8) + 2 * 4 * ec * 8;
    case K_RES32A: return r * 4 * nt * 8 + a16(r * 7 * nt * 4) + 2 * 2 * ec * 8;
    case K_RES32AS: return r * 4 * nt * 8 + a16(r * 6 * nt * 4) + 2 * 4 * ec * 8;
    default: return 0;
  }
}

// ------------------------------------------------------------ layout
// natural index p = i + nx*(j + ny*k)  ->  plan cell cell0 + rbT[k][i+j+k] + j.
// zero_face: 0 keep; 1..6 zero the coefficient on the face i=0, i=nx-1,
// j=0, j=ny-1, k=0, k=nz-1 (an entry that points out of the block).
// shift_axis: 0 read src[p]; 1/2/3 read src at the lower neighbour along
// i/j/k (0 on the lower face): builds AW/AS/AB of a symmetric matrix from AE/AN/AT.
template <typename TO>
__global__ void k_to_plan(const void *src, int src_is_f32, TO *dst, DevBlock hb, int zero_face,
                          int shift_axis) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % hb.nx);
    const int j = (int)((p / hb.nx) % hb.ny);
    const int k = (int)(p / ((long long)hb.nx * hb.ny));
    bool zero = (zero_face == 1 && i == 0) || (zero_face == 2 && i == hb.nx - 1) ||
                (zero_face == 3 && j == 0) || (zero_face == 4 && j == hb.ny - 1) ||
                (zero_face == 5 && k == 0) || (zero_face == 6 && k == hb.nz - 1);
    long long q = p;
    if (shift_axis == 1) { if (i == 0) zero = true; else q = p - 1; }
    if (shift_axis == 2) { if (j == 0) zero = true; else q = p - hb.nx; }
    if (shift_axis == 3) { if (k == 0) zero = true; else q = p - (long long)hb.nx * hb.ny; }
    double v = 0.0;
    if (!zero) v = src_is_f32 ? (double)((const float *)src)[q] : ((const double *)src)[q];
    dst[hb.cell0 + hb.rbT[(long long)k * hb.nplanes + i + j + k] + j] = (TO)v;
  }
}

template <typename TO>
static cudaError_t to_plan(const void *src, int src_is_f32, TO *dst, const DevBlock &hb, int zf, int sh,
                           cudaStream_t st) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  k_to_plan<TO><<<grid, 256, 0, st>>>(src, src_is_f32, dst, hb, zf, sh);
  return cudaGetLastError();
}

cudaError_t launch_to_plan_f64(const void *src, int src_is_f32, double *dst, const DevBlock &hb, int zf,
                               int sh, cudaStream_t st) {
  return to_plan<double>(src, src_is_f32, dst, hb, zf, sh, st);
}
cudaError_t launch_to_plan_f32(const void *src, int src_is_f32, float *dst, const DevBlock &hb, int zf,
                               int sh, cudaStream_t st) {
  return to_plan<float>(src, src_is_f32, dst, hb, zf, sh, st);
}

__global__ void k_from_plan(const double *src, double *dst, DevBlock hb) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % hb.nx);
    const int j = (int)((p / hb.nx) % hb.ny);
    const int k = (int)(p / ((long long)hb.nx * hb.ny));
    dst[p] = src[hb.cell0 + hb.rbT[(long long)k * hb.nplanes + i + j + k] + j];
  }
}

cudaError_t launch_from_plan_f64(const double *src, double *dst, const DevBlock &hb, cudaStream_t st) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  k_from_plan<<<grid, 256, 0, st>>>(src, dst, hb);
  return cudaGetLastError();
}

struct Ptr7 { const double *f[7]; double *o[7]; };
__global__ void k_export7(Ptr7 P, DevBlock hb) {
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % hb.nx);
    const int j = (int)((p / hb.nx) % hb.ny);
    const int k = (int)(p / ((long long)hb.nx * hb.ny));
    const long long a = hb.cell0 + hb.rbT[(long long)k * hb.nplanes + i + j + k] + j;
#pragma unroll
    for (int q = 0; q < 7; ++q) P.o[q][p] = P.f[q][a];
  }
}

cudaError_t launch_plan_to_natural_factors(const double *const f[7], double *const out[7], const DevBlock &hb,
                                           cudaStream_t st) {
  Ptr7 P;
  for (int q = 0; q < 7; ++q) { P.f[q] = f[q]; P.o[q] = out[q]; }
  const long long n = (long long)hb.nx * hb.ny * hb.nz;
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  k_export7<<<grid, 256, 0, st>>>(P, hb);
  return cudaGetLastError();
}

__global__ void k_f64_to_f32(const double *src, float *dst, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    dst[p] = (float)src[p];
}
cudaError_t launch_f64_to_f32(const double *src, float *dst, long long n, cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  k_f64_to_f32<<<grid, 256, 0, st>>>(src, dst, n);
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
