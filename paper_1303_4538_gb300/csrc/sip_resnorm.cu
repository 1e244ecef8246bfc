// sip_resnorm.cu -- residual norm of one block in its natural layout:
// ||b - A x||_2 and ||b||_2 (the residual of resforward3d, arXiv:1303.4538
// Sec. 4.1, evaluated directly on the caller's arrays instead of a plan's
// plane layout).  Used to check a returned solution independently of the
// solver's own residual kernels.
//
// Two launches, both with a fixed summation order (bitwise reproducible):
//   1. one CTA per chunk of kResChunk consecutive cells writes the pair
//      (sum r^2, sum b^2) of its chunk into scratch[2 * chunk + {0, 1}];
//   2. one CTA sums the pairs in chunk order and writes the two norms.
// The chunking depends only on N, so every launch configuration and every
// scratch placement gives the same bits.  Memory-bound: per cell the seven
// coefficients (four if symmetric), b and x are read once; x neighbours come
// from L1/L2.
#include <cuda_runtime.h>

#include "sip_internal.h"

namespace sipk {

namespace {

constexpr int kResThreads = 256;

template <typename TA, bool SYM>
__global__ void __launch_bounds__(kResThreads) k_resnorm_part(NatBlock nb, double *scratch) {
  __shared__ double red[2][kResThreads / 32];
  const long long n = (long long)nb.nx * nb.ny * nb.nz;
  const long long nxy = (long long)nb.nx * nb.ny;
  const TA *ap = (const TA *)nb.a[0], *aw = (const TA *)nb.a[1], *ae = (const TA *)nb.a[2];
  const TA *as = (const TA *)nb.a[3], *an = (const TA *)nb.a[4], *ab = (const TA *)nb.a[5];
  const TA *at = (const TA *)nb.a[6];
  const long long lo = (long long)blockIdx.x * kResChunk;
  const long long hi = lo + kResChunk < n ? lo + kResChunk : n;
  double rr = 0.0, bb = 0.0;
  for (long long p = lo + threadIdx.x; p < hi; p += kResThreads) {
    const int i = (int)(p % nb.nx);
    const int j = (int)((p / nb.nx) % nb.ny);
    const int k = (int)(p / nxy);
    const double xp = nb.x[p];
    double ax = (double)ap[p] * xp;
    if (i + 1 < nb.nx) ax = fma((double)ae[p], nb.x[p + 1], ax);
    if (j + 1 < nb.ny) ax = fma((double)an[p], nb.x[p + nb.nx], ax);
    if (k + 1 < nb.nz) ax = fma((double)at[p], nb.x[p + nxy], ax);
    if (SYM) {  // lower entries are the neighbours' upper entries
      if (i > 0) ax = fma((double)ae[p - 1], nb.x[p - 1], ax);
      if (j > 0) ax = fma((double)an[p - nb.nx], nb.x[p - nb.nx], ax);
      if (k > 0) ax = fma((double)at[p - nxy], nb.x[p - nxy], ax);
    } else {
      if (i > 0) ax = fma((double)aw[p], nb.x[p - 1], ax);
      if (j > 0) ax = fma((double)as[p], nb.x[p - nb.nx], ax);
      if (k > 0) ax = fma((double)ab[p], nb.x[p - nxy], ax);
    }
    const double bp = nb.b[p];
    const double r = bp - ax;
    rr = fma(r, r, rr);
    bb = fma(bp, bp, bb);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < kResThreads / 32; ++q) {
      s0 += red[0][q];
      s1 += red[1][q];
    }
    scratch[2 * (long long)blockIdx.x] = s0;
    scratch[2 * (long long)blockIdx.x + 1] = s1;
  }
}

__global__ void __launch_bounds__(kResThreads) k_resnorm_fin(const double *scratch, int nparts, double *out2) {
  __shared__ double red[2][kResThreads];
  double s0 = 0.0, s1 = 0.0;
  for (int q = threadIdx.x; q < nparts; q += kResThreads) {
    s0 += scratch[2 * q];
    s1 += scratch[2 * q + 1];
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = kResThreads >> 1; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = sqrt(red[0][0]);
    out2[1] = sqrt(red[1][0]);
  }
}

}  // namespace

long long resnorm_parts(const NatBlock &nb) {
  const long long n = (long long)nb.nx * nb.ny * nb.nz;
  return (n + kResChunk - 1) / kResChunk;
}

cudaError_t launch_resnorm(const NatBlock &nb, double *scratch, double *out2, cudaStream_t st) {
  const long long np = resnorm_parts(nb);
  if (np < 1 || np > (1ll << 30)) return cudaErrorInvalidValue;
  const bool f32 = nb.coef_f32 != 0, sym = nb.symmetric != 0;
  if (f32 && sym) k_resnorm_part<float, true><<<(unsigned)np, kResThreads, 0, st>>>(nb, scratch);
  else if (f32) k_resnorm_part<float, false><<<(unsigned)np, kResThreads, 0, st>>>(nb, scratch);
  else if (sym) k_resnorm_part<double, true><<<(unsigned)np, kResThreads, 0, st>>>(nb, scratch);
  else k_resnorm_part<double, false><<<(unsigned)np, kResThreads, 0, st>>>(nb, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resnorm_fin<<<1, kResThreads, 0, st>>>(scratch, (int)np, out2);
  return cudaGetLastError();
}

}  // namespace sipk
