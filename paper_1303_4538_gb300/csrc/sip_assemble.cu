// sip_assemble.cu -- pressure-correction coefficient assembly on the device
// (the routine celp2 of arXiv:1303.4538, Sec. 3.1, Table 1; its system is the
// symmetric pressure-correction system of Sec. 4.1), so that SIP's input is
// produced where it is consumed, with no host round trip.
//
// The paper does not print celp2's discretisation.  The geometry this library
// states: one block of nx x ny x nz hexahedral cells on a rectilinear grid
// (cell widths dx[i], dy[j], dz[k]); per cell a density rho and the momentum
// equation's V / a_P (g); face-normal velocities u* on every face.  The
// SIMPLE-type equation -div(rho g grad p') = -div(rho u*) in finite volumes:
//   interior face f between P and N:  rho_f = (rho_P + rho_N) / 2,
//     g_f = (g_P + g_N) / 2, rdelta_f = 1 / ((w_P + w_N) / 2) (the reciprocal
//     distance of the cell centres, w the widths along the face normal),
//     S_f = face area, A_N(P) = -((rho_f g_f) S_f) rdelta_f;
//   walls: no coefficient; the k = 0 face, when Dirichlet (p' = 0 beyond it),
//     adds ((rho_P g_P) S_z) (1 / (dz_0 / 2)) to AP;
//   AP = -(sum of the six off-diagonal entries) + the Dirichlet term;
//   b = -(F_e - F_w + F_n - F_s + F_t - F_b), F_f = rho_f u*_f S_f
//     (boundary faces: rho_f = rho_P), the negative net mass outflow.
// Every operation is an explicitly rounded double operation in that fixed
// order (no contraction into fused multiply-adds), so both cells of a face
// compute its entry bit for bit alike (the matrix is exactly symmetric) and
// the results equal a plain sequential evaluation of the same formulas.
//
// Work decomposition: one thread per cell, consecutive threads along i, so
// the per-cell arrays and the x-face velocities are read and the outputs
// written as contiguous runs; the neighbour values along j and k are reuses
// that the L1/L2 caches serve.  The reciprocal face distances depend on one
// axis each: every CTA first fills a shared-memory table of the nx-1 + ny-1 +
// nz-1 values (when it fits; otherwise each cell divides inline, with the
// same result), so the cells do no division.  What bounds the kernel is the
// FP64 pipe: per cell 6 faces x (2 adds, 5 multiplies) for the coefficients
// and face densities, 3 face areas, 6 adds for AP and 12 multiplies + 5 adds
// for b: 68 FP64 operations, against 16 B of cell data, ~24 B of face
// velocities and 40 B (symmetric storage) or 64 B of outputs.
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_internal.h"

namespace sipk {

namespace {

__device__ __forceinline__ double rdist(double wp, double wn) { return 1.0 / __dmul_rn(__dadd_rn(wp, wn), 0.5); }

__device__ __forceinline__ double face_coef(double rf, double gp, double gn, double S, double rd) {
  const double gf = __dmul_rn(__dadd_rn(gp, gn), 0.5);
  return -__dmul_rn(__dmul_rn(__dmul_rn(rf, gf), S), rd);
}

// TAB: reciprocal face distances from the CTA's shared-memory table
// (x faces at 0 .. nx-2, y faces at nx-1 .., z faces at nx-1 + ny-1 ..)
template <bool TAB>
__global__ void __launch_bounds__(256) k_assemble_pcorr(PcorrArgs a) {
  extern __shared__ double s_rd[];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long n = (long long)nx * ny * nz, nxy = (long long)nx * ny;
  const int oy = nx - 1, oz = nx - 1 + ny - 1;
  if constexpr (TAB) {
    for (int q = threadIdx.x; q < nx - 1; q += blockDim.x) s_rd[q] = rdist(a.dx[q], a.dx[q + 1]);
    for (int q = threadIdx.x; q < ny - 1; q += blockDim.x) s_rd[oy + q] = rdist(a.dy[q], a.dy[q + 1]);
    for (int q = threadIdx.x; q < nz - 1; q += blockDim.x) s_rd[oz + q] = rdist(a.dz[q], a.dz[q + 1]);
    __syncthreads();
  }
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(p / nxy);
    const long long r = p - (long long)k * nxy;
    const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
    const double dxi = a.dx[i], dyj = a.dy[j], dzk = a.dz[k];
    const double Sx = __dmul_rn(dyj, dzk), Sy = __dmul_rn(dxi, dzk), Sz = __dmul_rn(dxi, dyj);
    const double rp = a.rho[p], gp = a.g[p];
    double cw = 0.0, ce = 0.0, cs = 0.0, cn = 0.0, cb = 0.0, ct = 0.0;
    double rw = rp, re = rp, rs = rp, rn = rp, rb = rp, rt = rp;  // face densities of the fluxes
    // reciprocal distance of the face between index q and q + 1 along an axis
    auto rdx = [&](int q) { return TAB ? s_rd[q] : rdist(a.dx[q], a.dx[q + 1]); };
    auto rdy = [&](int q) { return TAB ? s_rd[oy + q] : rdist(a.dy[q], a.dy[q + 1]); };
    auto rdz = [&](int q) { return TAB ? s_rd[oz + q] : rdist(a.dz[q], a.dz[q + 1]); };
    if (i > 0) {
      rw = __dmul_rn(__dadd_rn(rp, a.rho[p - 1]), 0.5);
      cw = face_coef(rw, gp, a.g[p - 1], Sx, rdx(i - 1));
    }
    if (i < nx - 1) {
      re = __dmul_rn(__dadd_rn(rp, a.rho[p + 1]), 0.5);
      ce = face_coef(re, gp, a.g[p + 1], Sx, rdx(i));
    }
    if (j > 0) {
      rs = __dmul_rn(__dadd_rn(rp, a.rho[p - nx]), 0.5);
      cs = face_coef(rs, gp, a.g[p - nx], Sy, rdy(j - 1));
    }
    if (j < ny - 1) {
      rn = __dmul_rn(__dadd_rn(rp, a.rho[p + nx]), 0.5);
      cn = face_coef(rn, gp, a.g[p + nx], Sy, rdy(j));
    }
    if (k > 0) {
      rb = __dmul_rn(__dadd_rn(rp, a.rho[p - nxy]), 0.5);
      cb = face_coef(rb, gp, a.g[p - nxy], Sz, rdz(k - 1));
    }
    if (k < nz - 1) {
      rt = __dmul_rn(__dadd_rn(rp, a.rho[p + nxy]), 0.5);
      ct = face_coef(rt, gp, a.g[p + nxy], Sz, rdz(k));
    }
    double cB = 0.0;
    if (k == 0 && a.dirichlet_bottom) cB = __dmul_rn(__dmul_rn(__dmul_rn(rp, gp), Sz), 1.0 / __dmul_rn(a.dz[0], 0.5));
    double ap = __dadd_rn(-cw, -ce);
    ap = __dadd_rn(ap, -cs);
    ap = __dadd_rn(ap, -cn);
    ap = __dadd_rn(ap, -cb);
    ap = __dadd_rn(ap, -ct);
    ap = __dadd_rn(ap, cB);
    // face velocities: x faces (nx + 1 per row), y faces (ny + 1 rows per k), z faces (nz + 1 layers)
    const long long fx = ((long long)k * ny + j) * (nx + 1) + i;
    const long long fy = ((long long)k * (ny + 1) + j) * nx + i;
    const double uw = a.ux[fx], ue = a.ux[fx + 1];
    const double us = a.uy[fy], un = a.uy[fy + nx];
    const double ub = a.uz[p], ut = a.uz[p + nxy];
    const double Fw = __dmul_rn(__dmul_rn(rw, uw), Sx), Fe = __dmul_rn(__dmul_rn(re, ue), Sx);
    const double Fs = __dmul_rn(__dmul_rn(rs, us), Sy), Fn = __dmul_rn(__dmul_rn(rn, un), Sy);
    const double Fb = __dmul_rn(__dmul_rn(rb, ub), Sz), Ft = __dmul_rn(__dmul_rn(rt, ut), Sz);
    double net = __dadd_rn(Fe, -Fw);
    net = __dadd_rn(net, Fn);
    net = __dadd_rn(net, -Fs);
    net = __dadd_rn(net, Ft);
    net = __dadd_rn(net, -Fb);
    a.ap[p] = ap;
    a.ae[p] = ce;
    a.an[p] = cn;
    a.at[p] = ct;
    if (a.aw) a.aw[p] = cw;
    if (a.as) a.as[p] = cs;
    if (a.ab) a.ab[p] = cb;
    a.b[p] = -net;
  }
}

}  // namespace

cudaError_t launch_assemble_pcorr(const PcorrArgs &a, int grid, cudaStream_t st) {
  const long long tab = (long long)a.nx - 1 + a.ny - 1 + a.nz - 1;
  if (tab * 8 <= 48 * 1024) k_assemble_pcorr<true><<<grid, 256, (size_t)tab * 8, st>>>(a);
  else k_assemble_pcorr<false><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sipk
