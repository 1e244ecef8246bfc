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
//     g_f = (g_P + g_N) / 2, delta_f = (w_P + w_N) / 2 (widths along the
//     face normal), S_f = face area, A_N(P) = -rho_f g_f S_f / delta_f;
//   walls: no coefficient; the k = 0 face, when Dirichlet (p' = 0 beyond it),
//     adds rho_P g_P S_z / (dz_0 / 2) to AP;
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
// that the L1/L2 caches serve.  Memory-bound: per cell 16 B of cell data, 24 B
// of face velocities (each face array holds about one value per cell) and
// 40 B (symmetric storage: AP, AE, AN, AT, b) or 64 B of outputs.
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_internal.h"

namespace sipk {

namespace {

__device__ __forceinline__ double face_coef(double rp, double rn, double gp, double gn, double wp, double wn,
                                            double S) {
  const double rf = __dmul_rn(__dadd_rn(rp, rn), 0.5);
  const double gf = __dmul_rn(__dadd_rn(gp, gn), 0.5);
  const double delta = __dmul_rn(__dadd_rn(wp, wn), 0.5);
  return -(__dmul_rn(__dmul_rn(rf, gf), S) / delta);
}

__global__ void __launch_bounds__(256) k_assemble_pcorr(PcorrArgs a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long n = (long long)nx * ny * nz, nxy = (long long)nx * ny;
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
    if (i > 0) {
      cw = face_coef(rp, a.rho[p - 1], gp, a.g[p - 1], dxi, a.dx[i - 1], Sx);
      rw = __dmul_rn(__dadd_rn(rp, a.rho[p - 1]), 0.5);
    }
    if (i < nx - 1) {
      ce = face_coef(rp, a.rho[p + 1], gp, a.g[p + 1], dxi, a.dx[i + 1], Sx);
      re = __dmul_rn(__dadd_rn(rp, a.rho[p + 1]), 0.5);
    }
    if (j > 0) {
      cs = face_coef(rp, a.rho[p - nx], gp, a.g[p - nx], dyj, a.dy[j - 1], Sy);
      rs = __dmul_rn(__dadd_rn(rp, a.rho[p - nx]), 0.5);
    }
    if (j < ny - 1) {
      cn = face_coef(rp, a.rho[p + nx], gp, a.g[p + nx], dyj, a.dy[j + 1], Sy);
      rn = __dmul_rn(__dadd_rn(rp, a.rho[p + nx]), 0.5);
    }
    if (k > 0) {
      cb = face_coef(rp, a.rho[p - nxy], gp, a.g[p - nxy], dzk, a.dz[k - 1], Sz);
      rb = __dmul_rn(__dadd_rn(rp, a.rho[p - nxy]), 0.5);
    }
    if (k < nz - 1) {
      ct = face_coef(rp, a.rho[p + nxy], gp, a.g[p + nxy], dzk, a.dz[k + 1], Sz);
      rt = __dmul_rn(__dadd_rn(rp, a.rho[p + nxy]), 0.5);
    }
    double cB = 0.0;
    if (k == 0 && a.dirichlet_bottom) cB = __dmul_rn(__dmul_rn(rp, gp), Sz) / __dmul_rn(a.dz[0], 0.5);
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
  k_assemble_pcorr<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sipk
