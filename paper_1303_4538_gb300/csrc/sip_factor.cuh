// sip_factor.cuh -- Stone's factorisation (lu3d) as a wavefront over the
// plane layout, on the tile machinery of sip_sweeps.cuh (column tiles, staged
// cp.async ring, epoch-tagged J/K face records, bounded waits).  Included
// after sip_sweeps.cuh by the per-precision kernel units.
#pragma once

#include "sip_sweeps.cuh"

namespace sipk {

// ============================================================== factorisation
// Stone's factorisation, per cell after W, S, B (lu3d):
//   LB = AB / (1 + a (UN_B + UE_B)),  LW = AW / (1 + a (UN_W + UT_W)),
//   LS = AS / (1 + a (UE_S + UT_S)),
//   P1 = a (LB UN_B + LW UN_W),  P2 = a (LB UE_B + LS UE_S),  P3 = a (LW UT_W + LS UT_S),
//   LP = AP + P1 + P2 + P3 - LB UT_B - LW UE_W - LS UN_S,
//   UN = (AN - P1) / LP,  UE = (AE - P2) / LP,  UT = (AT - P3) / LP
// (each group of three quotients takes one FP64 division: LB, LW, LS through
// 1/(dB dW dS), the U entries through 1/LP; FP64 throughput bounds the steps).
// Arithmetic in FP64; stored (as TF) into the L record [LB LW LS 1/LP] and
// the U record [UE UN UT 0].  Faces carry (UN, UE, UT): 48 bytes.
// IEEE-754 binary64 tests on the exponent field with integer instructions
// (they keep the FP64 pipe, which bounds this kernel, for the arithmetic):
// finite: exponent field not all ones; in range: |x| within [2^-930, 2^930)
__device__ __forceinline__ bool finite64(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool midrange64(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;  // biased exponent
  return e > 1023 - 930 && e < 1023 + 930;
}

template <typename TF, int Q, int R>
__global__ void __launch_bounds__(512) k_factor(FacParams<TF> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim, s_blk;
  constexpr int W = 6;
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  if (threadIdx.x == 0) s_blk = -1;
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const SweepLayout L = fac_layout(Q, R, NT, c.tab_ints);
  int *sPO = reinterpret_cast<int *>(smem_raw);
  unsigned char *stage = smem_raw + L.tab;
  double *exB = reinterpret_cast<double *>(stage + (size_t)R * L.step);  // [2][3][NW][32]
  uint64_t *fst = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(exB) + L.exch);
  const int FS = L.fs;
  bool abort = false;

  for (;;) {
    const int m = claim_tile(c, &s_claim);
    if (m >= c.ntiles) break;
    const Tile tl = c.tiles[m];
    const DevBlock B = c.blocks[tl.blk];
    unsigned long long *tr = c.trace ? c.trace + (size_t)tl.gtile * kTraceWords : nullptr;
    load_tables(B, tl.blk, sPO, &s_blk);
    const int *sF = sPO + B.nplanes;
    const Geo<Q> g(B, tl);
    const int NW = g.NW, lane = g.lane, w = g.w;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *upJ = g.hasS ? tile_faces(c, B, tl.gtile - 1) : nullptr;
    uint64_t *upK = g.hasB ? tile_faces(c, B, tl.gtile - B.nTJ) : nullptr;
    {
      const int lead = min(R + 1, B.nx - 1);
      slack_gate<W>(upJ ? faceJ(upJ, B, lead + kTJ - 1, 0, W) : nullptr,
                    upK ? faceK(upK, B, lead + g.TK - 1, 0, W) : nullptr, expect, c, abort, tr);
    }
    auto rb = [&](int s, int k) { return plane_row_base(sPO, sF, B.mmax, B.nx, s, k); };

    auto issue = [&](int tt) {
      if (tt < g.nsteps) {
        const int s = g.s0 + tt;
        unsigned char *st = stage + (size_t)(tt % R) * L.step;
        uint64_t *fs = fst + (size_t)(tt % R) * FS * W;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int i = g.i(tt, q);
          const bool v = g.col(B, q) && i >= 0 && i < B.nx;
          const long long a = v ? B.cell0 + rb(s, g.k(q)) + g.j : 0;
          unsigned char *d = st + ((size_t)q * NT + tid) * 64;
          const unsigned char *src = reinterpret_cast<const unsigned char *>(P.a7 + a * 8);
#pragma unroll
          for (int z = 0; z < 4; ++z) cp_async_16_l2(d + 16 * z, src + 16 * z, v);
          if (lane == 0 && g.hasS && v) rec_prefetch<W>(fs + g.dk(q) * W, faceJ(upJ, B, tt + kTJ - 1, g.dk(q), W));
          if (q == 0 && g.eB && g.hasB && v)
            rec_prefetch<W>(fs + (g.TK + lane) * W, faceK(upK, B, tt + g.TK - 1, lane, W));
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int tt = 0; tt < R - 1; ++tt) issue(tt);

    double unW[Q], ueW[Q], utW[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) unW[q] = ueW[q] = utW[q] = 0.0;
    const double al = P.alpha;
    for (int t = 0; t < g.nsteps; ++t) {
      issue(t + R - 1);
      cp_async_wait<R - 1>();
      const unsigned char *st = stage + (size_t)(t % R) * L.step;
      const uint64_t *fs = fst + (size_t)(t % R) * FS * W;
      const int buf = t & 1;
      double *E = exB + (size_t)buf * 3 * NW * 32;
      E[(0 * NW + w) * 32 + lane] = unW[Q - 1];
      E[(1 * NW + w) * 32 + lane] = ueW[Q - 1];
      E[(2 * NW + w) * 32 + lane] = utW[Q - 1];
      double hK[3] = {0, 0, 0};
      if (g.eB) {
        const int i0 = g.i(t, 0);
        if (g.hasB && g.col(B, 0) && i0 >= 0 && i0 < B.nx) {
          uint64_t wv[W];
          rec_take<W>(fs + (g.TK + lane) * W, faceK(upK, B, t + g.TK - 1, lane, W), expect, wv, c, abort, tr);
          hK[0] = Face<double>::get(wv);
          hK[1] = Face<double>::get(wv + 2);
          hK[2] = Face<double>::get(wv + 4);
        }
      }
      __syncwarp();  // the face wait above diverges the warp: reconverge before the CTA barrier
      __syncthreads();
      double nUN[Q], nUE[Q], nUT[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int i = g.i(t, q);
        const bool act = g.col(B, q) && i >= 0 && i < B.nx;
        const double *a = reinterpret_cast<const double *>(st + ((size_t)q * NT + tid) * 64);
        const double ap = a[0], aw = a[1], ae = a[2], as = a[3], an = a[4], ab = a[5], at = a[6];
        // S neighbour (lane - 1, same row, previous step) or the J face
        double unS = shfl_up1(unW[q]), ueS = shfl_up1(ueW[q]), utS = shfl_up1(utW[q]);
        if (lane == 0) {
          unS = ueS = utS = 0.0;
          if (g.hasS && act) {
            uint64_t wv[W];
            rec_take<W>(fs + g.dk(q) * W, faceJ(upJ, B, t + kTJ - 1, g.dk(q), W), expect, wv, c, abort, tr);
            unS = Face<double>::get(wv);
            ueS = Face<double>::get(wv + 2);
            utS = Face<double>::get(wv + 4);
          }
        }
        // B neighbour (row q - 1 of this thread, the previous warp, or the K face)
        double unB, ueB, utB;
        if (q > 0) {
          unB = unW[q > 0 ? q - 1 : 0];
          ueB = ueW[q > 0 ? q - 1 : 0];
          utB = utW[q > 0 ? q - 1 : 0];
        } else if (w > 0) {
          const double *Ep = exB + (size_t)buf * 3 * NW * 32;
          unB = Ep[(0 * NW + w - 1) * 32 + lane];
          ueB = Ep[(1 * NW + w - 1) * 32 + lane];
          utB = Ep[(2 * NW + w - 1) * 32 + lane];
        } else {
          unB = hK[0];
          ueB = hK[1];
          utB = hK[2];
        }
        const double dB = 1.0 + al * (unB + ueB);
        const double dW = 1.0 + al * (unW[q] + utW[q]);
        const double dS = 1.0 + al * (ueS + utS);
        // one division for the three quotients: each is the other two
        // denominators times 1/(dB dW dS), within a few ulps; exact quotients
        // when that product lies outside [2^-930, 2^930) (or is not finite)
        double LB, LW, LS;
        {
          const double dBW = dB * dW;
          const double pr = dBW * dS;
          if (midrange64(pr)) {
            const double rq = 1.0 / pr;
            LB = ab * ((dW * dS) * rq);
            LW = aw * ((dB * dS) * rq);
            LS = as * (dBW * rq);
          } else {
            LB = ab / dB;
            LW = aw / dW;
            LS = as / dS;
          }
        }
        const double P1 = al * (LB * unB + LW * unW[q]);
        const double P2 = al * (LB * ueB + LS * ueS);
        const double P3 = al * (LW * utW[q] + LS * utS);
        const double LP = ap + P1 + P2 + P3 - LB * utB - LW * ueW[q] - LS * unS;
        double UN = 0, UE = 0, UT = 0;
        if (act) {
          // one division by LP: the U entries are products with its
          // reciprocal (which the L record stores anyway), within a few ulps
          // of three quotients and three FP64 divisions cheaper per cell
          const double RLP = 1.0 / LP;
          UN = (an - P1) * RLP;
          UE = (ae - P2) * RLP;
          UT = (at - P3) * RLP;
          if (LP == 0.0 || !finite64(RLP) || !finite64(LB) || !finite64(LW) || !finite64(LS) ||
              !finite64(UN) || !finite64(UE) || !finite64(UT) || !finite64(LP))
            atomicCAS(c.status, DEV_OK, DEV_BREAKDOWN);
          const long long cell = B.cell0 + rb(g.s0 + t, g.k(q)) + g.j;
          TF *fr = P.recF + cell * 4;
          fr[REC_LB] = (TF)LB;
          fr[REC_LW] = (TF)LW;
          fr[REC_LS] = (TF)LS;
          fr[REC_RLP] = (TF)RLP;
          TF *br = P.recB + cell * 4;
          br[RECB_UE] = (TF)UE;
          br[RECB_UN] = (TF)UN;
          br[RECB_UT] = (TF)UT;
          br[3] = (TF)0;
          if (lane == kTJ - 1 && g.hasN) {
            uint64_t *f = faceJ(myf, B, t, g.dk(q), W);
            Face<double>::put(f, UN, ep);
            Face<double>::put(f + 2, UE, ep);
            Face<double>::put(f + 4, UT, ep);
          }
          if (q == Q - 1 && g.eT && g.hasT) {
            uint64_t *f = faceK(myf, B, t, lane, W);
            Face<double>::put(f, UN, ep);
            Face<double>::put(f + 2, UE, ep);
            Face<double>::put(f + 4, UT, ep);
          }
        }
        nUN[q] = UN;
        nUE[q] = UE;
        nUT[q] = UT;
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        unW[q] = nUN[q];
        ueW[q] = nUE[q];
        utW[q] = nUT[q];
      }
    }
    cp_async_wait<0>();
    if (tr && threadIdx.x == 0) tr[2] = gtimer();
    __syncthreads();
  }
}

}  // namespace sipk
