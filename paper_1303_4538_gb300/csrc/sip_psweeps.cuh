// sip_psweeps.cuh -- substitution sweeps of Stone's SIP (arXiv:1303.4538,
// Sec. 1 / Sec. 4.1: the substitution part of resforward3d and backward3d)
// over the plan's tile layout.
//
// The recurrences make a cell depend on its lower neighbours W, S, B (forward)
// or on its upper neighbours E, N, T (backward); all cells of one hyperplane
// s = i + j + k are independent.  The (j, k) cross-section of a block is cut
// into 32 x TK column tiles; a tile is walked along i, hyperplane by
// hyperplane.  In the column layout (sip_internal.h: column (j, k) holds its
// cells along i contiguously, shifted so that element index = column base +
// plane s) every lane of a tile reads and writes its own column at
// consecutive positions, so a step's addresses are one running pointer per
// row and P planes of a row are one aligned, vectorised run:
//
//   * a step advances P planes.  With P > 1 a tile is one warp: lane = j,
//     the Q rows k0 .. k0 + Q - 1 in registers, so within a step plane m of
//     a row needs plane m - 1 of itself (W / E), of the lane j -+ 1 (S / N,
//     one shuffle) and of its neighbouring row (B / T, a register): P short
//     dependent sub-steps, the bookkeeping of the step paid once;
//   * with P = 1 a tile may span NWT warps of Q rows (the FP64 sweeps, whose
//     warp-wide FMAs take 64 cycles of a sub-partition's FP64 pipe on GB300):
//     a warp's edge row gets its neighbour row from the next warp through a
//     shared-memory ring guarded by per-warp progress counters (release /
//     acquire at CTA scope), so warps wait only for the warp that feeds them;
//   * each thread stages its own rows' records and scalars D - 1 steps ahead
//     with cp.async into its warp's private ring (16-byte copies, zero-filled
//     where a 4-cell group lies outside its column) and reads only what it
//     copied itself (cp.async.wait_group, no barrier);
//   * values cross tiles through epoch-tagged face words in global memory
//     (one 8-byte word per FP32 value, two per FP64 value, the launch's
//     epoch in each upper half, so every word validates itself), stored per
//     row (J) or lane (K) at consecutive planes; a consumer loads the words
//     of step u + 1 during step u and re-reads stale words with bounded
//     polls.  Every tile walks extra groups of planes before and after its
//     own, so every word a consumer reads is written by its producer;
//   * padding elements of the layout hold zero records and values, so the
//     arithmetic runs without branches and produces zeros there;
//   * every wait is bounded (max_spin polls): a lost producer gives an error
//     status (DEV_TIMEOUT), never a hang; every access is inside its column
//     or face region by construction and predicated on it.
#pragma once

#include <climits>

#include "sip_sweeps.cuh"

namespace sipk {

// ---------------------------------------------------------------- progress
__device__ __forceinline__ void prog_release(int *p, int v) {
  asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int prog_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
// Spin (bounded) until *p >= need; returns the value seen, or -1 after a
// timeout (recorded as DEV_TIMEOUT) or another thread's error.
static __device__ __noinline__ int prog_spin(const int *p, int need, long long max_spin, int *status,
                                             unsigned long long *tr) {
  const unsigned long long t0 = tr ? gtimer() : 0ull;
  long long spins = 0;
  int v = prog_acquire(p);
  while (v < need) {
    if (++spins > max_spin) {
      atomicCAS(status, DEV_OK, DEV_TIMEOUT);
      v = -1;
      break;
    }
    if ((spins & 255) == 0 && ld_relaxed(status) != DEV_OK) {
      v = -1;
      break;
    }
    v = prog_acquire(p);
  }
  if (tr && (threadIdx.x & 31) == 0) {
    atomicAdd(tr + 6, 1ull);
    atomicAdd(tr + 7, gtimer() - t0);
  }
  return v;
}
// Wait until *p >= need; `seen` caches the last value read (progress only
// grows); after an abort it is INT_MAX, so no later wait spins.
__device__ __forceinline__ void prog_wait(const int *p, int need, int &seen, const SweepCommon &c,
                                          unsigned long long *tr) {
  if (seen >= need) return;
  seen = prog_acquire(p);
  if (seen < need) {
    seen = prog_spin(p, need, c.max_spin, c.status, tr);
    if (seen < 0) seen = INT_MAX;
  }
}

// ---------------------------------------------------------------- face words
// One value: FP32 one word (payload | epoch << 32), FP64 two (low / high half
// | epoch << 32).
template <typename T>
struct WFace;
template <>
struct WFace<float> {
  static constexpr int WV = 1;
  __device__ static float get(const uint64_t *w) { return __uint_as_float((unsigned)w[0]); }
  __device__ static void make(float v, unsigned ep, uint64_t *w) {
    w[0] = ((uint64_t)ep << 32) | (uint64_t)__float_as_uint(v);
  }
};
template <>
struct WFace<double> {
  static constexpr int WV = 2;
  __device__ static double get(const uint64_t *w) {
    return __longlong_as_double((long long)((w[0] & 0xffffffffull) | (w[1] << 32)));
  }
  __device__ static void make(double v, unsigned ep, uint64_t *w) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const uint64_t tag = (uint64_t)ep << 32;
    w[0] = tag | (b & 0xffffffffull);
    w[1] = tag | (b >> 32);
  }
};

// predicated relaxed accesses (no branch; a load that does not happen yields zeros)
__device__ __forceinline__ void ld_relaxed_v2_if(const uint64_t *p, uint64_t &a, uint64_t &b, bool pred) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n mov.b64 %0, 0;\n mov.b64 %1, 0;\n"
      " @q ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];\n}\n"
      : "=l"(a), "=l"(b)
      : "l"(p), "r"((int)pred));
}
__device__ __forceinline__ void ld_relaxed_u64_if(const uint64_t *p, uint64_t &a, bool pred) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n mov.b64 %0, 0;\n @q ld.relaxed.gpu.global.u64 %0, [%1];\n}\n"
      : "=l"(a)
      : "l"(p), "r"((int)pred));
}
__device__ __forceinline__ void st_relaxed_u64_if(uint64_t *p, uint64_t a, bool pred) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.relaxed.gpu.global.u64 [%0], %1;\n}\n" ::"l"(p),
               "l"(a), "r"((int)pred));
}
// face stores need no compiler ordering against other memory accesses: their
// consumers are other CTAs, which validate every word by its tag
__device__ __forceinline__ void st_face_v2(uint64_t *p, uint64_t a, uint64_t b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b));
}
// cp.async of `BYTES` from a global address into a shared-window address;
// srcbytes 0 zero-fills the destination without reading (the address must
// still lie in an allocation: the column arrays carry margins for that)
__device__ __forceinline__ void cp_async_16_sz(unsigned sdst, const void *gsrc, int srcbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(gsrc), "r"(srcbytes) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_sz(unsigned sdst, const void *gsrc, int srcbytes) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(gsrc), "r"(srcbytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sdst), "l"(gsrc), "n"(BYTES), "r"(srcbytes)
                 : "memory");
}

// nonzero when any tag of w[0..N) differs from `expect`
template <int N>
__device__ __forceinline__ unsigned words_bad(const uint64_t *w, unsigned expect) {
  unsigned bad = 0;
#pragma unroll
  for (int q = 0; q < N; ++q) bad |= (unsigned)(w[q] >> 32) ^ expect;
  return bad;
}
// Re-read N words (bounded polls) until every tag matches (rare path).
template <int N>
__device__ __forceinline__ void words_wait(const uint64_t *p, uint64_t *w, unsigned expect, const SweepCommon &c,
                                           bool &abort, unsigned long long *tr) {
  long long spins = 0;
  const unsigned long long t0 = tr ? gtimer() : 0ull;
  while (!abort && words_bad<N>(w, expect)) {
    if (++spins > c.max_spin) {
      atomicCAS(c.status, DEV_OK, DEV_TIMEOUT);
      abort = true;
      break;
    }
    if ((spins & 63) == 0 && ld_relaxed(c.status) != DEV_OK) {
      abort = true;
      break;
    }
    __nanosleep(20);
#pragma unroll
    for (int q = 0; q < N; ++q) w[q] = ld_relaxed(p + q);
  }
  if (tr && spins > 0) {
    atomicAdd(tr + 3, 1ull);
    atomicAdd(tr + 4, gtimer() - t0);
  }
}


// ================================================================= sweep
// FWD: forward substitution y = L^-1 r,
//   y_P = (r_P - LB y_B - LW y_W - LS y_S) * (1/LP),   ascending planes,
// in place when out == sa (a cell's r is staged before its y is stored and
// no other cell reads it).
// !FWD: backward substitution with the update (backward3d),
//   d_P = y_P - UE d_E - UN d_N - UT d_T,  x_P <- x_P + d_P,   descending
// planes (ZX: x = 0 on entry, x_P <- d_P).
// A CTA of NW warps walks a 32 x (NW Q) tile one plane per step: step t is
// local position ps = t (FWD) or nsteps - 1 - t, and warp w's row q holds
// cell i = ps - lane - (w Q + q) of its column.  The warps march together
// (one barrier per step); a warp's edge row takes its neighbour row from the
// adjacent warp's value of the previous step through a double-buffered
// exchange in shared memory.
template <typename T, bool FWD, bool ZX, int Q, int D>
__global__ void __launch_bounds__(256) k_csweep(WParams<T> Pm) {
  using Cfg = CSweepCfg<sizeof(T), FWD, ZX, Q>;
  constexpr int NCH = Cfg::NCH;  // 16-byte chunks per record
  constexpr int NS = Cfg::NS;    // staged scalars per cell
  constexpr int WV = WFace<T>::WV;
  constexpr int DIR = FWD ? 1 : -1;
  const SweepCommon &c = Pm.c;
  __shared__ int s_claim;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned ep = sweep_prologue(c);
  if (__syncthreads_or(c.ctl->done || ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NW = blockDim.x >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const CLayout L = c_layout((int)sizeof(T), NS, Q, D, NW);
  const unsigned sm0 = smem_u32(smem_raw);
  // this warp's part of stage 0, the stage ring's end, the exchange buffers
  const int st0 = w * (int)L.warp_stage, stE = D * (int)L.stage;
  T *exch = reinterpret_cast<T *>(smem_raw + stE);  // [2][NW][32]
  // warps fed by / feeding the exchange: the warp below (FWD) or above
  const int wfeed = w - DIR;
  const bool has_feed = wfeed >= 0 && wfeed < NW;
  const int lane_in = FWD ? 0 : kTJ - 1, lane_out = FWD ? kTJ - 1 : 0;
  const int q_in = FWD ? 0 : Q - 1, q_out = FWD ? Q - 1 : 0;
  bool abort = false;

  for (;;) {
    const int mt = claim_tile(c, &s_claim);
    if (mt >= c.ntiles) break;
    const Tile tl = c.tiles[mt];
    const DevBlock B = c.blocks[tl.blk];
    unsigned long long *tr = c.trace ? c.trace + (size_t)tl.gtile * kTraceWords : nullptr;
    if (tr && threadIdx.x == 0) {
      tr[0] = gtimer();
      tr[5] = smid();
    }
    const int TK = NW * Q;
    const int j0 = tl.cj * kTJ, k0 = tl.ck * TK, j = j0 + lane;
    const int njt = min(kTJ, B.ny - j0), nkt = min(TK, B.nz - k0);
    const int nsteps = B.nx + njt + nkt - 2, last = nsteps - 1;
    const bool hasS = j0 > 0, hasN = j0 + kTJ < B.ny, hasB = k0 > 0, hasT = k0 + TK < B.nz;
    const bool inJ = FWD ? hasS : hasN, inK = FWD ? hasB : hasT;
    const bool outJ = FWD ? hasN : hasS, outK = FWD ? hasT : hasB;
    const bool w_in = w == (FWD ? 0 : NW - 1), w_out = w == (FWD ? NW - 1 : 0);
    // per row: cell i = ps - tlo at local position ps, valid iff
    // (unsigned)(ps - tlo) < nxq; element of position ps = rowb + 32 ps in
    // the tile layout (block-local; rows outside the block read nothing, at
    // the block start)
    int tlo[Q], rowb[Q];
    unsigned nxq[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int dk = w * Q + q, k = k0 + dk;
      const bool col = j < B.ny && k < B.nz;
      tlo[q] = lane + dk;
      nxq[q] = col ? (unsigned)B.nx : 0u;
      rowb[q] = (k < B.nz ? ((k * B.nTJ + tl.cj) * B.Lp - dk) * kTJ : 0) + lane;
    }
    const T *recb = Pm.rec + B.sk0 * 4;
    const T *sab = Pm.sa + B.sk0;
    const T *sbb = ((!FWD && !ZX) ? Pm.sb : Pm.sa) + B.sk0;
    T *outb = Pm.out + B.sk0;
    // faces: per tile J words [TK][NPOS][WV] then K words [32][NPOS][WV],
    // indexed by the producer's local position
    const int NPOS = B.nsteps_max;
    const long long kface = (long long)TK * NPOS * WV;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    const uint64_t *srcJ = inJ ? tile_faces(c, B, tl.gtile + (FWD ? -1 : 1)) : myf;
    const uint64_t *srcK = inK ? tile_faces(c, B, tl.gtile + (FWD ? -B.nTJ : B.nTJ)) : myf;
    // a consumer cell at position ps reads the producer's position ps + dJ (J) or ps + dK (K)
    const int dJ = DIR * (kTJ - 1), dK = DIR * (TK - 1);
    const bool jon = lane == lane_in && inJ, kon = w_in && inK;
    // J words of row q at position p: rowJ[q] + p * WV; K words: rowK + p * WV
    const uint64_t *rowJ = srcJ + (long long)(w * Q) * NPOS * WV;
    const uint64_t *rowK = srcK + kface + (long long)lane * NPOS * WV;
    uint64_t *outJrow = myf + (long long)(w * Q) * NPOS * WV;
    uint64_t *outKrow = myf + kface + (long long)lane * NPOS * WV;
    auto ps_of = [&](int t) { return FWD ? t : last - t; };
    struct FaceBuf {
      uint64_t j[Q][WV], k[WV];
    };
    // face words of step t (zeros where the cell is not valid)
    auto face_ld = [&](int t, FaceBuf &F) {
      const int ps = ps_of(t);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const bool v = jon && t < nsteps && (unsigned)(ps - tlo[q]) < nxq[q];
        const uint64_t *pj = rowJ + ((long long)q * NPOS + (v ? ps + dJ : 0)) * WV;
        if constexpr (WV == 2) ld_relaxed_v2_if(pj, F.j[q][0], F.j[q][1], v);
        else ld_relaxed_u64_if(pj, F.j[q][0], v);
      }
      const bool vk = kon && t < nsteps && (unsigned)(ps - tlo[q_in]) < nxq[q_in];
      const uint64_t *pk = rowK + (long long)(vk ? ps + dK : 0) * WV;
      if constexpr (WV == 2) ld_relaxed_v2_if(pk, F.k[0], F.k[1], vk);
      else ld_relaxed_u64_if(pk, F.k[0], vk);
    };
    auto face_bad = [&](int t, const FaceBuf &F) {
      const int ps = ps_of(t);
      unsigned bad = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (jon && (unsigned)(ps - tlo[q]) < nxq[q]) bad |= words_bad<WV>(F.j[q], expect);
      if (kon && (unsigned)(ps - tlo[q_in]) < nxq[q_in]) bad |= words_bad<WV>(F.k, expect);
      return bad;
    };
    auto face_wait = [&](int t, FaceBuf &F, unsigned long long *trp) {
      const int ps = ps_of(t);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (jon && (unsigned)(ps - tlo[q]) < nxq[q])
          words_wait<WV>(rowJ + ((long long)q * NPOS + ps + dJ) * WV, F.j[q], expect, c, abort, trp);
      if (kon && (unsigned)(ps - tlo[q_in]) < nxq[q_in])
        words_wait<WV>(rowK + (long long)(ps + dK) * WV, F.k, expect, c, abort, trp);
    };
    FaceBuf FA, FB;
    // start slack: before the walk, wait until the words needed `lead` steps
    // after the first need are published (J: each warp's edge lane; K: the
    // edge warp's first needing lane)
    {
      const int lead = min(c.lead, B.nx - 1);
      // the step where a row's first valid cell is met: FWD its lowest
      // position tlo, backward its highest tlo + nx - 1
      int tJ = nsteps, tK = nsteps;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (nxq[q]) tJ = min(tJ, FWD ? tlo[q] : last - (tlo[q] + B.nx - 1));
      if (nxq[q_in]) tK = FWD ? tlo[q_in] : last - (tlo[q_in] + B.nx - 1);
      const int uJ = min(tJ + lead, last), uK = min(tK + lead, last);
      face_ld(uJ, FA);
      face_ld(uK, FB);
      // FWD: lane 0 meets its first cells first; backward: the last valid lane
      const int lfirst = FWD ? 0 : njt - 1;
      bool gj = false, gk = false;
#pragma unroll
      for (int q = 0; q < Q; ++q) gj |= jon && (unsigned)(ps_of(uJ) - tlo[q]) < nxq[q];
      gk = kon && lane == lfirst && (unsigned)(ps_of(uK) - tlo[q_in]) < nxq[q_in];
      if (gj) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if ((unsigned)(ps_of(uJ) - tlo[q]) < nxq[q])
            words_wait<WV>(rowJ + ((long long)q * NPOS + ps_of(uJ) + dJ) * WV, FA.j[q], expect, c, abort, nullptr);
      }
      if (gk) words_wait<WV>(rowK + (long long)(ps_of(uK) + dK) * WV, FB.k, expect, c, abort, nullptr);
      __syncthreads();
      if (tr && threadIdx.x == 0) tr[1] = gtimer();
    }

    int oI = st0;  // this warp's part of the stage of the next issue step
    int tI = 0;    // next issue step
    auto issue = [&]() {
      const int ps = ps_of(tI);
      const unsigned sR = sm0 + oI + lane * 16, sS = sm0 + oI + Cfg::SREC + lane * (int)sizeof(T);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const bool v = (unsigned)(ps - tlo[q]) < nxq[q];
        const long long e = (long long)rowb[q] + 32ll * ps;  // element (inside the allocation's margins)
#pragma unroll
        for (int z = 0; z < NCH; ++z) cp_async_16_sz(sR + (q * NCH + z) * 512, recb + e * 4 + z * (16 / (int)sizeof(T)), v ? 16 : 0);
        cp_async_sz<sizeof(T)>(sS + q * 32 * (int)sizeof(T), sab + e, v ? (int)sizeof(T) : 0);
        if constexpr (NS == 2)
          cp_async_sz<sizeof(T)>(sS + (Q + q) * 32 * (int)sizeof(T), sbb + e, v ? (int)sizeof(T) : 0);
      }
      cp_async_commit();
      ++tI;
      oI += (int)L.stage;
      if (oI >= stE) oI -= stE;
    };

#pragma unroll
    for (int q = 0; q < D - 1; ++q) issue();
    T prev[Q];  // this lane's rows at the previous plane (the W / E neighbours)
#pragma unroll
    for (int q = 0; q < Q; ++q) prev[q] = T(0);
    face_ld(0, FA);
    face_ld(1, FB);
    int oC = st0;  // this warp's part of the stage being computed
    const bool jout = lane == lane_out && outJ, kout = w_out && outK;

    auto body = [&](int t, FaceBuf &F) {
      issue();
      cp_async_wait<D - 1>();
      const int ps = ps_of(t);
      // the adjacent warp's edge-row values of the previous step are in exch[(t - 1) & 1]
      __syncthreads();
      // faces of this step; stale words are re-read (rare, warp-uniform branch)
      if (__any_sync(0xffffffffu, face_bad(t, F) != 0)) face_wait(t, F, tr);
      T edge = WFace<T>::get(F.k);
      if (has_feed) edge = t > 0 ? exch[(((t - 1) & 1) * NW + wfeed) * 32 + lane] : T(0);
      const T *ss = reinterpret_cast<const T *>(smem_raw + oC + Cfg::SREC) + lane;
      T nv[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        T c0, c1, c2, c3;
        if constexpr (NCH == 1) {
          const float4 v = *reinterpret_cast<const float4 *>(smem_raw + oC + q * 512 + lane * 16);
          c0 = v.x; c1 = v.y; c2 = v.z; c3 = v.w;
        } else {
          const double2 v0 = *reinterpret_cast<const double2 *>(smem_raw + oC + (2 * q) * 512 + lane * 16);
          const double2 v1 = *reinterpret_cast<const double2 *>(smem_raw + oC + (2 * q + 1) * 512 + lane * 16);
          c0 = v0.x; c1 = v0.y; c2 = v1.x; c3 = v1.y;
        }
        const bool v = (unsigned)(ps - tlo[q]) < nxq[q];
        // lane neighbour (S for FWD, N backward): shuffle, the J face at the edge lane
        T ln = FWD ? shfl_up1(prev[q]) : shfl_dn1(prev[q]);
        if (lane == lane_in) ln = WFace<T>::get(F.j[q]);
        // row neighbour (B for FWD, T backward)
        T rn;
        if constexpr (FWD) rn = q > 0 ? prev[q > 0 ? q - 1 : 0] : edge;
        else rn = q < Q - 1 ? prev[q < Q - 1 ? q + 1 : 0] : edge;
        T val;
        if constexpr (FWD) {  // L record [LB LW LS 1/LP]
          val = fma(-c0, rn, ss[q * 32]);
          val = fma(-c1, prev[q], val);
          val = fma(-c2, ln, val);
          val *= c3;
        } else {              // U record [UE UN UT 0]
          val = fma(-c0, prev[q], ss[q * 32]);
          val = fma(-c1, ln, val);
          val = fma(-c2, rn, val);
          (void)c3;
        }
        nv[q] = v ? val : T(0);
        T ov = val;
        if constexpr (!FWD && !ZX) ov = ss[(Q + q) * 32] + val;
        if (v) outb[(long long)rowb[q] + 32ll * ps] = ov;
      }
      // this warp's edge row for the adjacent warp (read after the next barrier)
      exch[((t & 1) * NW + w) * 32 + lane] = nv[q_out];
      // faces for the downstream tiles: J (edge lane, the warp's rows), K (edge warp's edge row)
      if (jout) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          uint64_t wv[WV];
          WFace<T>::make(nv[q], ep, wv);
          uint64_t *dst = outJrow + ((long long)q * NPOS + ps) * WV;
          if constexpr (WV == 2) st_face_v2(dst, wv[0], wv[1]);
          else st_relaxed_u64_if(dst, wv[0], true);
        }
      }
      if (kout) {
        uint64_t wv[WV];
        WFace<T>::make(nv[q_out], ep, wv);
        uint64_t *dst = outKrow + (long long)ps * WV;
        if constexpr (WV == 2) st_face_v2(dst, wv[0], wv[1]);
        else st_relaxed_u64_if(dst, wv[0], true);
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) prev[q] = nv[q];
      oC += (int)L.stage;
      if (oC >= stE) oC -= stE;
      face_ld(t + 2, F);  // this buffer's next use is step t + 2
    };

    for (int t = 0; t < nsteps; t += 2) {
      body(t, FA);
      if (t + 1 < nsteps) body(t + 1, FB);
    }
    cp_async_wait<0>();
    __syncthreads();
    if (tr && threadIdx.x == 0) tr[2] = gtimer();
  }
}

}  // namespace sipk
