// sip_sweeps.cuh -- sm_103a kernels of Stone's SIP over the plane layout.
//
// The recurrences of the method (arXiv:1303.4538, Sec. 1 / Sec. 4.1: lu3d,
// resforward3d, backward3d) make a cell depend on its lower neighbours W, S,
// B (factorisation and forward substitution) or on its upper neighbours E, N,
// T (backward substitution).  All cells of one hyperplane i + j + k = s are
// independent, so the sweeps advance plane by plane.  Work decomposition:
//
//   * the (j, k) cross-section of a block is cut into TJ x TK column tiles;
//     one CTA owns a tile, one thread owns a (j, k) column and walks i, so at
//     local step t every thread of the tile is on global plane s = t + j0 + k0;
//   * inside the tile the neighbour values of the previous (or next) plane
//     pass through a double-buffered shared-memory exchange, one barrier per
//     step; W/E come from the thread's own registers;
//   * the cell data of each step (coefficients, factors, rhs, x) is staged
//     by cp.async into a per-thread ring of R shared-memory stages, R-1 steps
//     ahead of use; invalid cells are zero-filled, so the arithmetic runs
//     without branches and inactive threads produce zeros;
//   * between tiles, the recurrence's boundary values travel through "faces":
//     16-byte records of two 8-byte words whose upper halves carry the
//     launch's epoch tag.  A producer stores a record with one st.relaxed.gpu;
//     a consumer prefetches it with cp.async.cg into a shared-memory ring
//     together with the step's other data and accepts it when every tag
//     matches (each word is self-validating, so no fence or flag is needed);
//     a stale record is re-read from L2 with ld.relaxed.gpu until it matches.
//     Before a tile starts, one thread waits until the upstream tiles are a
//     few steps ahead ("slack"), so the prefetched records are normally valid
//     and no step pays an L2 round trip.  Every wait is bounded (max_spin
//     polls), then the kernel records DEV_TIMEOUT and runs to the end
//     without waiting again;
//   * CTAs claim tiles with an atomic ticket in a dependency-respecting order,
//     so a tile only waits for tiles claimed earlier by running CTAs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_internal.h"

namespace sipk {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void *sdst, const void *gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "n"(BYTES), "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_16_l2(void *sdst, const void *gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2(uint64_t *p, uint64_t a, uint64_t b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------- faces
// A face value is a 16-byte record (two words, each = payload32 | epoch32 << 32).
template <typename T>
struct Face;
template <>
struct Face<float> {
  __device__ static void put(uint64_t *p, float v, unsigned ep) {
    const uint64_t tag = (uint64_t)ep << 32;
    st_relaxed_v2(p, tag | (uint64_t)__float_as_uint(v), tag);
  }
  __device__ static float get(const uint64_t *w) { return __uint_as_float((unsigned)w[0]); }
};
template <>
struct Face<double> {
  __device__ static void put(uint64_t *p, double v, unsigned ep) {
    const uint64_t tag = (uint64_t)ep << 32;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_relaxed_v2(p, tag | (b & 0xffffffffull), tag | (b >> 32));
  }
  __device__ static double get(const uint64_t *w) {
    return __longlong_as_double((long long)((w[0] & 0xffffffffull) | (w[1] << 32)));
  }
};

template <int W>
__device__ __forceinline__ bool rec_ok(const uint64_t (&w)[W], unsigned expect) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < W; ++q) ok = ok && ((unsigned)(w[q] >> 32) == expect);
  return ok;
}

// Poll a W-word record in L2 until every tag equals `expect`.  Returns false
// (and zero words) after max_spin polls or once another thread recorded an
// error; `abort` then stays set so this thread never waits again.
template <int W>
__device__ __noinline__ bool face_wait(const uint64_t *p, unsigned expect, uint64_t (&w)[W],
                                       const SweepCommon &c, bool &abort) {
  if (!abort) {
    long long spins = 0;
    for (;;) {
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = ld_relaxed(p + q);
      if (rec_ok<W>(w, expect)) return true;
      ++spins;
      if (spins > c.max_spin) {
        atomicCAS(c.status, DEV_OK, DEV_TIMEOUT);
        abort = true;
        break;
      }
      if ((spins & 63) == 0 && ld_relaxed(c.status) != DEV_OK) {
        abort = true;
        break;
      }
      __nanosleep(32);
    }
  }
#pragma unroll
  for (int q = 0; q < W; ++q) w[q] = 0;
  return false;
}

// Take the record staged in shared memory; re-read it from L2 if it is stale.
template <int W>
__device__ __forceinline__ void rec_take(const uint64_t *staged, const uint64_t *g, unsigned expect,
                                         uint64_t (&w)[W], const SweepCommon &c, bool &abort) {
#pragma unroll
  for (int q = 0; q < W; ++q) w[q] = staged[q];
  if (!rec_ok<W>(w, expect)) face_wait<W>(g, expect, w, c, abort);
}

template <int W>
__device__ __forceinline__ void rec_prefetch(uint64_t *sdst, const uint64_t *g) {
#pragma unroll
  for (int q = 0; q < W; q += 2) cp_async_16_l2(sdst + q, g + q);
}

// Face storage of one tile: J face [nsteps_max][TK][W], then K face
// [nsteps_max][TJ][W], indexed by the producer's local step.
__device__ __forceinline__ uint64_t *tile_faces(const SweepCommon &c, const DevBlock &B, int gtile) {
  return c.faces + B.face0 + (long long)(gtile - B.tile0) * B.face_tile_words;
}
__device__ __forceinline__ uint64_t *faceJ(uint64_t *base, const DevBlock &B, int t, int lane, int W) {
  return base + ((long long)t * B.TK + lane) * W;
}
__device__ __forceinline__ uint64_t *faceK(uint64_t *base, const DevBlock &B, int t, int lane, int W) {
  return base + (long long)B.nsteps_max * B.TK * W + ((long long)t * B.TJ + lane) * W;
}

// Claim the next tile (thread 0), broadcast through shared memory.
__device__ __forceinline__ int claim_tile(const SweepCommon &c, int *s_claim) {
  if (threadIdx.x == 0) *s_claim = (ld_relaxed(c.status) != DEV_OK) ? c.ntiles : atomicAdd(c.ticket, 1);
  __syncthreads();
  const int m = *s_claim;
  __syncthreads();
  return m;
}

// Launch prologue shared by the ticketed kernels: zero the next launch's
// ticket and advance the other epoch slot (block 0, thread 0).  Returns the
// epoch this launch tags its faces with.
__device__ __forceinline__ unsigned sweep_prologue(const SweepCommon &c) {
  const unsigned ep = c.ctl->epochs[c.ep_slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (c.reset_ticket) *c.reset_ticket = 0;
    c.ctl->epochs[c.ep_slot ^ 1] = ep + 1u;
  }
  return ep;
}

__device__ __forceinline__ double block_sum(double v, double *s_red) {
  // deterministic: fixed shuffle tree, then warps summed in order by thread 0
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < nw; ++q) t += s_red[q];
  }
  __syncthreads();
  return t;
}

struct ColGeom {
  int dj, dk, j0, k0, j, k, nsteps, s0, njt, nkt;
  bool col, hasS, hasN, hasB, hasT;
  __device__ ColGeom(const DevBlock &B, const Tile &tl) {
    dj = threadIdx.x % B.TJ;
    dk = threadIdx.x / B.TJ;
    j0 = tl.cj * B.TJ;
    k0 = tl.ck * B.TK;
    j = j0 + dj;
    k = k0 + dk;
    col = (j < B.ny) && (k < B.nz) && (dk < B.TK);
    njt = min(B.TJ, B.ny - j0);
    nkt = min(B.TK, B.nz - k0);
    nsteps = B.nx + njt + nkt - 2;
    s0 = j0 + k0;
    hasS = j0 > 0;
    hasN = j0 + B.TJ < B.ny;
    hasB = k0 > 0;
    hasT = k0 + B.TK < B.nz;
  }
};

// Shared-memory carve-up of a sweep kernel: stage ring, exchange buffer, face ring.
template <typename T>
struct Smem {
  T *stage;       // [R][NV][NT]
  T *exch;        // [2][NE][EC]
  uint64_t *fst;  // [R][FS][W]
  __device__ Smem(unsigned char *raw, int R, int NV, int NT, int NE, int EC) {
    stage = reinterpret_cast<T *>(raw);
    size_t off = (size_t)R * NV * NT * sizeof(T);
    exch = reinterpret_cast<T *>(raw + off);
    off += (size_t)2 * NE * EC * sizeof(T);
    off = (off + 15) & ~(size_t)15;
    fst = reinterpret_cast<uint64_t *>(raw + off);
  }
};

// Slack gate: before a tile starts, wait until the records that the tile will
// consume `lead` steps after its first need are published, so the records
// prefetched during the walk are normally already valid.
template <int W>
__device__ __forceinline__ void slack_gate(const uint64_t *recJ, const uint64_t *recK, unsigned expect,
                                           const SweepCommon &c, bool &abort) {
  if (threadIdx.x == 0) {
    uint64_t w[W];
    if (recJ) face_wait<W>(recJ, expect, w, c, abort);
    if (recK) face_wait<W>(recK, expect, w, c, abort);
  }
  __syncthreads();
}

// ============================================================== factorisation
// Stone's factorisation, per cell after W, S, B (lu3d):
//   LB = AB / (1 + a (UN_B + UE_B)),  LW = AW / (1 + a (UN_W + UT_W)),
//   LS = AS / (1 + a (UE_S + UT_S)),
//   P1 = a (LB UN_B + LW UN_W),  P2 = a (LB UE_B + LS UE_S),  P3 = a (LW UT_W + LS UT_S),
//   LP = AP + P1 + P2 + P3 - LB UT_B - LW UE_W - LS UN_S,
//   UN = (AN - P1) / LP,  UE = (AE - P2) / LP,  UT = (AT - P3) / LP.
// Stored: LB, LW, LS, 1/LP, UN, UE, UT.  Faces carry (UN, UE, UT): 48 bytes.
template <int R>
__global__ void __launch_bounds__(512) k_factor(FacParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim;
  constexpr int NV = 7, W = 6;
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const int EC = c.exch_cells, FS = c.face_slots;
  Smem<double> sm(smem_raw, R, NV, NT, 3, EC);
  bool abort = false;

  for (;;) {
    const int m = claim_tile(c, &s_claim);
    if (m >= c.ntiles) break;
    const Tile tl = c.tiles[m];
    const DevBlock B = c.blocks[tl.blk];
    const ColGeom g(B, tl);
    const int *rbk = B.rbT + (long long)min(g.k, B.nz - 1) * B.nplanes;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *upJ = g.hasS ? tile_faces(c, B, tl.gtile - 1) : nullptr;
    uint64_t *upK = g.hasB ? tile_faces(c, B, tl.gtile - B.nTJ) : nullptr;
    const int TJ2 = B.TJ + 2;
    const int me = (g.dk + 1) * TJ2 + g.dj + 1;
    const bool cJ = g.dj == 0 && g.hasS, cK = g.dk == 0 && g.hasB;  // face consumers
    {
      const int lead = min(R + 1, B.nx - 1);
      slack_gate<W>(upJ ? faceJ(upJ, B, lead + B.TJ - 1, 0, W) : nullptr,
                    upK ? faceK(upK, B, lead + B.TK - 1, 0, W) : nullptr, expect, c, abort);
    }

    auto issue = [&](int tt) {
      if (tt < g.nsteps) {
        const int i = tt - g.dj - g.dk;
        const bool v = g.col && i >= 0 && i < B.nx;
        const long long a = v ? B.cell0 + rbk[g.s0 + tt] + g.j : 0;
        double *st = sm.stage + (size_t)(tt % R) * NV * NT + tid;
#pragma unroll
        for (int q = 0; q < NV; ++q) cp_async_zfill<8>(st + q * NT, P.a[q] + a, v);
        uint64_t *fs = sm.fst + (size_t)(tt % R) * FS * W;
        if (cJ && v) rec_prefetch<W>(fs + g.dk * W, faceJ(upJ, B, tt + B.TJ - 1, g.dk, W));
        if (cK && v) rec_prefetch<W>(fs + (B.TK + g.dj) * W, faceK(upK, B, tt + B.TK - 1, g.dj, W));
      }
      cp_async_commit();
    };
#pragma unroll
    for (int tt = 0; tt < R - 1; ++tt) issue(tt);

    double unW = 0, ueW = 0, utW = 0;
    const double al = P.alpha;
    for (int t = 0; t < g.nsteps; ++t) {
      issue(t + R - 1);
      cp_async_wait<R - 1>();
      const double *st = sm.stage + (size_t)(t % R) * NV * NT + tid;
      const uint64_t *fs = sm.fst + (size_t)(t % R) * FS * W;
      const int i = t - g.dj - g.dk;
      const bool act = g.col && i >= 0 && i < B.nx;
      double *E = sm.exch + (size_t)(t & 1) * 3 * EC;
      E[me] = unW;
      E[EC + me] = ueW;
      E[2 * EC + me] = utW;
      if (g.dj == 0) {
        uint64_t w[W] = {0, 0, 0, 0, 0, 0};
        if (act && cJ) rec_take<W>(fs + g.dk * W, faceJ(upJ, B, t + B.TJ - 1, g.dk, W), expect, w, c, abort);
        E[me - 1] = Face<double>::get(w);
        E[EC + me - 1] = Face<double>::get(w + 2);
        E[2 * EC + me - 1] = Face<double>::get(w + 4);
      }
      if (g.dk == 0) {
        uint64_t w[W] = {0, 0, 0, 0, 0, 0};
        if (act && cK)
          rec_take<W>(fs + (B.TK + g.dj) * W, faceK(upK, B, t + B.TK - 1, g.dj, W), expect, w, c, abort);
        E[me - TJ2] = Face<double>::get(w);
        E[EC + me - TJ2] = Face<double>::get(w + 2);
        E[2 * EC + me - TJ2] = Face<double>::get(w + 4);
      }
      __syncthreads();
      const double unS = E[me - 1], ueS = E[EC + me - 1], utS = E[2 * EC + me - 1];
      const double unB = E[me - TJ2], ueB = E[EC + me - TJ2], utB = E[2 * EC + me - TJ2];
      const double ap = st[0], aw = st[NT], ae = st[2 * NT], as = st[3 * NT], an = st[4 * NT],
                   ab = st[5 * NT], at = st[6 * NT];
      const double LB = ab / (1.0 + al * (unB + ueB));
      const double LW = aw / (1.0 + al * (unW + utW));
      const double LS = as / (1.0 + al * (ueS + utS));
      const double P1 = al * (LB * unB + LW * unW);
      const double P2 = al * (LB * ueB + LS * ueS);
      const double P3 = al * (LW * utW + LS * utS);
      const double LP = ap + P1 + P2 + P3 - LB * utB - LW * ueW - LS * unS;
      double UN = 0, UE = 0, UT = 0;
      if (act) {
        UN = (an - P1) / LP;
        UE = (ae - P2) / LP;
        UT = (at - P3) / LP;
        const double RLP = 1.0 / LP;
        if (LP == 0.0 || !isfinite(RLP) || !isfinite(LB) || !isfinite(LW) || !isfinite(LS) ||
            !isfinite(UN) || !isfinite(UE) || !isfinite(UT) || !isfinite(LP))
          atomicCAS(c.status, DEV_OK, DEV_BREAKDOWN);
        const long long a = B.cell0 + rbk[g.s0 + t] + g.j;
        const double outv[7] = {LB, LW, LS, RLP, UN, UE, UT};
#pragma unroll
        for (int q = 0; q < 7; ++q) P.f[q][a] = outv[q];
        if (P.f32[0]) {
#pragma unroll
          for (int q = 0; q < 7; ++q) P.f32[q][a] = (float)outv[q];
        }
        if (g.dj == B.TJ - 1 && g.hasN) {
          uint64_t *f = faceJ(myf, B, t, g.dk, W);
          Face<double>::put(f, UN, ep);
          Face<double>::put(f + 2, UE, ep);
          Face<double>::put(f + 4, UT, ep);
        }
        if (g.dk == B.TK - 1 && g.hasT) {
          uint64_t *f = faceK(myf, B, t, g.dj, W);
          Face<double>::put(f, UN, ep);
          Face<double>::put(f + 2, UE, ep);
          Face<double>::put(f + 4, UT, ep);
        }
      }
      unW = UN;
      ueW = UE;
      utW = UT;
    }
    cp_async_wait<0>();
    __syncthreads();
  }
}

// ============================================================ forward sweep
// resforward3d: r = b - A x (norm of r), then y = L^{-1} r with
//   y_P = (r_P - LB y_B - LW y_W - LS y_S) * (1/LP).
// SYM: A symmetric, only AP, AE, AN, AT are read; AW(P) = AE(W),
//      AS(P) = AN(S), AB(P) = AT(B) (the paper's Listing 1).
// ZX:  x = 0, so r = b (first inner iteration of the refinement).
// Staged values per thread and step (slot index):
template <bool SYM, bool ZX>
struct FwdSlots {
  // general: ap aw ae as an ab at lb lw ls rlp b xp1 hxj hxk
  // sym:     ap ae an at lb lw ls rlp b xp1 hxj hxk hanS hatB
  // zx:      lb lw ls rlp b
  static constexpr int NA = ZX ? 0 : (SYM ? 4 : 7);
  static constexpr int LB = NA, LW = NA + 1, LS = NA + 2, RLP = NA + 3, B = NA + 4;
  static constexpr int XP1 = NA + 5, HXJ = NA + 6, HXK = NA + 7;
  static constexpr int HANS = NA + 8, HATB = NA + 9;
  static constexpr int NV = ZX ? 5 : (SYM ? 14 : 15);
  static constexpr int NE = ZX ? 1 : (SYM ? 5 : 3);  // exchanged values: [ym1] or [xm1 xp1 ym1 (anm1 atm1)]
};

template <typename T, bool SYM, bool ZX, bool NORM, int R>
__global__ void __launch_bounds__(512) k_forward(FwdParams<T> P) {
  static_assert(!(SYM && ZX), "x = 0 needs no matrix");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim;
  __shared__ double s_red[32];
  using S = FwdSlots<SYM, ZX>;
  constexpr int NV = S::NV, NE = S::NE, W = 2;
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(c.ctl->done || ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const int EC = c.exch_cells, FS = c.face_slots;
  Smem<T> sm(smem_raw, R, NV, NT, NE, EC);
  const T *src[S::NA > 0 ? S::NA : 1];
  if constexpr (!ZX) {
    if constexpr (SYM) {
      src[0] = P.ap; src[1] = P.ae; src[2] = P.an; src[3] = P.at;
    } else {
      src[0] = P.ap; src[1] = P.aw; src[2] = P.ae; src[3] = P.as;
      src[4] = P.an; src[5] = P.ab; src[6] = P.at;
    }
  }
  constexpr int EB = (int)sizeof(T);
  bool abort = false;

  for (;;) {
    const int m = claim_tile(c, &s_claim);
    if (m >= c.ntiles) break;
    const Tile tl = c.tiles[m];
    const DevBlock B = c.blocks[tl.blk];
    const ColGeom g(B, tl);
    const int *rbk = B.rbT + (long long)min(g.k, B.nz - 1) * B.nplanes;
    const int *rbkB = B.rbT + (long long)max(g.k - 1, 0) * B.nplanes;
    const int *rbkT = B.rbT + (long long)min(g.k + 1, B.nz - 1) * B.nplanes;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *upJ = g.hasS ? tile_faces(c, B, tl.gtile - 1) : nullptr;
    uint64_t *upK = g.hasB ? tile_faces(c, B, tl.gtile - B.nTJ) : nullptr;
    const int TJ2 = B.TJ + 2;
    const int me = (g.dk + 1) * TJ2 + g.dj + 1;
    const bool eS = g.dj == 0, eN = g.dj == B.TJ - 1, eB = g.dk == 0, eT = g.dk == B.TK - 1;
    const bool cJ = eS && g.hasS, cK = eB && g.hasB;  // face consumers
    {
      const int lead = min(R + 1, B.nx - 1);
      slack_gate<W>(upJ ? faceJ(upJ, B, lead + B.TJ - 1, 0, W) : nullptr,
                    upK ? faceK(upK, B, lead + B.TK - 1, 0, W) : nullptr, expect, c, abort);
    }

    auto issue = [&](int tt) {
      if (tt < g.nsteps) {
        const int i = tt - g.dj - g.dk;
        const int s = g.s0 + tt;
        const bool v = g.col && i >= 0 && i < B.nx;
        const long long a = v ? B.cell0 + rbk[s] + g.j : 0;
        T *st = sm.stage + (size_t)(tt % R) * NV * NT + tid;
        if constexpr (!ZX) {
#pragma unroll
          for (int q = 0; q < S::NA; ++q) cp_async_zfill<EB>(st + q * NT, src[q] + a, v);
        }
        cp_async_zfill<EB>(st + S::LB * NT, P.lb + a, v);
        cp_async_zfill<EB>(st + S::LW * NT, P.lw + a, v);
        cp_async_zfill<EB>(st + S::LS * NT, P.ls + a, v);
        cp_async_zfill<EB>(st + S::RLP * NT, P.rlp + a, v);
        cp_async_zfill<EB>(st + S::B * NT, P.b + a, v);
        if constexpr (!ZX) {
          const bool vp = g.col && i + 1 >= 0 && i + 1 < B.nx;
          const long long ap1 = vp ? B.cell0 + rbk[s + 1] + g.j : 0;
          cp_async_zfill<EB>(st + S::XP1 * NT, P.x + ap1, vp);
          // halo x across the tile's j faces (S for dj = 0, N for dj = TJ-1)
          long long hj = 0;
          bool vj = false;
          if (eS && g.hasS && v) { hj = B.cell0 + rbk[s - 1] + g.j0 - 1; vj = true; }
          else if (eN && g.hasN && v) { hj = B.cell0 + rbk[s + 1] + g.j0 + B.TJ; vj = true; }
          cp_async_zfill<EB>(st + S::HXJ * NT, P.x + hj, vj);
          long long hk = 0;
          bool vk = false;
          if (eB && g.hasB && v) { hk = B.cell0 + rbkB[s - 1] + g.j; vk = true; }
          else if (eT && g.hasT && v) { hk = B.cell0 + rbkT[s + 1] + g.j; vk = true; }
          cp_async_zfill<EB>(st + S::HXK * NT, P.x + hk, vk);
          if constexpr (SYM) {
            cp_async_zfill<EB>(st + S::HANS * NT, P.an + hj, vj && eS);
            cp_async_zfill<EB>(st + S::HATB * NT, P.at + hk, vk && eB);
          }
        }
        uint64_t *fs = sm.fst + (size_t)(tt % R) * FS * W;
        if (cJ && v) rec_prefetch<W>(fs + g.dk * W, faceJ(upJ, B, tt + B.TJ - 1, g.dk, W));
        if (cK && v) rec_prefetch<W>(fs + (B.TK + g.dj) * W, faceK(upK, B, tt + B.TK - 1, g.dj, W));
      }
      cp_async_commit();
    };
#pragma unroll
    for (int tt = 0; tt < R - 1; ++tt) issue(tt);

    T xm1 = 0, x0 = 0, ym1 = 0, aem1 = 0, anm1 = 0, atm1 = 0;
    double acc = 0.0;
    // x of a column's first cell normally arrives as the previous step's x(i+1);
    // the tile's corner column starts at i = 0 on step 0, so it reads it here
    if constexpr (!ZX) {
      if (g.dj == 0 && g.dk == 0 && g.col) x0 = P.x[B.cell0 + rbk[g.s0] + g.j];
    }
    for (int t = 0; t < g.nsteps; ++t) {
      issue(t + R - 1);
      cp_async_wait<R - 1>();
      const T *st = sm.stage + (size_t)(t % R) * NV * NT + tid;
      const uint64_t *fs = sm.fst + (size_t)(t % R) * FS * W;
      const int i = t - g.dj - g.dk;
      const bool act = g.col && i >= 0 && i < B.nx;
      T *E = sm.exch + (size_t)(t & 1) * NE * EC;
      T *EY = E + (ZX ? 0 : 2) * EC;  // ym1 plane
      T xp1 = 0;
      if constexpr (!ZX) {
        xp1 = st[S::XP1 * NT];
        E[me] = xm1;
        E[EC + me] = xp1;
        if constexpr (SYM) {
          E[3 * EC + me] = anm1;
          E[4 * EC + me] = atm1;
        }
      }
      EY[me] = ym1;
      if (eS) {
        uint64_t w[W] = {0, 0};
        if (act && cJ) rec_take<W>(fs + g.dk * W, faceJ(upJ, B, t + B.TJ - 1, g.dk, W), expect, w, c, abort);
        EY[me - 1] = Face<T>::get(w);
        if constexpr (!ZX) {
          E[me - 1] = st[S::HXJ * NT];
          if constexpr (SYM) E[3 * EC + me - 1] = st[S::HANS * NT];
        }
      }
      if constexpr (!ZX) {
        if (eN) E[EC + me + 1] = st[S::HXJ * NT];
        if (eT) E[EC + me + TJ2] = st[S::HXK * NT];
      }
      if (eB) {
        uint64_t w[W] = {0, 0};
        if (act && cK)
          rec_take<W>(fs + (B.TK + g.dj) * W, faceK(upK, B, t + B.TK - 1, g.dj, W), expect, w, c, abort);
        EY[me - TJ2] = Face<T>::get(w);
        if constexpr (!ZX) {
          E[me - TJ2] = st[S::HXK * NT];
          if constexpr (SYM) E[4 * EC + me - TJ2] = st[S::HATB * NT];
        }
      }
      __syncthreads();
      T r = st[S::B * NT];
      if constexpr (!ZX) {
        const T xS = E[me - 1], xN = E[EC + me + 1], xB = E[me - TJ2], xT = E[EC + me + TJ2];
        if constexpr (SYM) {
          const T ap = st[0], ae = st[NT], an = st[2 * NT], at = st[3 * NT];
          const T asv = E[3 * EC + me - 1], abv = E[4 * EC + me - TJ2];
          r = fma(-ap, x0, r);
          r = fma(-aem1, xm1, r);
          r = fma(-ae, xp1, r);
          r = fma(-asv, xS, r);
          r = fma(-an, xN, r);
          r = fma(-abv, xB, r);
          r = fma(-at, xT, r);
          aem1 = ae;
          anm1 = an;
          atm1 = at;
        } else {
          r = fma(-st[0], x0, r);
          r = fma(-st[NT], xm1, r);
          r = fma(-st[2 * NT], xp1, r);
          r = fma(-st[3 * NT], xS, r);
          r = fma(-st[4 * NT], xN, r);
          r = fma(-st[5 * NT], xB, r);
          r = fma(-st[6 * NT], xT, r);
        }
      }
      const T yS = EY[me - 1], yB = EY[me - TJ2];
      T y = fma(-st[S::LB * NT], yB, r);
      y = fma(-st[S::LW * NT], ym1, y);
      y = fma(-st[S::LS * NT], yS, y);
      y = y * st[S::RLP * NT];
      if constexpr (NORM) acc = fma((double)r, (double)r, acc);
      if (act) {
        const long long a = B.cell0 + rbk[g.s0 + t] + g.j;
        P.y[a] = y;
        if (eN && g.hasN) Face<T>::put(faceJ(myf, B, t, g.dk, W), y, ep);
        if (eT && g.hasT) Face<T>::put(faceK(myf, B, t, g.dj, W), y, ep);
      }
      xm1 = x0;
      x0 = xp1;
      ym1 = act ? y : T(0);
    }
    cp_async_wait<0>();
    if constexpr (NORM) {
      const double tot = block_sum(acc, s_red);
      if (tid == 0) P.partials[tl.gtile] = tot;
    }
    __syncthreads();
  }
}

// =========================================================== backward sweep
// backward3d with the update: d_P = y_P - UE d_E - UN d_N - UT d_T
// (descending planes), x_P <- x_P + d_P.  ZX: x = 0 on entry (x_P <- d_P).
// UPD64 (refined mode, last inner iteration): x64_P += (double) x_P instead
// of storing x_P.
template <typename T, bool ZX, bool UPD64, int R>
__global__ void __launch_bounds__(512) k_backward(BwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim;
  constexpr int NV = (ZX ? 4 : 5) + (UPD64 ? 2 : 0);  // ue un ut y [x] [x64 as 2 slots]
  constexpr int W = 2;
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(c.ctl->done || ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const int EC = c.exch_cells, FS = c.face_slots;
  Smem<T> sm(smem_raw, R, NV, NT, 1, EC);
  constexpr int EB = (int)sizeof(T);
  bool abort = false;

  for (;;) {
    const int m = claim_tile(c, &s_claim);
    if (m >= c.ntiles) break;
    const Tile tl = c.tiles[m];
    const DevBlock B = c.blocks[tl.blk];
    const ColGeom g(B, tl);
    const int *rbk = B.rbT + (long long)min(g.k, B.nz - 1) * B.nplanes;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *dnJ = g.hasN ? tile_faces(c, B, tl.gtile + 1) : nullptr;
    uint64_t *dnK = g.hasT ? tile_faces(c, B, tl.gtile + B.nTJ) : nullptr;
    const int TJ2 = B.TJ + 2;
    const int me = (g.dk + 1) * TJ2 + g.dj + 1;
    const int last = g.nsteps - 1;
    const bool cJ = g.dj == B.TJ - 1 && g.hasN, cK = g.dk == B.TK - 1 && g.hasT;  // face consumers
    {
      // the consumer of the last valid row (column) needs, `lead` steps into
      // the walk, cell i = nx-1-lead, published on the producer's step i + lane
      const int lead = min(R + 1, B.nx - 1);
      const int i = B.nx - 1 - lead;
      slack_gate<W>(dnJ ? faceJ(dnJ, B, i + g.nkt - 1, g.nkt - 1, W) : nullptr,
                    dnK ? faceK(dnK, B, i + g.njt - 1, g.njt - 1, W) : nullptr, expect, c, abort);
    }

    // backward step u processes local plane t = last - u
    auto issue = [&](int uu) {
      if (uu < g.nsteps) {
        const int t = last - uu;
        const int i = t - g.dj - g.dk;
        const bool v = g.col && i >= 0 && i < B.nx;
        const long long a = v ? B.cell0 + rbk[g.s0 + t] + g.j : 0;
        T *st = sm.stage + (size_t)(uu % R) * NV * NT + tid;
        cp_async_zfill<EB>(st, P.ue + a, v);
        cp_async_zfill<EB>(st + NT, P.un + a, v);
        cp_async_zfill<EB>(st + 2 * NT, P.ut + a, v);
        cp_async_zfill<EB>(st + 3 * NT, P.y + a, v);
        if constexpr (!ZX) cp_async_zfill<EB>(st + 4 * NT, P.x + a, v);
        if constexpr (UPD64) {
          double *s64 = reinterpret_cast<double *>(sm.stage + (size_t)(uu % R) * NV * NT + (NV - 2) * NT) + tid;
          cp_async_zfill<8>(s64, P.x64 + a, v);
        }
        uint64_t *fs = sm.fst + (size_t)(uu % R) * FS * W;
        if (cJ && v) rec_prefetch<W>(fs + g.dk * W, faceJ(dnJ, B, t - (B.TJ - 1), g.dk, W));
        if (cK && v) rec_prefetch<W>(fs + (B.TK + g.dj) * W, faceK(dnK, B, t - (B.TK - 1), g.dj, W));
      }
      cp_async_commit();
    };
#pragma unroll
    for (int uu = 0; uu < R - 1; ++uu) issue(uu);

    T dE = 0;
    for (int u = 0; u < g.nsteps; ++u) {
      issue(u + R - 1);
      cp_async_wait<R - 1>();
      const T *st = sm.stage + (size_t)(u % R) * NV * NT + tid;
      const uint64_t *fs = sm.fst + (size_t)(u % R) * FS * W;
      const int t = last - u;
      const int i = t - g.dj - g.dk;
      const bool act = g.col && i >= 0 && i < B.nx;
      T *E = sm.exch + (size_t)(u & 1) * EC;
      E[me] = dE;
      if (g.dj == B.TJ - 1) {
        uint64_t w[W] = {0, 0};
        if (act && cJ) rec_take<W>(fs + g.dk * W, faceJ(dnJ, B, t - (B.TJ - 1), g.dk, W), expect, w, c, abort);
        E[me + 1] = Face<T>::get(w);
      }
      if (g.dk == B.TK - 1) {
        uint64_t w[W] = {0, 0};
        if (act && cK)
          rec_take<W>(fs + (B.TK + g.dj) * W, faceK(dnK, B, t - (B.TK - 1), g.dj, W), expect, w, c, abort);
        E[me + TJ2] = Face<T>::get(w);
      }
      __syncthreads();
      const T dN = E[me + 1], dT = E[me + TJ2];
      T d = fma(-st[0], dE, st[3 * NT]);
      d = fma(-st[NT], dN, d);
      d = fma(-st[2 * NT], dT, d);
      if (act) {
        const long long a = B.cell0 + rbk[g.s0 + t] + g.j;
        T xn = d;
        if constexpr (!ZX) xn = st[4 * NT] + d;
        if constexpr (UPD64) {
          const double *s64 =
              reinterpret_cast<const double *>(sm.stage + (size_t)(u % R) * NV * NT + (NV - 2) * NT) + tid;
          P.x64[a] = *s64 + (double)xn;
        } else {
          P.x[a] = xn;
        }
        if (g.dj == 0 && g.hasS) Face<T>::put(faceJ(myf, B, t, g.dk, W), d, ep);
        if (g.dk == 0 && g.hasB) Face<T>::put(faceK(myf, B, t, g.dj, W), d, ep);
      }
      dE = act ? d : T(0);
    }
    cp_async_wait<0>();
    __syncthreads();
  }
}

// ======================================================= FP64 residual (refinement)
// r = b - A x in FP64 arithmetic (A stored as TA, widened), sum r^2 per tile,
// r32 = (float) r.  No recurrence: every tile is independent.
template <typename TA, bool SYM, int R>
__global__ void __launch_bounds__(512) k_resid(ResParams<TA> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_red[32];
  constexpr int NA = SYM ? 4 : 7;
  constexpr int ND = 4;           // b xp1 hxj hxk
  constexpr int NS = SYM ? 2 : 0; // hanS hatB (TA)
  if (__syncthreads_or(P.ctl->done || ld_relaxed(P.status) != DEV_OK)) return;
  const int NT = blockDim.x, tid = threadIdx.x;
  double *sd = reinterpret_cast<double *>(smem_raw);           // [R][ND][NT]
  TA *sa = reinterpret_cast<TA *>(sd + (size_t)R * ND * NT);   // [R][NA+NS][NT]
  const size_t sa_bytes = ((size_t)R * (NA + NS) * NT * sizeof(TA) + 15) & ~(size_t)15;
  double *exch = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(sa) + sa_bytes);
  const int EC = P.exch_cells;
  constexpr int NE = SYM ? 4 : 2;  // xm1 xp1 (anm1 atm1)
  constexpr int EBA = (int)sizeof(TA);
  const TA *src[NA];
  if constexpr (SYM) {
    src[0] = P.ap; src[1] = P.ae; src[2] = P.an; src[3] = P.at;
  } else {
    src[0] = P.ap; src[1] = P.aw; src[2] = P.ae; src[3] = P.as;
    src[4] = P.an; src[5] = P.ab; src[6] = P.at;
  }

  for (int m = blockIdx.x; m < P.ntiles; m += gridDim.x) {
    const Tile tl = P.tiles[m];
    const DevBlock B = P.blocks[tl.blk];
    const ColGeom g(B, tl);
    const int *rbk = B.rbT + (long long)min(g.k, B.nz - 1) * B.nplanes;
    const int *rbkB = B.rbT + (long long)max(g.k - 1, 0) * B.nplanes;
    const int *rbkT = B.rbT + (long long)min(g.k + 1, B.nz - 1) * B.nplanes;
    const int TJ2 = B.TJ + 2;
    const int me = (g.dk + 1) * TJ2 + g.dj + 1;
    const bool eS = g.dj == 0, eN = g.dj == B.TJ - 1, eB = g.dk == 0, eT = g.dk == B.TK - 1;

    auto issue = [&](int tt) {
      if (tt < g.nsteps) {
        const int i = tt - g.dj - g.dk;
        const int s = g.s0 + tt;
        const bool v = g.col && i >= 0 && i < B.nx;
        const long long a = v ? B.cell0 + rbk[s] + g.j : 0;
        double *d = sd + (size_t)(tt % R) * ND * NT + tid;
        TA *q = sa + (size_t)(tt % R) * (NA + NS) * NT + tid;
#pragma unroll
        for (int z = 0; z < NA; ++z) cp_async_zfill<EBA>(q + z * NT, src[z] + a, v);
        cp_async_zfill<8>(d, P.b + a, v);
        const bool vp = g.col && i + 1 >= 0 && i + 1 < B.nx;
        const long long ap1 = vp ? B.cell0 + rbk[s + 1] + g.j : 0;
        cp_async_zfill<8>(d + NT, P.x + ap1, vp);
        long long hj = 0;
        bool vj = false;
        if (eS && g.hasS && v) { hj = B.cell0 + rbk[s - 1] + g.j0 - 1; vj = true; }
        else if (eN && g.hasN && v) { hj = B.cell0 + rbk[s + 1] + g.j0 + B.TJ; vj = true; }
        cp_async_zfill<8>(d + 2 * NT, P.x + hj, vj);
        long long hk = 0;
        bool vk = false;
        if (eB && g.hasB && v) { hk = B.cell0 + rbkB[s - 1] + g.j; vk = true; }
        else if (eT && g.hasT && v) { hk = B.cell0 + rbkT[s + 1] + g.j; vk = true; }
        cp_async_zfill<8>(d + 3 * NT, P.x + hk, vk);
        if constexpr (SYM) {
          cp_async_zfill<EBA>(q + NA * NT, P.an + hj, vj && eS);
          cp_async_zfill<EBA>(q + (NA + 1) * NT, P.at + hk, vk && eB);
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int tt = 0; tt < R - 1; ++tt) issue(tt);

    double xm1 = 0, x0 = 0, aem1 = 0, anm1 = 0, atm1 = 0, acc = 0;
    if (g.dj == 0 && g.dk == 0 && g.col) x0 = P.x[B.cell0 + rbk[g.s0] + g.j];
    for (int t = 0; t < g.nsteps; ++t) {
      issue(t + R - 1);
      cp_async_wait<R - 1>();
      const double *d = sd + (size_t)(t % R) * ND * NT + tid;
      const TA *q = sa + (size_t)(t % R) * (NA + NS) * NT + tid;
      const int i = t - g.dj - g.dk;
      const bool act = g.col && i >= 0 && i < B.nx;
      double *E = exch + (size_t)(t & 1) * NE * EC;
      const double xp1 = d[NT];
      E[me] = xm1;
      E[EC + me] = xp1;
      if constexpr (SYM) {
        E[2 * EC + me] = anm1;
        E[3 * EC + me] = atm1;
      }
      if (eS) {
        E[me - 1] = d[2 * NT];
        if constexpr (SYM) E[2 * EC + me - 1] = (double)q[NA * NT];
      }
      if (eN) E[EC + me + 1] = d[2 * NT];
      if (eB) {
        E[me - TJ2] = d[3 * NT];
        if constexpr (SYM) E[3 * EC + me - TJ2] = (double)q[(NA + 1) * NT];
      }
      if (eT) E[EC + me + TJ2] = d[3 * NT];
      __syncthreads();
      const double xS = E[me - 1], xN = E[EC + me + 1], xB = E[me - TJ2], xT = E[EC + me + TJ2];
      double r = d[0];
      if constexpr (SYM) {
        const double ap = q[0], ae = q[NT], an = q[2 * NT], at = q[3 * NT];
        r = fma(-ap, x0, r);
        r = fma(-aem1, xm1, r);
        r = fma(-ae, xp1, r);
        r = fma(-E[2 * EC + me - 1], xS, r);
        r = fma(-an, xN, r);
        r = fma(-E[3 * EC + me - TJ2], xB, r);
        r = fma(-at, xT, r);
        aem1 = ae;
        anm1 = an;
        atm1 = at;
      } else {
        r = fma(-(double)q[0], x0, r);
        r = fma(-(double)q[NT], xm1, r);
        r = fma(-(double)q[2 * NT], xp1, r);
        r = fma(-(double)q[3 * NT], xS, r);
        r = fma(-(double)q[4 * NT], xN, r);
        r = fma(-(double)q[5 * NT], xB, r);
        r = fma(-(double)q[6 * NT], xT, r);
      }
      acc = fma(r, r, acc);
      if (act) P.r32[B.cell0 + rbk[g.s0 + t] + g.j] = (float)r;
      xm1 = x0;
      x0 = xp1;
    }
    cp_async_wait<0>();
    const double tot = block_sum(acc, s_red);
    if (tid == 0) P.partials[tl.gtile] = tot;
    __syncthreads();
  }
}

}  // namespace sipk
