// sip_sweeps.cuh -- sm_103a kernels of Stone's SIP over the plane layout.
//
// The recurrences of the method (arXiv:1303.4538, Sec. 1 / Sec. 4.1: lu3d,
// the substitution part of resforward3d, backward3d) make a cell depend on
// its lower neighbours W, S, B (factorisation and forward substitution) or on
// its upper neighbours E, N, T (backward substitution).  The residual part of
// resforward3d has no recurrence and runs in the row-parallel kernel of
// sip_resrow.cu.  All cells of one hyperplane i + j + k = s are
// independent, so the sweeps advance plane by plane.  Work decomposition:
//
//   * the (j, k) cross-section of a block is cut into 32 x TK column tiles;
//     one CTA owns a tile; lane = j, and warp w owns the Q rows
//     k = k0 + w Q .. k0 + w Q + Q - 1, so a thread walks Q columns along i.
//     At local step t every cell the CTA touches lies on plane s = t + j0 + k0;
//   * neighbours of the previous (next) plane: W/E from the thread's own
//     registers, S/N from lanes j -+ 1 by warp shuffles, B/T from the
//     thread's own neighbouring row, and across warps through a
//     shared-memory exchange with one slot per stage (one barrier per step);
//   * each cell's static data (factors, or A for the factorisation) is one
//     16-byte aligned record, staged with cp.async.cg (L2 only) R-1 steps
//     ahead into a ring of shared-memory stages together with the cell's
//     values (r; y and x for the backward sweep); invalid
//     cells are zero-filled, so the arithmetic runs without branches and
//     inactive threads produce zeros;
//   * row addresses come from two small per-block tables held in shared
//     memory (plane offsets PO and the diagonal prefix sums F);
//   * between tiles, the recurrence's boundary values travel through "faces":
//     16-byte records of two 8-byte words whose upper halves carry the
//     launch's epoch tag.  A producer stores a record with one st.relaxed.gpu;
//     a consumer prefetches it with cp.async.cg with the step's other data and
//     accepts it when every tag matches (each word is self-validating, so no
//     fence or flag is needed); a stale record is re-read from L2 with
//     ld.relaxed.gpu until it matches.  Before a tile starts, one thread waits
//     until the upstream tiles are a few steps ahead ("slack"), so prefetched
//     records are normally valid.  Every wait is bounded (max_spin polls),
//     then the kernel records DEV_TIMEOUT and runs to the end without waiting;
//   * CTAs claim tiles with an atomic ticket in a dependency-respecting order,
//     so a tile only waits for tiles claimed earlier by running CTAs.
// This file holds the shared machinery and the forward and backward
// substitutions; the factorisation kernel is in sip_factor.cuh.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

#include "sip_internal.h"
#include "sip_layout.h"

namespace sipk {

// Compile-time loop: f(std::integral_constant<int, U>{}) for U = B .. E - 1.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

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
__device__ __forceinline__ void cp_async_16_l2(void *sdst, const void *gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}
// The same copies without a compiler memory clobber, for the substitution
// sweeps: there a stage slot is written only by these copies and read only
// after the step's cp.async.wait_group (which keeps its clobber) and CTA
// barrier, and every step ends with the face stores (asm with a clobber,
// executed by every thread), so no load of a slot can move past the copy
// that refills it.  Without the clobber the compiler may interleave the
// next stage's address arithmetic with the current step's shared loads.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill_nc(void *sdst, const void *gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(sdst)), "l"(gsrc), "n"(BYTES),
               "r"(valid ? BYTES : 0));
}
__device__ __forceinline__ void cp_async_16_l2_nc(void *sdst, const void *gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_16_if_nc(void *sdst, const void *gsrc, bool pred) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"((int)pred));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2(uint64_t *p, uint64_t a, uint64_t b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
// predicated forms (no branch in the caller): nothing happens when !pred
__device__ __forceinline__ void st_relaxed_v2_if(uint64_t *p, uint64_t a, uint64_t b, bool pred) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %3, 0;\n @q st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};\n}\n" ::"l"(p),
      "l"(a), "l"(b), "r"((int)pred)
      : "memory");
}
__device__ __forceinline__ void cp_async_16_if(void *sdst, const void *gsrc, bool pred) {
  asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"((int)pred)
               : "memory");
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

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) {
  return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
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
  __device__ static void put_if(uint64_t *p, float v, unsigned ep, bool pred) {
    const uint64_t tag = (uint64_t)ep << 32;
    st_relaxed_v2_if(p, tag | (uint64_t)__float_as_uint(v), tag, pred);
  }
  // two values in one record (one per word): the J faces of a thread's row pair
  __device__ static void put2_if(uint64_t *p, float a, float b, unsigned ep, bool pred) {
    const uint64_t tag = (uint64_t)ep << 32;
    st_relaxed_v2_if(p, tag | (uint64_t)__float_as_uint(a), tag | (uint64_t)__float_as_uint(b), pred);
  }
  __device__ static float get_hi(const uint64_t *w) { return __uint_as_float((unsigned)w[1]); }
  __device__ static float get(const uint64_t *w) { return __uint_as_float((unsigned)w[0]); }
};
template <>
struct Face<double> {
  __device__ static void put(uint64_t *p, double v, unsigned ep) {
    const uint64_t tag = (uint64_t)ep << 32;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_relaxed_v2(p, tag | (b & 0xffffffffull), tag | (b >> 32));
  }
  __device__ static void put_if(uint64_t *p, double v, unsigned ep, bool pred) {
    const uint64_t tag = (uint64_t)ep << 32;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_relaxed_v2_if(p, tag | (b & 0xffffffffull), tag | (b >> 32), pred);
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

// Poll a W-word record in L2 until every tag equals `expect`.  Gives up
// (zero words, abort set) after max_spin polls or once another thread
// recorded an error.  The slow path is kept out of line and returns its
// words by value: a caller's record array whose address reached an
// out-of-line call would have to live in local memory on the fast path too.
template <int W>
struct Polled {
  uint64_t w[W];
  bool abort;
};
template <int W>
__device__ __noinline__ Polled<W> face_poll(const uint64_t *p, unsigned expect, const SweepCommon &c, bool abort,
                                            unsigned long long *tr) {
  Polled<W> o;
  o.abort = abort;
  if (!abort) {
    long long spins = 0;
    const unsigned long long t0 = tr ? gtimer() : 0ull;
    for (;;) {
#pragma unroll
      for (int q = 0; q < W; ++q) o.w[q] = ld_relaxed(p + q);
      if (rec_ok<W>(o.w, expect)) {
        if (tr) {
          atomicAdd(tr + 3, 1ull);
          atomicAdd(tr + 4, gtimer() - t0);
        }
        return o;
      }
      ++spins;
      if (spins > c.max_spin) {
        atomicCAS(c.status, DEV_OK, DEV_TIMEOUT);
        o.abort = true;
        break;
      }
      if ((spins & 63) == 0 && ld_relaxed(c.status) != DEV_OK) {
        o.abort = true;
        break;
      }
      __nanosleep(32);
    }
  }
#pragma unroll
  for (int q = 0; q < W; ++q) o.w[q] = 0;
  return o;
}

// Returns false (and zero words) when the wait gave up; `abort` then stays
// set so this thread never waits again.
template <int W>
__device__ __forceinline__ bool face_wait(const uint64_t *p, unsigned expect, uint64_t (&w)[W],
                                          const SweepCommon &c, bool &abort, unsigned long long *tr) {
  const Polled<W> o = face_poll<W>(p, expect, c, abort, tr);
#pragma unroll
  for (int q = 0; q < W; ++q) w[q] = o.w[q];
  abort = o.abort;
  return !o.abort;
}

// Take the record staged in shared memory; re-read it from L2 if it is stale.
template <int W>
__device__ __forceinline__ void rec_take(const uint64_t *staged, const uint64_t *g, unsigned expect,
                                         uint64_t (&w)[W], const SweepCommon &c, bool &abort,
                                         unsigned long long *tr) {
#pragma unroll
  for (int q = 0; q < W; ++q) w[q] = staged[q];
  if (!rec_ok<W>(w, expect)) face_wait<W>(g, expect, w, c, abort, tr);
}

template <int W>
__device__ __forceinline__ void rec_prefetch(uint64_t *sdst, const uint64_t *g) {
#pragma unroll
  for (int q = 0; q < W; q += 2) cp_async_16_l2(sdst + q, g + q, true);
}

// The two words of a face record staged in shared memory (one 16-byte load).
__device__ __forceinline__ void staged_words(const uint64_t *staged, uint64_t (&w)[2]) {
  const ulonglong2 s2 = *reinterpret_cast<const ulonglong2 *>(staged);
  w[0] = s2.x;
  w[1] = s2.y;
}

// The same, only where `pred` holds (zero words elsewhere): a predicated
// load instead of a branch around it.
__device__ __forceinline__ void staged_words_if(const uint64_t *staged, uint64_t (&w)[2], bool pred) {
  unsigned long long a = 0, b = 0;
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p ld.shared.v2.u64 {%0, %1}, [%2];\n}\n"
               : "+l"(a), "+l"(b)
               : "r"(smem_u32(staged)), "r"((int)pred));
  w[0] = a;
  w[1] = b;
}

// Row bases of a warp's Q rows for C = 32 / Q consecutive steps, one per
// lane: lane l holds the base of row k0 + w Q + l % Q on local plane t of
// step `first + l / Q` (0 where that plane row does not exist).  A step's
// bases are then fetched with one shuffle per row.
template <int Q>
__device__ __forceinline__ int rowbase_chunk(const DevBlock &B, const int *sPO, const int *sF, int s0, int k,
                                             int t, int nsteps) {
  const int s = s0 + t, m = s - k;
  const bool ok = t >= 0 && t < nsteps && k < B.nz && m >= 0 && m <= B.mmax;
  return ok ? plane_row_base(sPO, sF, B.mmax, B.nx, s, k) : 0;
}

// Face storage of one tile: J face [nsteps_max][TK][W], then K face
// [nsteps_max][32][W], indexed by the producer's local step.
__device__ __forceinline__ uint64_t *tile_faces(const SweepCommon &c, const DevBlock &B, int gtile) {
  return c.faces + B.face0 + (long long)(gtile - B.tile0) * B.face_tile_words;
}
__device__ __forceinline__ uint64_t *faceJ(uint64_t *base, const DevBlock &B, int t, int lane, int W) {
  return base + ((long long)t * B.TK + lane) * W;
}
__device__ __forceinline__ uint64_t *faceK(uint64_t *base, const DevBlock &B, int t, int lane, int W) {
  return base + (long long)B.nsteps_max * B.TK * W + ((long long)t * kTJ + lane) * W;
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

// Copy the block's PO and F tables into shared memory when the CTA moves to a
// tile of another block (block-uniform: s_blk is read after a barrier).
__device__ __forceinline__ void load_tables(const DevBlock &B, int blk, int *sPO, int *s_blk) {
  if (*s_blk != blk) {
    for (int q = threadIdx.x; q < B.nplanes; q += blockDim.x) sPO[q] = B.PO[q];
    int *sF = sPO + B.nplanes;
    for (int q = threadIdx.x; q <= B.mmax; q += blockDim.x) sF[q] = B.F[q];
    __syncthreads();
    if (threadIdx.x == 0) *s_blk = blk;
  }
}

// Geometry of the calling thread inside tile (cj, ck): lane = j - j0,
// warp w owns rows k0 + w Q + q.
template <int Q>
struct Geo {
  int lane, w, NW, TK, j0, k0, j, s0, nsteps, njt, nkt;
  bool jok, hasS, hasN, hasB, hasT, eB, eT;
  __device__ Geo(const DevBlock &B, const Tile &tl) {
    lane = threadIdx.x & 31;
    w = threadIdx.x >> 5;
    NW = blockDim.x >> 5;
    TK = NW * Q;
    j0 = tl.cj * kTJ;
    k0 = tl.ck * TK;
    j = j0 + lane;
    jok = j < B.ny;
    njt = min(kTJ, B.ny - j0);
    nkt = min(TK, B.nz - k0);
    nsteps = B.nx + njt + nkt - 2;
    s0 = j0 + k0;
    hasS = j0 > 0;
    hasN = j0 + kTJ < B.ny;
    hasB = k0 > 0;
    hasT = k0 + TK < B.nz;
    eB = w == 0;
    eT = w == NW - 1;
  }
  __device__ int k(int q) const { return k0 + w * Q + q; }
  __device__ int dk(int q) const { return w * Q + q; }
  __device__ bool col(const DevBlock &B, int q) const { return jok && k(q) < B.nz; }
  __device__ int i(int t, int q) const { return t - lane - dk(q); }
};

// Slack gate: before a tile starts, wait until the records that the tile will
// consume `lead` steps after its first need are published, so the records
// prefetched during the walk are normally already valid.
template <int W>
__device__ __forceinline__ void slack_gate(const uint64_t *recJ, const uint64_t *recK, unsigned expect,
                                           const SweepCommon &c, bool &abort, unsigned long long *tr) {
  if (threadIdx.x == 0) {
    uint64_t w[W];
    if (tr) {
      tr[0] = gtimer();
      tr[5] = smid();
    }
    if (recJ) face_wait<W>(recJ, expect, w, c, abort, nullptr);
    if (recK) face_wait<W>(recK, expect, w, c, abort, nullptr);
    if (tr) tr[1] = gtimer();
  }
  __syncwarp();  // thread 0's wait diverges its warp: reconverge before the CTA barrier
  __syncthreads();
}

template <typename T, int N>
struct Vec {
  T v[N];
};

// J face records carry one row's value, or in FP32 a row pair's (one value
// per 8-byte word), so a warp moves Q/2 records per step instead of Q.
template <typename T, int Q>
__host__ __device__ constexpr int face_pair() {
  return (sizeof(T) == 4 && Q % 2 == 0) ? 2 : 1;
}
template <typename T, int PJ>
__device__ __forceinline__ T face_row(const uint64_t (&w)[2], int q) {
  if constexpr (PJ == 2) return (q & 1) ? Face<T>::get_hi(w) : Face<T>::get(w);
  else return Face<T>::get(w);
}
template <typename T, int PJ, int Q>
__device__ __forceinline__ void face_put(uint64_t *p, const T (&v)[Q], int q, unsigned ep, bool pred) {
  if constexpr (PJ == 2) Face<T>::put2_if(p, v[q], v[q + 1], ep, pred);
  else Face<T>::put_if(p, v[q], ep, pred);
}

// ============================================================ forward sweep
// The substitution half of resforward3d: y = L^{-1} r with
//   y_P = (r_P - LB y_B - LW y_W - LS y_S) * (1/LP),  ascending planes.
// The residual r = b - A x (and its norm) is computed beforehand by the
// row-parallel kernel, so the wavefront carries only this recurrence.  r and y
// may alias (in place): a cell's r is staged before its y is stored, and no
// other cell reads it.
//
// Per step a thread issues the copies of step t + R - 1 (row bases from the
// warp's row-base chunk, one shuffle per row; the cell offsets are kept in the
// stage for the store) and computes step t from its stage.
template <typename T, int Q, int R>
__global__ void __launch_bounds__(512, 1) k_forward(FwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim, s_blk;
  constexpr int W = 2;
  constexpr int RBY = 4 * (int)sizeof(T);  // bytes of an L record
  constexpr int C = 32 / Q;                // steps per row-base chunk
  constexpr int PJ = face_pair<T, Q>();    // rows per J face record
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  if (threadIdx.x == 0) s_blk = -1;
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(c.ctl->done || ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const SweepLayout L = fwd_layout((int)sizeof(T), Q, R, NT, c.tab_ints);
  int *sPO = reinterpret_cast<int *>(smem_raw);
  unsigned char *stage = smem_raw + L.tab;
  T *exB = reinterpret_cast<T *>(stage + (size_t)R * L.step);  // [R][NW][32]: y of a warp's last row
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
    const int NW = g.NW, lane = g.lane, w = g.w, TK = g.TK;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *upJ = g.hasS ? tile_faces(c, B, tl.gtile - 1) : myf;
    uint64_t *upK = g.hasB ? tile_faces(c, B, tl.gtile - B.nTJ) : myf;
    {
      const int lead = min(sweep_lead((int)sizeof(T)), B.nx - 1);
      slack_gate<W>(g.hasS ? faceJ(upJ, B, lead + kTJ - 1, 0, W) : nullptr,
                    g.hasB ? faceK(upK, B, lead + TK - 1, 0, W) : nullptr, expect, c, abort, tr);
    }
    // per-row invariants: cell of row q at local step t is i = t - tlo[q]
    int tlo[Q];
    bool colq[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      tlo[q] = lane + g.dk(q);
      colq[q] = g.col(B, q);
    }
    const unsigned nxu = (unsigned)B.nx;
    const long long kface = (long long)B.nsteps_max * TK * W;  // K faces follow the J faces
    int chunk = 0, cb = -C;  // row-base chunk of issue steps [cb, cb + C)
    const int kchunk = g.k0 + w * Q + lane % Q;
    // the block's arrays (cell offsets inside a block fit in 32 bits; a
    // record offset, 4 values a cell, is scaled in 64 bits)
    const T *recb = P.rec + B.cell0 * 4;
    const T *rb = P.r + B.cell0;
    T *yb = P.y + B.cell0;
    // face records read by the copies of issue step tt (the producers' steps
    // tt + kTJ - 1 and tt + TK - 1) and written at compute step t (row slot
    // w Q; K slot lane): per-tile bases plus 32-bit step offsets, computed
    // from the step (no pointer carried from step to step)
    const uint64_t *fjb = upJ + ((long long)(kTJ - 1) * TK + w * Q) * W;
    const uint64_t *fkb = upK + kface + ((long long)(TK - 1) * kTJ + lane) * W;
    uint64_t *pjb = myf + (long long)w * Q * W;
    uint64_t *pkb = myf + kface + (long long)lane * W;
    const int TKW = TK * W, TJW = kTJ * W;

    // Step t uses stage slot, exchange slot and store-offset registers
    // t % R: the step loop is unrolled by R, so every slot index is a
    // compile-time constant and the offsets never leave registers.
    int offr[R][Q];
    auto issue = [&](int tt, auto slot) {
      constexpr int sl = decltype(slot)::value;
      // past the last step every copy is predicated off (no cell is valid)
      {
        if (tt - cb >= C) {
          cb += C;
          chunk = rowbase_chunk<Q>(B, sPO, sF, g.s0, kchunk, cb + lane / Q, g.nsteps);
        }
        unsigned char *st = stage + (size_t)sl * L.step;
        T *sr = reinterpret_cast<T *>(st + L.rec) + tid;
        uint64_t *fs = fst + (size_t)sl * FS * W;
        // addresses of every row first, then the copies
        bool v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          offr[sl][q] = __shfl_sync(0xffffffffu, chunk, (tt - cb) * Q + q) + g.j;
          v[q] = colq[q] && (unsigned)(tt - tlo[q]) < nxu;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int o = v[q] ? offr[sl][q] : 0;
          unsigned char *d = st + ((size_t)q * NT + tid) * RBY;
          const unsigned char *src = reinterpret_cast<const unsigned char *>(recb + (size_t)o * 4);
#pragma unroll
          for (int z = 0; z < RBY / 16; ++z) cp_async_16_l2_nc(d + 16 * z, src + 16 * z, v[q]);
          cp_async_zfill_nc<sizeof(T)>(sr + q * NT, rb + o, v[q]);
        }
#pragma unroll
        for (int q = 0; q < Q; q += PJ) {
          const bool vq = PJ == 2 ? (v[q] || v[q + PJ - 1]) : v[q];
          cp_async_16_if_nc(fs + (w * Q + q) * W, fjb + tt * TKW + q * W, lane == 0 && g.hasS && vq);
        }
        cp_async_16_if_nc(fs + (TK + lane) * W, fkb + tt * TJW, g.eB && g.hasB && v[0]);
      }
      cp_async_commit();
    };
    static_for<0, R - 1>([&](auto u) { issue(decltype(u)::value, u); });

    T ym1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) ym1[q] = T(0);
    // the walk is padded to a multiple of R steps: the extra steps touch no
    // cell (every copy, store and face store is predicated off), so the
    // unrolled body needs no exit test
    for (int t0 = 0; t0 < g.nsteps; t0 += R) {
      static_for<0, R>([&](auto uc) {
        constexpr int sl = decltype(uc)::value;
        const int t = t0 + sl;
        issue(t + R - 1, std::integral_constant<int, (sl + R - 1) % R>{});
        cp_async_wait<R - 1>();
        const unsigned char *st = stage + (size_t)sl * L.step;
        const T *sr = reinterpret_cast<const T *>(st + L.rec) + tid;
        const uint64_t *fs = fst + (size_t)sl * FS * W;
        T *E = exB + (size_t)sl * NW * 32;
        E[w * 32 + lane] = ym1[Q - 1];
        __syncthreads();
        // faces of this step: J (lane 0, one record per row, or per row pair
        // in FP32) and K (warp 0, row 0); a stale staged copy is re-read from
        // L2 (rare: one warp-uniform branch)
        bool act[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) act[q] = colq[q] && (unsigned)(t - tlo[q]) < nxu;
        constexpr int NJ = Q / PJ;
        bool needJ[NJ];
        uint64_t jw[NJ][2], kw[2] = {0, 0};
        bool stale = false;
#pragma unroll
        for (int r = 0; r < NJ; ++r) {
          const int q = r * PJ;
          needJ[r] = lane == 0 && g.hasS && (PJ == 2 ? (act[q] || act[q + PJ - 1]) : act[q]);
          staged_words(fs + (w * Q + q) * W, jw[r]);
          stale |= needJ[r] && !rec_ok<2>(jw[r], expect);
        }
        const bool needK = g.eB && g.hasB && act[0];
        staged_words_if(fs + (TK + lane) * W, kw, g.eB);
        stale |= needK && !rec_ok<2>(kw, expect);
        if (__any_sync(0xffffffffu, stale)) {
#pragma unroll
          for (int r = 0; r < NJ; ++r)
            if (needJ[r] && !rec_ok<2>(jw[r], expect))
              face_wait<2>(upJ + ((long long)(t + kTJ - 1) * TK + w * Q + r * PJ) * W, expect, jw[r], c, abort, tr);
          if (needK && !rec_ok<2>(kw, expect))
            face_wait<2>(upK + kface + ((long long)(t + TK - 1) * kTJ + lane) * W, expect, kw, c, abort, tr);
        }
        const T yK = needK ? Face<T>::get(kw) : T(0);
        T ny[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const T *rec = reinterpret_cast<const T *>(st + ((size_t)q * NT + tid) * RBY);
          const T r = sr[q * NT];
          T yS = shfl_up1(ym1[q]);
          if (lane == 0) yS = (g.hasS && act[q]) ? face_row<T, PJ>(jw[q / PJ], q) : T(0);
          T yB;
          if (q > 0) yB = ym1[q > 0 ? q - 1 : 0];
          else if (w > 0) yB = E[(w - 1) * 32 + lane];
          else yB = yK;
          T y = fma(-rec[REC_LB], yB, r);
          y = fma(-rec[REC_LW], ym1[q], y);
          y = fma(-rec[REC_LS], yS, y);
          ny[q] = act[q] ? y * rec[REC_RLP] : T(0);
        }
        // stores last: y, then the face records (ordered memory operations)
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (act[q]) yb[offr[sl][q]] = ny[q];
#pragma unroll
        for (int q = 0; q < Q; q += PJ)
          face_put<T, PJ>(pjb + t * TKW + q * W, ny, q, ep,
                          lane == kTJ - 1 && g.hasN && (PJ == 2 ? (act[q] || act[q + PJ - 1]) : act[q]));
        Face<T>::put_if(pkb + t * TJW, ny[Q - 1], ep, g.eT && g.hasT && act[Q - 1]);
#pragma unroll
        for (int q = 0; q < Q; ++q) ym1[q] = ny[q];
      });
    }
    cp_async_wait<0>();
    if (tr && threadIdx.x == 0) tr[2] = gtimer();
    __syncthreads();
  }
}

// =========================================================== backward sweep
// backward3d with the update: d_P = y_P - UE d_E - UN d_N - UT d_T
// (descending planes), x_P <- x_P + d_P.  ZX: x = 0 on entry (x_P <- d_P).
// Backward step u processes local plane t = last - u.
template <typename T, bool ZX, int Q, int R>
__global__ void __launch_bounds__(512, 1) k_backward(BwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_claim, s_blk;
  constexpr int W = 2;
  constexpr int RBY = 4 * (int)sizeof(T);  // bytes of a U record
  constexpr int C = 32 / Q;
  constexpr int SY = 0, SX = Q;  // scalar slots
  constexpr int PJ = face_pair<T, Q>();  // rows per J face record
  const SweepCommon &c = P.c;
  const unsigned ep = sweep_prologue(c);
  if (threadIdx.x == 0) s_blk = -1;
  // block-uniform exit decision (the status word may change during the launch)
  if (__syncthreads_or(c.ctl->done || ld_relaxed(c.status) != DEV_OK)) return;
  const unsigned expect = ep + (c.stall ? 0x40000000u : 0u);
  const int NT = blockDim.x, tid = threadIdx.x;
  const SweepLayout L = bwd_layout((int)sizeof(T), ZX, Q, R, NT, c.tab_ints);
  int *sPO = reinterpret_cast<int *>(smem_raw);
  unsigned char *stage = smem_raw + L.tab;
  T *exT = reinterpret_cast<T *>(stage + (size_t)R * L.step);  // [R][NW][32]: d of a warp's first row
  uint64_t *fst = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(exT) + L.exch);
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
    const int NW = g.NW, lane = g.lane, w = g.w, TK = g.TK;
    uint64_t *myf = tile_faces(c, B, tl.gtile);
    uint64_t *dnJ = g.hasN ? tile_faces(c, B, tl.gtile + 1) : myf;
    uint64_t *dnK = g.hasT ? tile_faces(c, B, tl.gtile + B.nTJ) : myf;
    const int last = g.nsteps - 1;
    {
      // the consumer of the last valid row (column) needs, `lead` steps into
      // the walk, cell i = nx-1-lead, published on the producer's step i + lane
      const int lead = min(sweep_lead((int)sizeof(T)), B.nx - 1);
      const int i = B.nx - 1 - lead;
      // (J records of row pairs sit in the slot of the pair's first row)
      slack_gate<W>(g.hasN ? faceJ(dnJ, B, i + g.nkt - 1, (g.nkt - 1) / PJ * PJ, W) : nullptr,
                    g.hasT ? faceK(dnK, B, i + g.njt - 1, g.njt - 1, W) : nullptr, expect, c, abort, tr);
    }
    int tlo[Q];
    bool colq[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      tlo[q] = lane + g.dk(q);
      colq[q] = g.col(B, q);
    }
    const unsigned nxu = (unsigned)B.nx;
    const long long kface = (long long)B.nsteps_max * TK * W;
    int chunk = 0, cb = -C;  // row-base chunk of issue steps [cb, cb + C)
    const int kchunk = g.k0 + w * Q + lane % Q;
    const T *recb = P.rec + B.cell0 * 4;
    const T *yb = P.y + B.cell0;
    T *xb = P.x + B.cell0;
    // face records (descending planes) read by the copies of issue step uu
    // (plane t = last - uu: the producers' steps t - (kTJ - 1) and
    // t - (TK - 1)) and written at step u (plane last - u): per-tile bases
    // plus 32-bit step offsets (negative past the walk's end, where every
    // copy and store is predicated off)
    const uint64_t *fjb = dnJ + ((long long)(-(kTJ - 1)) * TK + w * Q) * W;
    const uint64_t *fkb = dnK + kface + ((long long)(-(TK - 1)) * kTJ + lane) * W;
    uint64_t *pjb = myf + (long long)w * Q * W;
    uint64_t *pkb = myf + kface + (long long)lane * W;
    const int TKW = TK * W, TJW = kTJ * W;

    // slots as in the forward sweep: stage, exchange and offsets of step u
    // at u % R, the loop unrolled by R
    int offr[R][Q];
    auto issue = [&](int uu, auto slot) {
      constexpr int sl = decltype(slot)::value;
      // past the last step every copy is predicated off (no cell is valid)
      {
        if (uu - cb >= C) {
          cb += C;
          chunk = rowbase_chunk<Q>(B, sPO, sF, g.s0, kchunk, last - (cb + lane / Q), g.nsteps);
        }
        const int t = last - uu;
        unsigned char *st = stage + (size_t)sl * L.step;
        T *sc = reinterpret_cast<T *>(st + L.rec) + tid;
        uint64_t *fs = fst + (size_t)sl * FS * W;
        bool v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          offr[sl][q] = __shfl_sync(0xffffffffu, chunk, (uu - cb) * Q + q) + g.j;
          v[q] = colq[q] && (unsigned)(t - tlo[q]) < nxu;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int o = v[q] ? offr[sl][q] : 0;
          unsigned char *d = st + ((size_t)q * NT + tid) * RBY;
          const unsigned char *src = reinterpret_cast<const unsigned char *>(recb + (size_t)o * 4);
#pragma unroll
          for (int z = 0; z < RBY / 16; ++z) cp_async_16_l2_nc(d + 16 * z, src + 16 * z, v[q]);
          cp_async_zfill_nc<sizeof(T)>(sc + (SY + q) * NT, yb + o, v[q]);
          if constexpr (!ZX) cp_async_zfill_nc<sizeof(T)>(sc + (SX + q) * NT, xb + o, v[q]);
        }
#pragma unroll
        for (int q = 0; q < Q; q += PJ) {
          const bool vq = PJ == 2 ? (v[q] || v[q + PJ - 1]) : v[q];
          cp_async_16_if_nc(fs + (w * Q + q) * W, fjb + t * TKW + q * W, lane == kTJ - 1 && g.hasN && vq);
        }
        cp_async_16_if_nc(fs + (TK + lane) * W, fkb + t * TJW, g.eT && g.hasT && v[Q - 1]);
      }
      cp_async_commit();
    };
    static_for<0, R - 1>([&](auto u) { issue(decltype(u)::value, u); });

    T dE[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) dE[q] = T(0);
    // walk padded to a multiple of R steps, as in the forward sweep
    for (int u0 = 0; u0 < g.nsteps; u0 += R) {
      static_for<0, R>([&](auto uc) {
        constexpr int sl = decltype(uc)::value;
        const int u = u0 + sl;
        issue(u + R - 1, std::integral_constant<int, (sl + R - 1) % R>{});
        cp_async_wait<R - 1>();
        const unsigned char *st = stage + (size_t)sl * L.step;
        const T *sc = reinterpret_cast<const T *>(st + L.rec) + tid;
        const uint64_t *fs = fst + (size_t)sl * FS * W;
        const int t = last - u;
        T *E = exT + (size_t)sl * NW * 32;
        E[w * 32 + lane] = dE[0];
        __syncthreads();
        // faces of this step: J (lane 31, per row or row pair) and K (last warp, last row)
        bool act[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) act[q] = colq[q] && (unsigned)(t - tlo[q]) < nxu;
        constexpr int NJ = Q / PJ;
        bool needJ[NJ];
        uint64_t jw[NJ][2], kw[2] = {0, 0};
        bool stale = false;
#pragma unroll
        for (int r = 0; r < NJ; ++r) {
          const int q = r * PJ;
          needJ[r] = lane == kTJ - 1 && g.hasN && (PJ == 2 ? (act[q] || act[q + PJ - 1]) : act[q]);
          staged_words(fs + (w * Q + q) * W, jw[r]);
          stale |= needJ[r] && !rec_ok<2>(jw[r], expect);
        }
        const bool needK = g.eT && g.hasT && act[Q - 1];
        staged_words_if(fs + (TK + lane) * W, kw, g.eT);
        stale |= needK && !rec_ok<2>(kw, expect);
        if (__any_sync(0xffffffffu, stale)) {
#pragma unroll
          for (int r = 0; r < NJ; ++r)
            if (needJ[r] && !rec_ok<2>(jw[r], expect))
              face_wait<2>(dnJ + ((long long)(t - (kTJ - 1)) * TK + w * Q + r * PJ) * W, expect, jw[r], c, abort, tr);
          if (needK && !rec_ok<2>(kw, expect))
            face_wait<2>(dnK + kface + ((long long)(t - (TK - 1)) * kTJ + lane) * W, expect, kw, c, abort, tr);
        }
        const T dK = needK ? Face<T>::get(kw) : T(0);
        T nd[Q], xv[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const T *rec = reinterpret_cast<const T *>(st + ((size_t)q * NT + tid) * RBY);
          T dN = shfl_dn1(dE[q]);
          if (lane == kTJ - 1) dN = (g.hasN && act[q]) ? face_row<T, PJ>(jw[q / PJ], q) : T(0);
          T dT;
          if (q < Q - 1) dT = dE[q < Q - 1 ? q + 1 : 0];
          else if (w < NW - 1) dT = E[(w + 1) * 32 + lane];
          else dT = dK;
          T d = fma(-rec[RECB_UE], dE[q], sc[(SY + q) * NT]);
          d = fma(-rec[RECB_UN], dN, d);
          d = fma(-rec[RECB_UT], dT, d);
          T xn = d;
          if constexpr (!ZX) xn = sc[(SX + q) * NT] + d;
          xv[q] = xn;
          nd[q] = act[q] ? d : T(0);
        }
        // stores last: the update, then the face records (ordered memory operations)
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (act[q]) xb[offr[sl][q]] = xv[q];
#pragma unroll
        for (int q = 0; q < Q; q += PJ)
          face_put<T, PJ>(pjb + t * TKW + q * W, nd, q, ep,
                          lane == 0 && g.hasS && (PJ == 2 ? (act[q] || act[q + PJ - 1]) : act[q]));
        Face<T>::put_if(pkb + t * TJW, nd[0], ep, g.eB && g.hasB && act[0]);
#pragma unroll
        for (int q = 0; q < Q; ++q) dE[q] = nd[q];
      });
    }
    cp_async_wait<0>();
    if (tr && threadIdx.x == 0) tr[2] = gtimer();
    __syncthreads();
  }
}

}  // namespace sipk
