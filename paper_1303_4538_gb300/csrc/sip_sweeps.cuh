// sip_sweeps.cuh -- wavefront machinery of Stone's SIP over the plane layout,
// used by the factorisation (lu3d, arXiv:1303.4538 Sec. 1 / Sec. 4.1;
// sip_factor.cuh) and, for its PTX helpers and face words, by the
// substitution sweeps over the column layout (sip_psweeps.cuh).
//
// The factorisation makes a cell depend on its lower neighbours W, S, B;
// all cells of one hyperplane i + j + k = s are independent, so it advances
// plane by plane.  Work decomposition:
//
//   * the (j, k) cross-section of a block is cut into 32 x TK column tiles;
//     one CTA owns a tile; lane = j, and warp w owns the Q rows
//     k = k0 + w Q .. k0 + w Q + Q - 1, so a thread walks Q columns along i.
//     At local step t every cell the CTA touches lies on plane s = t + j0 + k0;
//   * neighbours of the previous plane: W from the thread's own registers, S
//     from lane j - 1 by warp shuffles, B from the thread's own neighbouring
//     row, and across warps through a double-buffered shared-memory exchange
//     (one barrier per step);
//   * each cell's input record (A) is staged with cp.async.cg (L2 only) R-1
//     steps ahead into a ring of shared-memory stages; invalid cells are
//     zero-filled;
//   * row addresses of the plane layout come from two small per-block tables
//     held in shared memory (plane offsets PO and the diagonal prefix sums F);
//   * between tiles, the recurrence's boundary values travel through "faces":
//     records of 8-byte words whose upper halves carry the launch's epoch tag.
//     A producer stores them with st.relaxed.gpu; a consumer prefetches them
//     with cp.async.cg and accepts a record when every tag matches (each word
//     is self-validating, so no fence or flag is needed); a stale record is
//     re-read from L2 with ld.relaxed.gpu until it matches.  Before a tile
//     starts, one thread waits until the upstream tiles are a few steps ahead
//     ("slack").  Every wait is bounded (max_spin polls), then the kernel
//     records DEV_TIMEOUT and runs to the end without waiting;
//   * CTAs claim tiles with an atomic ticket in a dependency-respecting order,
//     so a tile only waits for tiles claimed earlier by running CTAs.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_internal.h"
#include "sip_layout.h"

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
__device__ __forceinline__ void cp_async_16_l2(void *sdst, const void *gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
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

// Poll a W-word record in L2 until every tag equals `expect`.  Returns false
// (and zero words) after max_spin polls or once another thread recorded an
// error; `abort` then stays set so this thread never waits again.
template <int W>
__device__ __noinline__ bool face_wait(const uint64_t *p, unsigned expect, uint64_t (&w)[W],
                                       const SweepCommon &c, bool &abort, unsigned long long *tr) {
  if (!abort) {
    long long spins = 0;
    const unsigned long long t0 = tr ? gtimer() : 0ull;
    for (;;) {
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = ld_relaxed(p + q);
      if (rec_ok<W>(w, expect)) {
        if (tr) {
          atomicAdd(tr + 3, 1ull);
          atomicAdd(tr + 4, gtimer() - t0);
        }
        return true;
      }
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

}  // namespace sipk
