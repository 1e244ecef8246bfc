// sip_layout.h -- shared-memory layout of the wavefront kernels, used by the
// kernels to carve their dynamic shared memory and by the host to size it.
//
// The factorisation's dynamic shared memory is
//   [ PO + F tables of the current block ]
//   [ R stages: per step the staged A7 records of the thread's Q rows ]
//   [ exchange between neighbouring warps, double buffered ]
//   [ R stages of face records consumed by the tile's edge threads ]
// The substitution sweeps' layout (PLayout) follows below.
#pragma once
#include <cstddef>

namespace sipk {

__host__ __device__ inline size_t lay_a16(size_t b) { return (b + 15) & ~(size_t)15; }

struct SweepLayout {
  size_t tab;    // bytes of the PO/F tables
  size_t step;   // bytes of one stage
  size_t rec;    // bytes of the staged records inside a stage (Q * NT * rsb)
  size_t off;    // offset inside a stage of the cells' block-local offsets (Q * NT ints)
  size_t exch;   // bytes of the exchange area
  size_t faces;  // bytes of the face ring
  size_t total;
  int rsb;       // staged record bytes per row
  int nsv;       // scalar slots per thread per step
  int fs;        // face slots per stage (TK + 32)
};

// factorisation: A7 record (8 doubles) per row, no scalars, faces of 3 FP64 values
__host__ __device__ inline SweepLayout fac_layout(int Q, int R, int NT, int tab_ints) {
  SweepLayout L{};
  const int NW = NT / 32, TK = NW * Q;
  L.rsb = 64;
  L.nsv = 0;
  L.fs = TK + 32;
  L.tab = lay_a16((size_t)tab_ints * 4);
  L.rec = (size_t)Q * NT * L.rsb;
  L.step = L.rec;
  L.exch = lay_a16((size_t)2 * 3 * NW * 32 * 8);
  L.faces = (size_t)R * L.fs * 6 * 8;
  L.total = L.tab + (size_t)R * L.step + L.exch + L.faces;
  return L;
}

constexpr int kRingSlots = 8;  // steps a warp may run ahead of the warp it feeds

// ---------------------------------------------------------------------------
// Substitution sweeps over the column layout (sip_psweeps.cuh).  A stage
// holds, per warp, the records of its Q rows as 16-byte chunks
// (lane-contiguous, 512 bytes per chunk row), then NS x Q x 32 scalars; a
// CTA's stage is its NW warps' parts back to back, D stages form the ring,
// and a double-buffered exchange of NW x 32 values follows.
template <int ES, bool FWD, bool ZX, int Q>
struct CSweepCfg {
  static constexpr int NCH = 4 * ES / 16;            // 16-byte chunks per record (FP32 1, FP64 2)
  static constexpr int NS = FWD ? 1 : (ZX ? 1 : 2);  // staged scalars: r; or y (and x)
  static constexpr int SREC = Q * NCH * 512;         // bytes of a warp's records in a stage
};

struct CLayout {
  size_t warp_stage;  // bytes of one warp's part of a stage
  size_t stage;       // bytes of one stage (all warps)
  size_t total;
};

__host__ __device__ inline CLayout c_layout(int esize, int nsca, int Q, int D, int NW) {
  CLayout L{};
  L.warp_stage = lay_a16((size_t)Q * (4 * esize / 16) * 512 + (size_t)nsca * Q * 32 * esize);
  L.stage = (size_t)NW * L.warp_stage;
  L.total = (size_t)D * L.stage + (size_t)2 * NW * 32 * esize;
  return L;
}
}  // namespace sipk
