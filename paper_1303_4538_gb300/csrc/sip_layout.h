// sip_layout.h -- shared-memory layout of the sweep kernels, used by the
// kernels to carve their dynamic shared memory and by the host to size it.
//
// Every sweep kernel's dynamic shared memory is
//   [ PO + F tables of the current block ]
//   [ R stages: per step the staged records of the thread's Q rows, then
//     scalar slots (r; y and x) ]
//   [ exchange between neighbouring warps, one slot per stage ]
//   [ R stages of face records consumed by the tile's edge threads ]
#pragma once
#include <cstddef>

namespace sipk {

__host__ __device__ inline size_t lay_a16(size_t b) { return (b + 15) & ~(size_t)15; }

struct SweepLayout {
  size_t tab;    // bytes of the PO/F tables
  size_t step;   // bytes of one stage
  size_t rec;    // bytes of the staged records inside a stage (Q * NT * rsb)
  size_t exch;   // bytes of the exchange area
  size_t faces;  // bytes of the face ring
  size_t total;
  int rsb;       // staged record bytes per row
  int nsv;       // scalar slots per thread per step
  int fs;        // face slots per stage (TK + 32)
};

// forward sweep (esize: 4 or 8): L record [LB LW LS 1/LP] and r per row;
// the exchange carries y of a warp's last row
__host__ __device__ inline SweepLayout fwd_layout(int esize, int Q, int R, int NT, int tab_ints) {
  SweepLayout L{};
  const int NW = NT / 32, TK = NW * Q;
  L.rsb = 4 * esize;
  L.nsv = Q;
  L.fs = TK + 32;
  L.tab = lay_a16((size_t)tab_ints * 4);
  L.rec = (size_t)Q * NT * L.rsb;
  L.step = lay_a16(L.rec + (size_t)L.nsv * NT * esize);
  L.exch = lay_a16((size_t)R * NW * 32 * esize);
  L.faces = (size_t)R * L.fs * 2 * 8;
  L.total = L.tab + (size_t)R * L.step + L.exch + L.faces;
  return L;
}

// backward sweep: record [UE UN UT 0]; scalars y, x per row
__host__ __device__ inline SweepLayout bwd_layout(int esize, bool zx, int Q, int R, int NT, int tab_ints) {
  SweepLayout L{};
  const int NW = NT / 32, TK = NW * Q;
  L.rsb = 4 * esize;
  L.nsv = Q * (zx ? 1 : 2);
  L.fs = TK + 32;
  L.tab = lay_a16((size_t)tab_ints * 4);
  L.rec = (size_t)Q * NT * L.rsb;
  L.step = lay_a16(L.rec + (size_t)L.nsv * NT * esize);
  L.exch = lay_a16((size_t)R * NW * 32 * esize);
  L.faces = (size_t)R * L.fs * 2 * 8;
  L.total = L.tab + (size_t)R * L.step + L.exch + L.faces;
  return L;
}

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

}  // namespace sipk
