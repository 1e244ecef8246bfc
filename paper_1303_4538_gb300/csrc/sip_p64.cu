// sip_p64.cu -- instantiations of the FP64 substitution sweeps over the
// column layout (forward y = L^-1 r; backward d = U^-1 y with x += d), by
// rows per warp Q and stage depth D.
#include "sip_kernels.h"
#include "sip_psweeps.cuh"

namespace sipk {

template <int Q, int D>
static const void *ppick64(int kind) {
  switch (kind) {
    case K_FWD64: return (const void *)k_csweep<double, true, false, Q, D>;
    case K_BWD64: return (const void *)k_csweep<double, false, false, Q, D>;
    default: return nullptr;
  }
}

template <int Q>
static const void *ppick64_d(int kind, int D) {
  return D == 4 ? ppick64<Q, 4>(kind) : D == 8 ? ppick64<Q, 8>(kind) : nullptr;
}

const void *wkernel_ptr_64(int kind, int Q, int D) {
  if (Q == 1) return ppick64_d<1>(kind, D);
  if (Q == 2) return ppick64_d<2>(kind, D);
  if (Q == 4) return ppick64_d<4>(kind, D);
  return nullptr;
}

}  // namespace sipk
