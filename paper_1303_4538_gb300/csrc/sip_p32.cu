// sip_p32.cu -- instantiations of the FP32 substitution sweeps over the
// column layout (the inner iterations of the mixed-precision refinement and
// the pure single-precision relaxation), by rows per warp Q and stage depth D.
#include "sip_kernels.h"
#include "sip_psweeps.cuh"

namespace sipk {

template <int Q, int D>
static const void *ppick32(int kind) {
  switch (kind) {
    case K_FWD32: return (const void *)k_csweep<float, true, false, Q, D>;
    case K_BWD32: return (const void *)k_csweep<float, false, false, Q, D>;
    case K_BWD32Z: return (const void *)k_csweep<float, false, true, Q, D>;
    default: return nullptr;
  }
}

template <int Q>
static const void *ppick32_d(int kind, int D) {
  return D == 4 ? ppick32<Q, 4>(kind) : D == 8 ? ppick32<Q, 8>(kind) : nullptr;
}

const void *wkernel_ptr_32(int kind, int Q, int D) {
  if (Q == 1) return ppick32_d<1>(kind, D);
  if (Q == 2) return ppick32_d<2>(kind, D);
  if (Q == 4) return ppick32_d<4>(kind, D);
  return nullptr;
}

}  // namespace sipk
