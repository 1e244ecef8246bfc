// sip_k32.cu -- instantiations of the FP32 sweep kernels (inner iterations of
// the mixed-precision refinement and the pure single-precision relaxation).
#include "sip_kernels.h"
#include "sip_sweeps.cuh"

namespace sipk {

template <int Q, int R>
static const void *pick32(int kind) {
  switch (kind) {
    case K_FWD32: return (const void *)k_forward<float, false, false, false, Q, R>;
    case K_FWD32S: return (const void *)k_forward<float, true, false, false, Q, R>;
    case K_FWD32Z: return (const void *)k_forward<float, false, true, false, Q, R>;
    case K_FWD32N: return (const void *)k_forward<float, false, false, true, Q, R>;
    case K_FWD32SN: return (const void *)k_forward<float, true, false, true, Q, R>;
    case K_BWD32: return (const void *)k_backward<float, false, false, Q, R>;
    case K_BWD32Z: return (const void *)k_backward<float, true, false, Q, R>;
    case K_BWD32U: return (const void *)k_backward<float, false, true, Q, R>;
    case K_BWD32ZU: return (const void *)k_backward<float, true, true, Q, R>;
    default: return nullptr;
  }
}

const void *kernel_ptr_32(int kind, int Q, int R) {
  if (Q == 2) return R == 4 ? pick32<2, 4>(kind) : R == 6 ? pick32<2, 6>(kind) : nullptr;
  if (Q == 4) return R == 4 ? pick32<4, 4>(kind) : R == 6 ? pick32<4, 6>(kind) : nullptr;
  return nullptr;
}

}  // namespace sipk
