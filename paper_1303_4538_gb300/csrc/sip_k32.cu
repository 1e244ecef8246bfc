// sip_k32.cu -- instantiations of the FP32 sweep kernels (inner iterations of
// the mixed-precision refinement and the pure single-precision relaxation).
#include "sip_kernels.h"
#include "sip_sweeps.cuh"

namespace sipk {

template <int R>
static const void *pick32(int kind) {
  switch (kind) {
    case K_FWD32: return (const void *)k_forward<float, false, false, false, R>;
    case K_FWD32S: return (const void *)k_forward<float, true, false, false, R>;
    case K_FWD32Z: return (const void *)k_forward<float, false, true, false, R>;
    case K_FWD32N: return (const void *)k_forward<float, false, false, true, R>;
    case K_FWD32SN: return (const void *)k_forward<float, true, false, true, R>;
    case K_BWD32: return (const void *)k_backward<float, false, false, R>;
    case K_BWD32Z: return (const void *)k_backward<float, true, false, R>;
    case K_BWD32U: return (const void *)k_backward<float, false, true, R>;
    case K_BWD32ZU: return (const void *)k_backward<float, true, true, R>;
    default: return nullptr;
  }
}

const void *kernel_ptr_32(int kind, int stages) {
  return stages == 3 ? pick32<3>(kind) : stages == 6 ? pick32<6>(kind) : nullptr;
}

}  // namespace sipk
