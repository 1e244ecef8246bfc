// sip_k64.cu -- instantiations of the FP64 sweep kernels (factorisation,
// FP64 forward / backward, FP64 residual of the refinement loop).
#include "sip_kernels.h"
#include "sip_sweeps.cuh"

namespace sipk {

template <int R>
static const void *pick64(int kind) {
  switch (kind) {
    case K_FACTOR: return (const void *)k_factor<R>;
    case K_FWD64: return (const void *)k_forward<double, false, false, true, R>;
    case K_FWD64S: return (const void *)k_forward<double, true, false, true, R>;
    case K_BWD64: return (const void *)k_backward<double, false, false, R>;
    case K_RES64: return (const void *)k_resid<double, false, R>;
    case K_RES64S: return (const void *)k_resid<double, true, R>;
    case K_RES32A: return (const void *)k_resid<float, false, R>;
    case K_RES32AS: return (const void *)k_resid<float, true, R>;
    default: return nullptr;
  }
}

const void *kernel_ptr_64(int kind, int stages) {
  return stages == 3 ? pick64<3>(kind) : stages == 6 ? pick64<6>(kind) : nullptr;
}

}  // namespace sipk
