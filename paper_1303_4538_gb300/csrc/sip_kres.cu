// sip_kres.cu -- instantiations of the FP64 residual kernels of the
// refinement loop and of the factorisation with FP32 factors.
#include "sip_kernels.h"
#include "sip_sweeps.cuh"

namespace sipk {

template <int Q, int R>
static const void *pickres(int kind) {
  switch (kind) {
    case K_RES64: return (const void *)k_resid<double, false, Q, R>;
    case K_RES64S: return (const void *)k_resid<double, true, Q, R>;
    case K_RES32A: return (const void *)k_resid<float, false, Q, R>;
    case K_RES32AS: return (const void *)k_resid<float, true, Q, R>;
    case K_FACTOR32: return (const void *)k_factor<float, Q, R>;
    default: return nullptr;
  }
}

const void *kernel_ptr_res(int kind, int Q, int R) {
  if (Q == 2) return R == 4 ? pickres<2, 4>(kind) : R == 6 ? pickres<2, 6>(kind) : nullptr;
  if (Q == 4) return R == 4 ? pickres<4, 4>(kind) : R == 6 ? pickres<4, 6>(kind) : nullptr;
  return nullptr;
}

}  // namespace sipk
