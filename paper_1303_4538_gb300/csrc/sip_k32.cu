// sip_k32.cu -- instantiations of the FP32 sweep kernels (factorisation with
// FP32 factors, inner iterations of the mixed-precision refinement and the
// pure single-precision relaxation).
#include "sip_kernels.h"
#include "sip_factor.cuh"
#include "sip_sweeps.cuh"

namespace sipk {

template <int Q, int R>
static const void *pick32(int kind) {
  if constexpr (R == 2) return kind == K_FACTOR32 ? (const void *)k_factor<float, Q, R> : nullptr;
  switch (kind) {
    case K_FACTOR32: return (const void *)k_factor<float, Q, R>;
    case K_FWD32: return (const void *)k_forward<float, Q, R>;
    case K_BWD32: return (const void *)k_backward<float, false, Q, R>;
    case K_BWD32Z: return (const void *)k_backward<float, true, Q, R>;
    default: return nullptr;
  }
}

// one row per warp: the factorisation's own tile decomposition
template <int R>
static const void *pickfac1_float(int kind) {
  return kind == K_FACTOR32 ? (const void *)k_factor<float, 1, R> : nullptr;
}

const void *kernel_ptr_32(int kind, int Q, int R) {
  if (Q == 1) return R == 2 ? pickfac1_float<2>(kind) : R == 3 ? pick32<1, 3>(kind) : R == 4 ? pick32<1, 4>(kind) : R == 6 ? pick32<1, 6>(kind) : nullptr;
  if (Q == 2) return R == 2 ? pick32<2, 2>(kind) : R == 3 ? pick32<2, 3>(kind) : R == 4 ? pick32<2, 4>(kind) : R == 6 ? pick32<2, 6>(kind) : nullptr;
  if (Q == 4) return R == 2 ? pick32<4, 2>(kind) : R == 3 ? pick32<4, 3>(kind) : R == 4 ? pick32<4, 4>(kind) : R == 6 ? pick32<4, 6>(kind) : nullptr;
  return nullptr;
}

}  // namespace sipk
