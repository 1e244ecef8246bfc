// sip_k64.cu -- instantiations of the FP64 sweep kernels (factorisation with
// FP64 factors, FP64 forward / backward substitution).
#include "sip_kernels.h"
#include "sip_factor.cuh"
#include "sip_sweeps.cuh"

namespace sipk {

template <int Q, int R>
static const void *pick64(int kind) {
  if constexpr (R == 2) return kind == K_FACTOR ? (const void *)k_factor<double, Q, R> : nullptr;
  switch (kind) {
    case K_FACTOR: return (const void *)k_factor<double, Q, R>;
    case K_FWD64: return (const void *)k_forward<double, Q, R>;
    case K_BWD64: return (const void *)k_backward<double, false, Q, R>;
    default: return nullptr;
  }
}

// one row per warp: the factorisation's own tile decomposition
template <int R>
static const void *pickfac1_double(int kind) {
  return kind == K_FACTOR ? (const void *)k_factor<double, 1, R> : nullptr;
}

const void *kernel_ptr_64(int kind, int Q, int R) {
  if (Q == 1) return R == 2 ? pickfac1_double<2>(kind) : R == 3 ? pick64<1, 3>(kind) : R == 4 ? pick64<1, 4>(kind) : R == 6 ? pick64<1, 6>(kind) : nullptr;
  if (Q == 2) return R == 2 ? pick64<2, 2>(kind) : R == 3 ? pick64<2, 3>(kind) : R == 4 ? pick64<2, 4>(kind) : R == 6 ? pick64<2, 6>(kind) : nullptr;
  if (Q == 4) return R == 2 ? pick64<4, 2>(kind) : R == 3 ? pick64<4, 3>(kind) : R == 4 ? pick64<4, 4>(kind) : R == 6 ? pick64<4, 6>(kind) : nullptr;
  return nullptr;
}

}  // namespace sipk
