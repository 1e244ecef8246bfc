// sip_kernels.h -- kernel registry of libsip.so: every sweep kernel variant is
// addressed by (kind, rows per thread Q, stages R) so the host runtime can size
// shared memory, query occupancy and launch it with cudaLaunchKernel.
#pragma once
#include <cstddef>

namespace sipk {

enum KernelKind {
  // wavefront sweeps (ticketed; addressed by Q and R)
  K_FACTOR = 0,   // Stone factorisation, FP64 factors
  K_FWD64,        // FP64 forward substitution y = L^-1 r
  K_BWD64,        // FP64 backward substitution + update
  K_FACTOR32,     // Stone factorisation (FP64 arithmetic), FP32 factors
  K_FWD32,        // FP32 forward substitution
  K_BWD32,        // FP32 backward + update
  K_BWD32Z,       // FP32 backward with x = 0 on entry
  // row-parallel residual r = b - A x (sip_resrow.cu; not ticketed, no Q/R)
  K_RES64,        // FP64: r into the substitution buffer, with the norm
  K_RES32,        // FP32, no norm (inner iterations of the refinement)
  K_RES32N,       // FP32 with the norm (single-precision mode)
  K_RES64R,       // FP64 residual of the refinement (A in FP64 or FP32), r rounded to FP32, norm
  K_UPD64,        // refinement update x64 += (double) d (element-wise)
  K_NKINDS
};

constexpr int kQs[3] = {1, 2, 4};
constexpr int kRs[4] = {2, 3, 4, 6};  // 2: the factorisation only (wide tiles)

// sweep kernel of a kind (nullptr for the row kinds)
const void *kernel_ptr(int kind, int Q, int R);
// dynamic shared memory of a sweep launch with `nthreads` threads per CTA
size_t kernel_smem(int kind, int Q, int R, int nthreads, int tab_ints);

const void *kernel_ptr_64(int kind, int Q, int R);
const void *kernel_ptr_32(int kind, int Q, int R);

}  // namespace sipk
