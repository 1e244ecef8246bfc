// sip_kernels.h -- kernel registry of libsip.so: every sweep kernel variant is
// addressed by (kind, rows per thread Q, stages R) so the host runtime can size
// shared memory, query occupancy and launch it with cudaLaunchKernel.
#pragma once
#include <cstddef>

namespace sipk {

enum KernelKind {
  K_FACTOR = 0,   // Stone factorisation, FP64 factors
  K_FWD64,        // FP64 residual + norm + forward substitution, general A
  K_FWD64S,       // same, symmetric A (Listing 1 residual)
  K_BWD64,        // FP64 backward substitution + update
  K_FWD32,        // FP32 forward, general, no norm (inner refinement sweeps)
  K_FWD32S,       // FP32 forward, symmetric, no norm
  K_FWD32Z,       // FP32 forward with x = 0 (r = b)
  K_FWD32N,       // FP32 forward, general, with norm (pure single-precision mode)
  K_FWD32SN,      // FP32 forward, symmetric, with norm
  K_BWD32,        // FP32 backward + update
  K_BWD32Z,       // FP32 backward with x = 0 on entry
  K_BWD32U,       // FP32 backward + update, then x64 += x
  K_BWD32ZU,      // x = 0 on entry, then x64 += x
  K_RES64,        // FP64 residual of the refinement loop, A in FP64
  K_RES64S,       // same, symmetric
  K_RES32A,       // FP64 residual, A stored in FP32 (widened)
  K_RES32AS,      // same, symmetric
  K_FACTOR32,     // Stone factorisation (FP64 arithmetic), FP32 factors
  K_NKINDS
};

constexpr int kQs[2] = {2, 4};
constexpr int kRs[2] = {4, 6};

const void *kernel_ptr(int kind, int Q, int R);
// dynamic shared memory of a launch with `nthreads` threads per CTA
size_t kernel_smem(int kind, int Q, int R, int nthreads, int tab_ints);
bool kernel_is_ticketed(int kind);

const void *kernel_ptr_64(int kind, int Q, int R);
const void *kernel_ptr_32(int kind, int Q, int R);
const void *kernel_ptr_res(int kind, int Q, int R);

}  // namespace sipk
