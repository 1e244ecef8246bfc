// sip_noalloc.cu -- scratch of sip_residual_norm_noalloc: the residual norm
// of sip_residual_norm (same kernels, same chunking, same bits) with its
// partial sums in a fixed array of this library's device image instead of
// device memory allocated for each call.
//
// Why: some callers cannot allocate device memory at the point where they
// want a norm.  A solver step that runs inside a fixed memory budget (all of
// it already handed to a caching allocator such as PyTorch's) has no room
// for a raw cudaMalloc, which may fail or fragment the pool; and a caller
// that keeps several streams busy cannot afford cudaFree, which waits for
// all work on the device.  Such callers get a call that performs no
// allocation and no host transfer: only two kernel launches on the
// context's stream.
//
// Limits and rules (also stated in include/sip.h):
//   * the scratch holds kNoallocParts partial pairs, i.e. blocks of at most
//     kNoallocParts * kResChunk = 67,108,864 cells; larger blocks are
//     rejected before anything is launched;
//   * nothing in the scratch has to start at zero: every slot a call reads
//     is written earlier in the same call;
//   * there is one scratch array per device, so calls whose work can overlap
//     on the device (different streams, contexts or host threads) race on it
//     and must be ordered by the caller;
//   * the device address of the array is looked up once per device (with
//     that device current) and cached; that first call may also load this
//     library's device code, so it belongs before any stream capture and
//     outside time-critical regions.  A cudaDeviceReset (or anything else
//     that destroys the device's primary context) unloads the array, so the
//     cached address is only valid until then; a failed launch drops it.
#include <cuda_runtime.h>

#include <mutex>

#include "sip_internal.h"

namespace sipk {

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocParts];

static std::mutex g_mu;
static void *g_addr[kNoallocMaxDevices] = {};

cudaError_t noalloc_scratch(int device, double **out) {
  std::mutex &mu = g_mu;
  void **addr = g_addr;
  *out = nullptr;
  if (device < 0 || device >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // device must be current
    if (e != cudaSuccess) return e;
    addr[device] = p;
  }
  *out = static_cast<double *>(addr[device]);
  return cudaSuccess;
}

void noalloc_forget(int device) {
  if (device < 0 || device >= kNoallocMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_mu);
  g_addr[device] = nullptr;
}

}  // namespace sipk
