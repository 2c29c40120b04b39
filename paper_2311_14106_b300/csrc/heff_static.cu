// Fixed device scratch for the allocation-free split-path H_eff*psi entry
// point (dmrg_heff_apply_split_static).
//
// Callers that run inside a memory pool they do not own -- a host framework
// whose device allocator must not be bypassed, a code path that may not
// synchronise the device the way cudaMalloc/cudaFree can, or a process that
// has handed all device memory to another allocator -- cannot let the library
// allocate scratch for every call.  For them the scratch of the split path
// (psi^T in FP16 hi/lo, the stage-1 intermediate, the stage-2 partial tiles and
// the work tables) lives in this file-scope array instead.  Every GPU that
// loads the library holds these bytes until the process exits.
#include <cuda_runtime.h>

#include <mutex>

namespace dmrg {

constexpr size_t kStaticScratchBytes = 64ull << 20;   // 64 MiB per device

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the scratch on the current device.  The symbol's host
// name is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
cudaError_t static_scratch(void **ptr, size_t *bytes) {
  static std::mutex mu;
  static void *addr[256] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *ptr = addr[dev];
  *bytes = kStaticScratchBytes;
  return cudaSuccess;
}

}  // namespace dmrg
