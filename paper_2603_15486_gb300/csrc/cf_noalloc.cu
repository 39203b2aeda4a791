// cf_insert_noalloc: the insert of cf_insert for callers that cannot
// allocate device memory.
//
// cf_insert keeps its eviction work queue (4 bytes per key) in memory the
// library cudaMalloc's on a filter's first large insert.  This entry point
// runs the plain two-kernel insert (direct insertion, then the eviction
// loop) with the queue in a fixed array compiled into the library instead,
// so it calls no cudaMalloc or cudaFree.  The array is a file-scope
// __device__ variable: every GPU that loads the library holds it (4 MiB)
// until the process exits.
#include <cuda_runtime.h>

#include <cstdint>

#include "cf.h"
#include "cf_internal.h"

namespace {

static __device__ __align__(256) uint32_t g_noalloc_queue[CF_NOALLOC_MAX_KEYS];

// Device address of g_noalloc_queue in the current device's context.  In
// host code the symbol's name is only a host-side stand-in; the kernels
// must be given this address.  It is looked up on every call (a host-side
// table lookup once the library's device code is loaded): a context that
// was torn down and rebuilt (cudaDeviceReset) places the array anew, and a
// cached address would then point at memory the context no longer maps.
cf_status queue_address(uint32_t** out) {
  uint32_t* ptr = nullptr;
  const cudaError_t e =
      cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_queue);
  if (e != cudaSuccess || ptr == nullptr) {
    cfk::set_error("cudaGetSymbolAddress(g_noalloc_queue)",
                   e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    return CF_ECUDA;
  }
  *out = ptr;
  return CF_OK;
}

}  // namespace

extern "C" cf_status cf_insert_noalloc(cf_filter* f, const uint64_t* keys,
                                       uint64_t n, uint8_t* out_flags,
                                       void* stream) {
  if (!f) return CF_EINVAL;
  if (n == 0) return CF_OK;
  if (!keys) return CF_EINVAL;
  if (n > CF_NOALLOC_MAX_KEYS) {
    cfk::set_error_text(
        "cf_insert_noalloc: n exceeds CF_NOALLOC_MAX_KEYS (2^20 keys); "
        "split the batch or use cf_insert");
    return CF_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cfk::set_error("cudaGetDevice", e);
    return CF_ECUDA;
  }
  if (dev != f->device) {
    cfk::set_error_text("cf_insert_noalloc: the filter's device is not current");
    return CF_EINVAL;
  }
  uint32_t* queue = nullptr;
  cf_status st = queue_address(&queue);
  if (st != CF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = cfk::order_on(f, s);
  if (st != CF_OK) return st;
  e = f->ops->insert_chunk(f->d, keys, uint32_t(n), out_flags, nullptr, queue,
                           cfk::EvictMap{}, s, f->timer);
  if (e != cudaSuccess) {
    cfk::set_error("cf_insert_noalloc launch", e);
    return CF_ECUDA;
  }
  return cfk::mark(f, s);
}
