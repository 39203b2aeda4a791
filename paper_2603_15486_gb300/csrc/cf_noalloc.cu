// cf_insert_noalloc: the insert of cf_insert for callers that cannot
// allocate device memory.
//
// cf_insert keeps its eviction work queue (4 bytes per key) in memory the
// library cudaMalloc's on a filter's first large insert.  This entry point
// runs the same two kernels with the queue in a fixed array compiled into
// the library instead, so it calls no cudaMalloc or cudaFree.  The array is
// a file-scope __device__ variable: every GPU that loads the library holds
// it (4 MiB) until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cf.h"
#include "cf_internal.h"

namespace {

static __device__ __align__(256) uint32_t g_noalloc_queue[CF_NOALLOC_MAX_KEYS];

// Device address of g_noalloc_queue, looked up once per device.  In host
// code the symbol's name is only a host-side stand-in; the kernels must be
// given this address.
std::mutex g_mu;
uint32_t* g_queue_dev[64] = {};

cf_status queue_for_device(int dev, uint32_t** out) {
  if (dev < 0 || dev >= 64) return CF_ENOTSUP;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_queue_dev[dev]) {
    uint32_t* ptr = nullptr;
    const cudaError_t e =
        cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_queue);
    if (e != cudaSuccess) {
      cfk::set_error("cudaGetSymbolAddress(g_noalloc_queue)", e);
      return CF_ECUDA;
    }
    g_queue_dev[dev] = ptr;
  }
  *out = g_queue_dev[dev];
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
  cf_status st = queue_for_device(dev, &queue);
  if (st != CF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = cfk::order_on(f, s);
  if (st != CF_OK) return st;
  e = f->ops->insert_chunk(f->d, keys, uint32_t(n), out_flags, nullptr, queue, s,
                           f->timer);
  if (e != cudaSuccess) {
    cfk::set_error("cf_insert_noalloc launch", e);
    return CF_ECUDA;
  }
  return cfk::mark(f, s);
}
