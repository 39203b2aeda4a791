// Measurement helpers: the random-gather ceiling of the memory system and
// the L2 fetch-granularity control.
//
// The cuckoo filter's probes are independent random reads of one bucket
// (8-32 bytes) spread over a table much larger than L2.  Their ceiling is not
// the streaming copy bandwidth but the rate at which HBM serves random
// sectors; cf_probe_gather measures that rate with the same load
// instructions the query kernel uses, so the roofline of the filter kernels
// can be read against both numbers.
#include <cuda_runtime.h>

#include <cstdint>

#include "cf.h"
#include "cf_kernels.cuh"

namespace {

constexpr int kProbeBlock = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Each thread issues kProbeK independent loads of `W` 64-bit words at
// random W*8-aligned offsets, then folds them into one value per thread.
// n_slots is a power of two (the offset is a mask of a 64-bit mix).
template <int W, int kProbeK>
__global__ void __launch_bounds__(kProbeBlock)
k_gather(const unsigned long long* __restrict__ buf, uint64_t n_slots,
         uint64_t n_access, uint64_t seed, unsigned long long* sink) {
  unsigned long long acc = 0;
  const uint64_t tid = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  const uint64_t nth = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t base = tid * kProbeK; base < n_access; base += nth * kProbeK) {
    unsigned long long v[kProbeK][W];
#pragma unroll
    for (int k = 0; k < kProbeK; ++k) {
      const uint64_t slot = mix64(seed + base + k) & (n_slots - 1);
      const unsigned long long* p = buf + slot * W;
      if (base + k < n_access) {
        if constexpr (W == 1) {
          v[k][0] = cfk::ld_nc_u64(p);
        } else if constexpr (W == 2) {
          cfk::ld_nc_v2(p, v[k][0], v[k][1]);
        } else {
          cfk::ld_nc_v4(p, v[k][0], v[k][1], v[k][2], v[k][3]);
        }
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) v[k][w] = 0;
      }
    }
#pragma unroll
    for (int k = 0; k < kProbeK; ++k)
#pragma unroll
      for (int w = 0; w < W; ++w) acc ^= v[k][w];
  }
  if (acc == 0x5EEDull) atomicAdd(sink, 1ull);  // keeps the loads alive
}

template <int W, int KP>
cudaError_t launch_gather(const unsigned long long* p, uint64_t slots,
                          uint64_t n_access, uint64_t seed,
                          unsigned long long* sink, cudaStream_t s) {
  auto fn = k_gather<W, KP>;
  const int occ = cfk::cached_occupancy(reinterpret_cast<const void*>(fn), kProbeBlock);
  const uint64_t cap = uint64_t(cfk::device_sm_count()) * uint64_t(occ);
  uint64_t want = (n_access + kProbeBlock * KP - 1) / (kProbeBlock * KP);
  fn<<<unsigned(want < cap ? want : cap), kProbeBlock, 0, s>>>(p, slots, n_access, seed, sink);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_gather_k(const unsigned long long* p, uint64_t slots,
                            uint64_t n_access, uint32_t loads, uint64_t seed,
                            unsigned long long* sink, cudaStream_t s) {
  switch (loads) {
    case 4: return launch_gather<W, 4>(p, slots, n_access, seed, sink, s);
    case 16: return launch_gather<W, 16>(p, slots, n_access, seed, sink, s);
    default: return launch_gather<W, 8>(p, slots, n_access, seed, sink, s);
  }
}

}  // namespace

extern "C" {

cf_status cf_probe_gather(const void* buf, uint64_t bytes, uint64_t n_access,
                          uint32_t access_bytes, uint32_t loads_per_thread,
                          uint64_t seed, unsigned long long* sink,
                          void* stream) {
  if (!buf || !sink) return CF_EINVAL;
  if (access_bytes != 8 && access_bytes != 16 && access_bytes != 32)
    return CF_EINVAL;
  if (loads_per_thread != 4 && loads_per_thread != 8 && loads_per_thread != 16)
    return CF_EINVAL;
  if ((reinterpret_cast<uintptr_t>(buf) & 31) != 0) return CF_EINVAL;
  uint64_t slots = bytes / access_bytes;
  if (slots == 0 || n_access == 0) return CF_EINVAL;
  while (slots & (slots - 1)) slots &= slots - 1;  // round down to 2^k
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned long long* p = static_cast<const unsigned long long*>(buf);
  cudaError_t e;
  switch (access_bytes) {
    case 8: e = launch_gather_k<1>(p, slots, n_access, loads_per_thread, seed, sink, s); break;
    case 16: e = launch_gather_k<2>(p, slots, n_access, loads_per_thread, seed, sink, s); break;
    default: e = launch_gather_k<4>(p, slots, n_access, loads_per_thread, seed, sink, s); break;
  }
  return e == cudaSuccess ? CF_OK : CF_ECUDA;
}

cf_status cf_set_l2_fetch_granularity(uint32_t bytes) {
  if (bytes > 128) return CF_EINVAL;
  return cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, bytes) == cudaSuccess
             ? CF_OK
             : CF_ECUDA;
}

cf_status cf_get_l2_fetch_granularity(uint32_t* bytes) {
  if (!bytes) return CF_EINVAL;
  size_t v = 0;
  if (cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity) != cudaSuccess)
    return CF_ECUDA;
  *bytes = uint32_t(v);
  return CF_OK;
}

}  // extern "C"
