// Seeded synthetic inputs for the cuckoo-filter workloads.
//
// This module produces INPUTS only (keys, query mixes).  It holds none of the
// filter's arithmetic: no fingerprint, bucket index, slot layout or eviction
// logic lives here.  Both the CPU oracle tests and the GPU path draw their
// keys from these functions so that both sides see identical bytes.
//
// Every generator is counter-based: element i of a stream is a pure function
// of (seed, i), so the host loop and the device kernel produce the same bytes
// and any slice of a stream can be generated independently.
//
// splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): the state advances by the odd constant
// 0x9E3779B97F4A7C15 and each state is passed through a bijective 64-bit
// finaliser.  Because the state sequence seed + (i+1)*gamma visits distinct
// values mod 2^64 and the finaliser is a bijection, the first N outputs of one
// seed are pairwise distinct.  The workloads use this to get disjoint positive
// and negative key sets without rejection sampling.
//
// The paper's synthetic setup uses uniformly distributed 64-bit keys
// (Sec. 5.2) and, for the FPR experiment, positives from [0, 2^32) and
// negatives from [2^32, 2^64) (Sec. 5.3).

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#define WL_HD __host__ __device__ __forceinline__

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

WL_HD uint64_t splitmix64_finalise(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Output i (0-based) of the splitmix64 stream started from `seed`.
WL_HD uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  return splitmix64_finalise(seed + (i + 1) * kGamma);
}

// murmur3's 32-bit finaliser: a bijection on uint32 (xor-shifts and odd
// multiplies are each invertible), used to enumerate distinct keys in
// [0, 2^32).
WL_HD uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Element j of the 50/50 query mix: even j -> a positive drawn uniformly
// (with replacement) from keys[0, n_keys) by stream `pos_seed`; odd j -> a
// negative taken from stream `neg_seed` at index neg_start + j/2.
WL_HD uint64_t query_mix_at(uint64_t j, const uint64_t* keys, uint64_t n_keys,
                            uint64_t pos_seed, uint64_t neg_seed,
                            uint64_t neg_start) {
  const uint64_t half = j >> 1;
  if ((j & 1) == 0) return keys[splitmix64_at(pos_seed, half) % n_keys];
  return splitmix64_at(neg_seed, neg_start + half);
}

WL_HD uint64_t low32_key_at(uint32_t seed, uint64_t i) {
  return (uint64_t)fmix32((uint32_t)i + seed);
}

WL_HD uint64_t high_key_at(uint64_t seed, uint64_t i) {
  // Force a nonzero upper half so the key lies in [2^32, 2^64).
  return splitmix64_at(seed, i) | (1ull << 32);
}

__global__ void k_splitmix(uint64_t* out, uint64_t n, uint64_t seed,
                           uint64_t start) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = splitmix64_at(seed, start + i);
}

__global__ void k_query_mix(uint64_t* out, uint64_t n, const uint64_t* keys,
                            uint64_t n_keys, uint64_t pos_seed,
                            uint64_t neg_seed, uint64_t neg_start) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x)
    out[j] = query_mix_at(j, keys, n_keys, pos_seed, neg_seed, neg_start);
}

__global__ void k_low32(uint64_t* out, uint64_t n, uint32_t seed,
                        uint64_t start) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = low32_key_at(seed, start + i);
}

__global__ void k_high(uint64_t* out, uint64_t n, uint64_t seed,
                       uint64_t start) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = high_key_at(seed, start + i);
}

unsigned grid_for(uint64_t n) {
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152ull * 64) blocks = 152ull * 64;
  return blocks ? (unsigned)blocks : 1u;
}

int launch_status() { return cudaGetLastError() == cudaSuccess ? 0 : 1; }

}  // namespace

extern "C" {

// ---- host versions (plain loops; usable without a GPU) ----
void wl_splitmix64_host(uint64_t* out, uint64_t n, uint64_t seed,
                        uint64_t start) {
  for (uint64_t i = 0; i < n; ++i) out[i] = splitmix64_at(seed, start + i);
}

void wl_query_mix_host(uint64_t* out, uint64_t n, const uint64_t* keys,
                       uint64_t n_keys, uint64_t pos_seed, uint64_t neg_seed,
                       uint64_t neg_start) {
  for (uint64_t j = 0; j < n; ++j)
    out[j] = query_mix_at(j, keys, n_keys, pos_seed, neg_seed, neg_start);
}

void wl_low32_host(uint64_t* out, uint64_t n, uint32_t seed, uint64_t start) {
  for (uint64_t i = 0; i < n; ++i) out[i] = low32_key_at(seed, start + i);
}

void wl_high_host(uint64_t* out, uint64_t n, uint64_t seed, uint64_t start) {
  for (uint64_t i = 0; i < n; ++i) out[i] = high_key_at(seed, start + i);
}

// ---- device versions: `out` and `keys` are device pointers, `stream` is a
// cudaStream_t (NULL = legacy default stream).  Return 0 on a clean launch.
int wl_splitmix64_dev(uint64_t* out, uint64_t n, uint64_t seed, uint64_t start,
                      void* stream) {
  if (n == 0) return 0;
  k_splitmix<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, n, seed,
                                                            start);
  return launch_status();
}

int wl_query_mix_dev(uint64_t* out, uint64_t n, const uint64_t* keys,
                     uint64_t n_keys, uint64_t pos_seed, uint64_t neg_seed,
                     uint64_t neg_start, void* stream) {
  if (n == 0) return 0;
  if (n_keys == 0) return 2;
  k_query_mix<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
      out, n, keys, n_keys, pos_seed, neg_seed, neg_start);
  return launch_status();
}

int wl_low32_dev(uint64_t* out, uint64_t n, uint32_t seed, uint64_t start,
                 void* stream) {
  if (n == 0) return 0;
  k_low32<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, n, seed, start);
  return launch_status();
}

int wl_high_dev(uint64_t* out, uint64_t n, uint64_t seed, uint64_t start,
                void* stream) {
  if (n == 0) return 0;
  k_high<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, n, seed, start);
  return launch_status();
}

// Zipf(s)-duplicated keys (host only): element i draws a rank r in [1, U]
// from the continuous power-law approximation of Zipf(s) by inverse CDF,
//   r = floor(((U^(1-s) - 1) * u + 1)^(1/(1-s))),  u uniform in [0, 1),
// and returns the r-th key of the splitmix64 stream `key_seed` (so the
// key universe has U distinct keys and popular keys repeat).  Host only:
// floating-point pow may differ between host and device libraries, and the
// stream must be the same bytes for every consumer; copy it to the device.
void wl_zipf_host(uint64_t* out, uint64_t n, uint64_t rank_seed,
                  uint64_t key_seed, uint64_t universe, double s) {
  const double a = 1.0 - s;
  const double top = pow((double)universe, a) - 1.0;
  for (uint64_t i = 0; i < n; ++i) {
    const double u = (double)(splitmix64_at(rank_seed, i) >> 11) * 0x1.0p-53;
    double r = floor(pow(top * u + 1.0, 1.0 / a));
    if (r < 1.0) r = 1.0;
    if (r > (double)universe) r = (double)universe;
    out[i] = splitmix64_at(key_seed, (uint64_t)r - 1);
  }
}

}  // extern "C"
