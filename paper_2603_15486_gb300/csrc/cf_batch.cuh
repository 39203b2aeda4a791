// Multi-filter launch: the insert / query / delete batches of many filters
// (of one geometry) in one persistent kernel, plus one eviction kernel over
// their combined queue.
//
// Every item (filter, op, keys) is cut into warp tiles of 32*K keys; a warp
// takes the next tile from a global counter, finds its item by binary
// search over the items' first-tile indices, and runs the same tile body as
// the single-filter kernels.  Warps therefore stay busy across items of
// very different sizes (10^2 to 10^6 keys), and no host loop launches per
// filter.  All descriptors live in device memory, so the pair of launches
// (plus the descriptor upload) can be captured once in a CUDA graph and
// replayed for new batches.
#pragma once

#include "cf_kernels.cuh"

namespace cfk {

enum : uint32_t { kOpInsert = 0, kOpContains = 1, kOpRemove = 2 };

struct BatchItemDev {
  DevFilter d;
  const uint64_t* keys;
  uint8_t* flags;
  uint64_t n;
  uint32_t op;
  uint32_t pad;
};

// Header of a batch plan's device buffer.  The host uploads it with every
// launch, so the counters start at zero each time.
struct BatchCtl {
  uint32_t n_items;
  uint32_t has_insert;
  uint64_t n_tiles;
  unsigned long long next_tile;
  unsigned int queue_count;
  unsigned int pad0;
  unsigned long long pad[4];
};
static_assert(sizeof(BatchCtl) == 64, "batch header is 64 bytes");

// Appends (item, key index) to the combined eviction queue: one atomic per
// warp tile.
struct BatchPush {
  unsigned int* count;
  uint2* queue;
  uint32_t item;
  template <int K>
  __device__ __forceinline__ void push_all(const bool (&need)[K],
                                           const uint32_t (&idx)[K],
                                           uint32_t lane) const {
    unsigned bal[K];
    uint32_t total = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      bal[k] = __ballot_sync(0xFFFFFFFFu, need[k]);
      total += __popc(bal[k]);
    }
    if (!total) return;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(count, total);
    pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (need[k]) queue[pos + __popc(bal[k] & lt)] = make_uint2(item, idx[k]);
      pos += __popc(bal[k]);
    }
  }
};

// Index of the item owning tile t: the last i with begins[i] <= t (items
// without keys own no tile).
__device__ __forceinline__ uint32_t find_item(const uint64_t* __restrict__ begins,
                                              uint32_t n_items, uint64_t t) {
  uint32_t lo = 0, hi = n_items;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (begins[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void warp_add(unsigned long long* dst, uint32_t v,
                                         uint32_t lane, bool negate = false) {
  const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, v);
  if (lane == 0 && s) atomicAdd(dst, negate ? (0ull - s) : (unsigned long long)s);
}

// A warp's CAS counts added to the histogram (every lane must call it).
__device__ __forceinline__ void cas_count_warp_add(const DevFilter& d, const CasCount& cc,
                                                   uint32_t lane) {
  if (!CF_CAS_HIST) return;
  warp_add(&d.ctrl->cas_retry[0], cc.first, lane);
  if (__any_sync(0xFFFFFFFFu, cc.deep != 0)) {
#pragma unroll
    for (int bin = 1; bin <= 6; ++bin)
      warp_add(&d.ctrl->cas_retry[bin], (cc.deep >> (5 * (bin - 1))) & 31u, lane);
  }
}

template <class G, int K, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_batch_tiles(BatchCtl* ctl, const BatchItemDev* __restrict__ items,
              const uint64_t* __restrict__ begins, uint2* __restrict__ queue) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t n_items = ctl->n_items;
  const uint64_t n_tiles = ctl->n_tiles;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&ctl->next_tile, 1ull);
    t = __shfl_sync(0xFFFFFFFFu, t, 0);
    if (t >= n_tiles) break;
    uint32_t it = 0;
    if (lane == 0) it = find_item(begins, n_items, t);
    it = __shfl_sync(0xFFFFFFFFu, it, 0);
    const BatchItemDev& I = items[it];
    const DevFilter d = I.d;
    const uint64_t base = (t - begins[it]) * (32u * K);
    TileCounts c;
    if (I.op == kOpContains) {
      tile_contains<G, K>(d, I.keys, I.n, base, lane, I.flags);
    } else if (I.op == kOpInsert) {
      const BatchPush push{&ctl->queue_count, queue, it};
      tile_insert<G, K>(d, I.keys, I.n, base, lane, I.flags, nullptr, push, c);
      warp_add(&d.ctrl->occupancy, c.ok, lane);
      warp_add(&d.ctrl->insert_ok, c.ok, lane);
      warp_add(&d.ctrl->insert_fail, c.cont, lane);
      warp_add(&d.ctrl->contention, c.cont, lane);
      cas_count_warp_add(d, c.cas, lane);
    } else {
      tile_remove<G, K>(d, I.keys, I.n, base, lane, I.flags, c);
      warp_add(&d.ctrl->occupancy, c.ok, lane, /*negate=*/true);
      warp_add(&d.ctrl->remove_ok, c.ok, lane);
      warp_add(&d.ctrl->remove_fail, c.fail + c.cont, lane);
      warp_add(&d.ctrl->contention, c.cont, lane);
      cas_count_warp_add(d, c.cas, lane);
    }
  }
}

// The combined eviction queue of all inserting items, with the lane
// refill of k_insert_evict over per-warp shares of the queue.
template <class G, int FW, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_batch_evict(BatchCtl* ctl, const BatchItemDev* __restrict__ items,
              const uint2* __restrict__ queue) {
  const uint32_t qn = *reinterpret_cast<const volatile unsigned int*>(&ctl->queue_count);
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t n_warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t next = uint32_t(uint64_t(qn) * warp / n_warps);
  const uint32_t end = uint32_t(uint64_t(qn) * (warp + 1) / n_warps);
  Chain<G> c{};
  uint2 q{};
  bool active = false;
  for (;;) {
    if (next < end) {
      const unsigned need = __ballot_sync(0xFFFFFFFFu, !active);
      if (!active) {
        const uint32_t e = next + __popc(need & ((1u << lane) - 1u));
        if (e < end) {
          q = queue[e];
          const BatchItemDev& I = items[q.x];
          const DevFilter d = I.d;
          const KeyHash kh = hash_key<G>(d, I.keys[q.y]);
          if (d.max_ev == 0) {
            log_victim(d, kh.fp, kh.i1);
            if (I.flags) st_flag(I.flags + q.y, EV_FAIL);
            atomicAdd(&d.ctrl->insert_fail, 1ull);
          } else {
            c = chain_start<G>(d, kh);
            active = true;
          }
        }
      }
      next += __popc(need);
    }
    if (!__any_sync(0xFFFFFFFFu, active)) {
      if (next >= end) break;
      continue;
    }
    if (active) {
      const BatchItemDev& I = items[q.x];
      const DevFilter d = I.d;
      EvictCounters ec;
      uint32_t vt = 0;
      uint64_t vb = 0;
      const int r = evict_round<G, FW>(d, c, vt, vb, ec);
      if (ec.contention) {
        atomicAdd(&d.ctrl->contention, (unsigned long long)ec.contention);
        atomicOr(&d.ctrl->error_word, 1u);
      }
      if (ec.cas.first | ec.cas.deep) cas_count_add(d, ec.cas);
      if (r != ROUND_CONTINUE) {
        if (r != EV_OK) log_victim(d, vt, vb);
        if (I.flags) st_flag(I.flags + q.y, uint8_t(r));
        if (r == EV_OK) {
          atomicAdd(&d.ctrl->occupancy, 1ull);
          atomicAdd(&d.ctrl->insert_ok, 1ull);
        } else {
          atomicAdd(&d.ctrl->insert_fail, 1ull);
        }
        if (c.ev) atomicAdd(&d.ctrl->evictions, (unsigned long long)c.ev);
        active = false;
      }
    }
  }
}

// One tunable configuration of the multi-filter launch.
struct BatchVariant {
  int keys_per_thread;  // K: keys per thread per tile
  int block;            // threads per block of the tile kernel
  int frontier;         // BFS candidates probed together (1 .. b/2)
  const void* tiles_fn;
  const void* evict_fn;
  cudaError_t (*tiles)(BatchCtl*, const BatchItemDev*, const uint64_t*, uint2*,
                       unsigned, cudaStream_t);
  cudaError_t (*evict)(BatchCtl*, const BatchItemDev*, const uint2*,
                       unsigned, cudaStream_t);
};

template <class G, int K, int BLOCK, int FW>
struct BatchLaunch {
  static cudaError_t tiles(BatchCtl* c, const BatchItemDev* it,
                           const uint64_t* b, uint2* q, unsigned grid,
                           cudaStream_t s) {
    k_batch_tiles<G, K, BLOCK><<<grid, BLOCK, 0, s>>>(c, it, b, q);
    return cudaGetLastError();
  }
  static cudaError_t evict(BatchCtl* c, const BatchItemDev* it,
                           const uint2* q, unsigned grid, cudaStream_t s) {
    k_batch_evict<G, FW, kBlock><<<grid, kBlock, 0, s>>>(c, it, q);
    return cudaGetLastError();
  }
  static BatchVariant make() {
    return BatchVariant{K, BLOCK, FW,
                        reinterpret_cast<const void*>(k_batch_tiles<G, K, BLOCK>),
                        reinterpret_cast<const void*>(k_batch_evict<G, FW, kBlock>),
                        &tiles, &evict};
  }
};

// The variants of one geometry: the default first.  The geometry of the
// large-filter workloads (16-bit fingerprints, 4 slots, XOR) and the
// paper's default bucket (16 slots) get the full tuning space.
template <class G>
struct BatchVariants {
  static const BatchVariant* get(int* count) {
    constexpr int KD = Tiles<G, true>::K;
    constexpr int H = G::B / 2;
    if constexpr (G::F == 16 && G::POLICY == 0 && (G::B == 4 || G::B == 16)) {
      static const BatchVariant v[] = {
          BatchLaunch<G, KD, 256, H>::make(),
          BatchLaunch<G, 2, 256, H>::make(),
          BatchLaunch<G, (KD >= 8 ? 4 : 8), 256, H>::make(),
          BatchLaunch<G, KD, 128, H>::make(),
          BatchLaunch<G, KD, 512, H>::make(),
          BatchLaunch<G, KD, 256, 1>::make(),
      };
      *count = int(sizeof(v) / sizeof(v[0]));
      return v;
    } else {
      static const BatchVariant v[] = {BatchLaunch<G, KD, 256, H>::make()};
      *count = 1;
      return v;
    }
  }
};

// One per translation unit (fingerprint width).
const BatchVariant* batch_variants_f8(int b, int policy, int* count);
const BatchVariant* batch_variants_f16(int b, int policy, int* count);
const BatchVariant* batch_variants_f32(int b, int policy, int* count);

inline const BatchVariant* batch_variants(int f, int b, int policy, int* count) {
  *count = 0;
  switch (f) {
    case 8: return batch_variants_f8(b, policy, count);
    case 16: return batch_variants_f16(b, policy, count);
    case 32: return batch_variants_f32(b, policy, count);
    default: return nullptr;
  }
}

}  // namespace cfk
