// Kernels of the cuckoo filter and their launchers, templated on the
// geometry (fingerprint bits, slots per bucket, bucket policy).
//
// Work distribution: a persistent grid (SM count x resident blocks) walks
// the batch in warp tiles of 32*K keys.  Lane l of a warp owns keys
// tile + k*32 + l for k < K, so every key load and flag store of a warp is
// one contiguous 256 B / 32 B access, and each thread keeps K independent
// random bucket accesses in flight (memory-level parallelism for HBM).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cf_device.cuh"

namespace cfk {

constexpr int kBlock = 256;

// Keys per thread: enough independent bucket loads in flight while keeping
// K buckets in registers.  CF_K_QUERY / CF_K_MUT override the default for
// 8-byte buckets (compile-time tuning); CF_MINB_MUT is the minimum resident
// blocks per SM requested for the mutating kernels.
#ifndef CF_K_QUERY
#define CF_K_QUERY 8
#endif
#ifndef CF_K_MUT
#define CF_K_MUT 4
#endif
#ifndef CF_MINB_MUT
#define CF_MINB_MUT 2
#endif
// The same for tables that L2 holds (at most kL2TableBytes): their CAS round
// trips end in L2, and more warps in flight pay (2^22 slots, ms per insert /
// delete of 0.95 * 2^22 keys at 2 -> 4 blocks per SM: f16 b16 0.259 / 0.166
// -> 0.230 / 0.133, f16 b4 0.516 / 0.203 -> 0.505 / 0.150, f8 b8 0.236 /
// 0.237 -> 0.223 / 0.185).  16-byte buckets keep CF_MINB_MUT: with four
// keys of two words each per thread, 64 registers spill and they got
// slower (f16 b8 0.237 -> 0.267 ms per insert).  DRAM-resident tables keep
// it too (plain large workload 160.7 -> 169.6 ms per step at 4).
#ifndef CF_MINB_MUT_L2
#define CF_MINB_MUT_L2 4
#endif
constexpr uint64_t kL2TableBytes = 64ull << 20;
// Minimum resident blocks per SM requested for the eviction kernel: 2, the
// grid's own blocks per SM (evict_grid), so that every geometry fits them;
// only f32 b16 needed the cap (159 -> 128 registers, a few spilled): on a
// 256 MiB table its eviction loop went from 1.23 to 1.06 ms (BFS) and from
// 1.90 to 1.48 ms (DFS) per fill to LF 0.95.
#ifndef CF_MINB_EVICT
#define CF_MINB_EVICT 2
#endif
// The eviction loop prepares each lane's next chain while the current one
// runs (1) or starts every chain from its queue entry when the lane is free
// (0).
#ifndef CF_EVICT_PREP
#define CF_EVICT_PREP 1
#endif
// BFS frontier width of the single-filter eviction kernel: the number of
// candidates whose alternate buckets are loaded together, groups in
// candidate order up to the first open bucket (CF_EVICT_FW; 0 or an invalid
// value means b/2, all at once).  2: with b = 16 the last quarter of a fill
// to LF 0.95 / 0.98 ran at 13.4 / 10.4 G inserts/s against 11.4 / 8.7 with
// all eight at once and 13.0 / 10.3 with four (2^28 slots): the early exit
// saves DRAM accesses.  b = 4 has b/2 = 2 anyway.
#ifndef CF_EVICT_FW
#define CF_EVICT_FW 2
#endif
template <class G>
struct EvictFW {
  static constexpr int H = G::B / 2;
  static constexpr int value =
      (CF_EVICT_FW > 0 && CF_EVICT_FW <= H && H % (CF_EVICT_FW > 0 ? CF_EVICT_FW : 1) == 0)
          ? CF_EVICT_FW
          : H;
};

template <class G, bool MUT>
struct Tiles {
  static constexpr int K = G::kBucketBytes <= 8 ? (MUT ? CF_K_MUT : CF_K_QUERY)
                           : G::kBucketBytes <= 16 ? 4
                           : G::kBucketBytes <= 32 ? 2 : 1;
};

__device__ __forceinline__ void st_flag(uint8_t* p, uint8_t v) {
  asm volatile("st.global.cs.u8 [%0], %1;" ::"l"(p), "h"((unsigned short)v));
}

// ---------------------------------------------------------------------------
// K keys' CAS attempts on one bucket each, issued together per round.
// INSERT: CAS the tag into the lowest empty lane (TryInsert, Alg. 1).
// REMOVE: CAS the lowest lane equal to the tag to zero (TryRemove, Alg. 3).
// Scan order per key: words from (tag mod b) / tpw with wrap-around.
// ---------------------------------------------------------------------------
// One-word buckets (b*f <= 64): the loaded word is the whole bucket, so a
// key's state is just its current word.
template <class G, int K, bool INSERT, bool RT = true>
__device__ __forceinline__ void cas_many_1w(const DevFilter& d,
                                            const uint32_t (&bkt)[K],
                                            const uint32_t (&tag)[K],
                                            const bool (&act)[K],
                                            int (&res)[K], CasCount& first) {
  using W = typename G::Word;
  W cur[K];
  bool live[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    res[k] = TI_FULL;
    live[k] = act[k];
    cur[k] = 0;
    if (live[k]) cur[k] = load_bucket<G, false>(bucket_ptr<G>(d, bkt[k])).w[0];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
    if (live[k] && !zero_lanes<G>(cur[k] ^ pat)) live[k] = false;
  }
  for (uint32_t round = 0; round < cas_bound<RT>(d); ++round) {
    W old[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
      const int lane = first_lane<G>(zero_lanes<G>(cur[k] ^ pat));
      const W desired = INSERT ? (cur[k] | (W(tag[k]) << (lane * G::F)))
                               : (cur[k] & ~(G::kLaneMask << (lane * G::F)));
      old[k] = atomicCAS(bucket_ptr<G>(d, bkt[k]), cur[k], desired);
    }
    bool any = false;
    uint32_t nf = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      if (old[k] == cur[k]) {
        res[k] = TI_OK;
        live[k] = false;
        continue;
      }
      ++nf;
      cur[k] = old[k];
      const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
      if (!zero_lanes<G>(cur[k] ^ pat)) {
        live[k] = false;
        continue;
      }
      any = true;
    }
    if (nf) note_cas_fails(d, round, nf, first);
    if (!any) break;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (live[k]) res[k] = TI_CONTENTION;
}

template <class G, int K, bool INSERT, bool RT = true>
__device__ __forceinline__ void cas_many_nw(const DevFilter& d,
                                            const uint32_t (&bkt)[K],
                                            const uint32_t (&tag)[K],
                                            const bool (&act)[K], int (&res)[K],
                                            CasCount& first) {
  using W = typename G::Word;
  Bucket<G> bk[K];
  W cur[K];
  int start[K], pos[K];
  bool live[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    res[k] = TI_FULL;
    live[k] = act[k];
    if (live[k]) bk[k] = load_bucket<G, false>(bucket_ptr<G>(d, bkt[k]));
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    start[k] = int((tag[k] % G::B) / G::kTpw);
    pos[k] = G::kWpb;
    cur[k] = 0;
    if (!live[k]) continue;
    const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
#pragma unroll
    for (int i = G::kWpb - 1; i >= 0; --i) {
      const W w = select_word<G>(bk[k], (start[k] + i) & (G::kWpb - 1));
      if (zero_lanes<G>(w ^ pat)) {
        pos[k] = i;
        cur[k] = w;
      }
    }
    if (pos[k] == G::kWpb) live[k] = false;
  }
  for (uint32_t round = 0; round < cas_bound<RT>(d); ++round) {
    W old[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
      const int lane = first_lane<G>(zero_lanes<G>(cur[k] ^ pat));
      const W desired = INSERT ? (cur[k] | (W(tag[k]) << (lane * G::F)))
                               : (cur[k] & ~(G::kLaneMask << (lane * G::F)));
      W* p = bucket_ptr<G>(d, bkt[k]) + ((start[k] + pos[k]) & (G::kWpb - 1));
      old[k] = atomicCAS(p, cur[k], desired);
    }
    bool any = false;
    uint32_t nf = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      if (old[k] == cur[k]) {
        res[k] = TI_OK;
        live[k] = false;
        continue;
      }
      ++nf;
      cur[k] = old[k];
      const W pat = INSERT ? W(0) : broadcast<G>(tag[k]);
      if (!zero_lanes<G>(cur[k] ^ pat)) {
        // This word has nothing left; continue with the next word of the
        // scan that (as first loaded) had a candidate lane.
        int np = G::kWpb;
#pragma unroll
        for (int i = G::kWpb - 1; i >= 1; --i) {
          if (i <= pos[k]) continue;
          const W w = select_word<G>(bk[k], (start[k] + i) & (G::kWpb - 1));
          if (zero_lanes<G>(w ^ pat)) {
            np = i;
            cur[k] = w;
          }
        }
        pos[k] = np;
        if (np == G::kWpb) {
          live[k] = false;
          continue;
        }
      }
      any = true;
    }
    if (nf) note_cas_fails(d, round, nf, first);
    if (!any) break;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (live[k]) res[k] = TI_CONTENTION;
}

template <class G, int K, bool INSERT, bool RT = true>
__device__ __forceinline__ void cas_many(const DevFilter& d,
                                         const uint32_t (&bkt)[K],
                                         const uint32_t (&tag)[K],
                                         const bool (&act)[K], int (&res)[K],
                                         CasCount& first) {
  static_assert(K <= 30, "a round's failure tally must fit a histogram field");
  if constexpr (G::kWpb == 1)
    cas_many_1w<G, K, INSERT, RT>(d, bkt, tag, act, res, first);
  else
    cas_many_nw<G, K, INSERT, RT>(d, bkt, tag, act, res, first);
}

// ---------------------------------------------------------------------------
// Per-tile bodies.  A tile is 32*K consecutive keys of one batch handled by
// one warp (lane l owns keys base + k*32 + l).  The single-filter kernels
// walk a batch tile by tile; the multi-filter kernel (cf_batch.cu) hands
// each warp tiles of many filters.  Every lane of the warp must call these
// (they use warp votes).
// ---------------------------------------------------------------------------
struct TileCounts {
  uint32_t ok = 0, fail = 0, cont = 0;
  CasCount cas;  // failed CAS attempts by retry depth (note_cas_fail)
};

// Appends key indices to a filter's eviction queue: the K keys of every
// lane of a warp tile with one atomic on the queue counter (a single
// counter that all warps share).
struct QueuePush {
  unsigned int* count;
  uint32_t* queue;
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
      if (need[k]) queue[pos + __popc(bal[k] & lt)] = idx[k];
      pos += __popc(bal[k]);
    }
  }
};

// Insert, phase 1 (Alg. 1 direct insertion into i1, then i2).  Keys whose
// two buckets are both full go to the eviction queue; phase 2 runs them
// separately so that the few long eviction chains do not hold whole warps
// of finished keys.
template <class G, int K, class Push, bool RT = true>
__device__ __forceinline__ void tile_insert(const DevFilter& d,
                                            const uint64_t* __restrict__ keys,
                                            uint64_t n, uint64_t base,
                                            uint32_t lane,
                                            uint8_t* __restrict__ flags,
                                            uint32_t* __restrict__ evout,
                                            const Push& push, TileCounts& c) {
  bool valid[K];
  uint32_t bkt[K], tag[K];
  int r1[K], r2[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t i = base + uint64_t(k) * 32 + lane;
    valid[k] = i < n;
    const KeyHash kh = hash_primary<G>(d, valid[k] ? ld_stream_u64(keys + i) : 0ull);
    bkt[k] = kh.i1;
    tag[k] = kh.fp;
  }
  cas_many<G, K, true, RT>(d, bkt, tag, valid, r1, c.cas);
  // Alternate buckets only for the keys whose primary bucket was full.
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    act[k] = valid[k] && r1[k] == TI_FULL;
    if (act[k]) {
      bkt[k] = alt_index<G>(d, bkt[k], tag[k]);
      tag[k] |= G::kChoice;
    }
  }
  cas_many<G, K, true, RT>(d, bkt, tag, act, r2, c.cas);
  bool need[K];
  uint32_t qidx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t idx = uint32_t(base + uint64_t(k) * 32 + lane);
    need[k] = act[k] && r2[k] == TI_FULL;
    qidx[k] = idx;
    const bool ok = valid[k] && (r1[k] == TI_OK || (act[k] && r2[k] == TI_OK));
    const bool cont = valid[k] && (r1[k] == TI_CONTENTION ||
                                   (act[k] && r2[k] == TI_CONTENTION));
    if (ok) {
      c.ok++;
      if (flags) st_flag(flags + idx, 1);
      if (evout) evout[idx] = 0;
    } else if (cont) {
      // bkt/tag hold the bucket and tag of the attempt that ran out.
      c.cont++;
      log_victim(d, tag[k], bkt[k]);
      if (flags) st_flag(flags + idx, 2);
      if (evout) evout[idx] = 0;
    }
  }
  push.push_all(need, qidx, lane);
}

// Query (Alg. 2): Find(i1) or Find(i2).  All K first-bucket loads of a
// thread are issued together; the second bucket is hashed and loaded only
// for the keys not found in the first (the short-circuit of Alg. 2).  Whole
// buckets are loaded with single vector loads (up to 256 bits), so the scan
// order of Alg. 2 does not matter: any word matching decides.
template <class G, int K>
__device__ __forceinline__ void tile_contains(const DevFilter& d,
                                              const uint64_t* __restrict__ keys,
                                              uint64_t n, uint64_t base,
                                              uint32_t lane,
                                              uint8_t* __restrict__ flags) {
  bool valid[K], hit[K];
  uint32_t fp[K], bkt[K];
  Bucket<G> bk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t i = base + uint64_t(k) * 32 + lane;
    valid[k] = i < n;
    const KeyHash kh = hash_primary<G>(d, valid[k] ? ld_stream_u64(keys + i) : 0ull);
    fp[k] = kh.fp;
    bkt[k] = kh.i1;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (valid[k]) bk[k] = load_bucket<G, true>(bucket_ptr<G>(d, bkt[k]));
#pragma unroll
  for (int k = 0; k < K; ++k) {
    hit[k] = valid[k] && bucket_has<G>(bk[k], fp[k]);
    if (valid[k] && !hit[k]) {
      bkt[k] = alt_index<G>(d, bkt[k], fp[k]);
      bk[k] = load_bucket<G, true>(bucket_ptr<G>(d, bkt[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (valid[k] && !hit[k]) hit[k] = bucket_has<G>(bk[k], fp[k] | G::kChoice);
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (valid[k]) st_flag(flags + base + uint64_t(k) * 32 + lane, hit[k] ? 1 : 0);
}

// Delete (Alg. 3): TryRemove(i1) or TryRemove(i2), the K keys' CASes
// issued together.
template <class G, int K, bool RT = true>
__device__ __forceinline__ void tile_remove(const DevFilter& d,
                                            const uint64_t* __restrict__ keys,
                                            uint64_t n, uint64_t base,
                                            uint32_t lane,
                                            uint8_t* __restrict__ flags,
                                            TileCounts& c) {
  bool valid[K];
  uint32_t bkt[K], tag[K];
  int r1[K], r2[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint64_t i = base + uint64_t(k) * 32 + lane;
    valid[k] = i < n;
    const KeyHash kh = hash_primary<G>(d, valid[k] ? ld_stream_u64(keys + i) : 0ull);
    bkt[k] = kh.i1;
    tag[k] = kh.fp;
  }
  cas_many<G, K, false, RT>(d, bkt, tag, valid, r1, c.cas);
  bool act[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    act[k] = valid[k] && r1[k] == TI_FULL;
    if (act[k]) {
      bkt[k] = alt_index<G>(d, bkt[k], tag[k]);
      tag[k] |= G::kChoice;
    }
  }
  cas_many<G, K, false, RT>(d, bkt, tag, act, r2, c.cas);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!valid[k]) continue;
    int r;
    if (r1[k] == TI_OK || (act[k] && r2[k] == TI_OK)) {
      r = 1;
      c.ok++;
    } else if (r1[k] == TI_CONTENTION || (act[k] && r2[k] == TI_CONTENTION)) {
      r = 2;
      c.cont++;
    } else {
      r = 0;
      c.fail++;
    }
    if (flags) st_flag(flags + base + uint64_t(k) * 32 + lane, uint8_t(r));
  }
}

// Phase 2 of the insert for one queued key: the eviction loop, its victim,
// its flag.  Returns the flag value; adds the overwrites to *ev_total.
template <class G, int FW = G::B / 2>
__device__ __forceinline__ int evict_one(const DevFilter& d, uint64_t key,
                                         uint32_t i, uint8_t* flags,
                                         uint32_t* evout, uint32_t& ev_total,
                                         EvictCounters& ec) {
  const KeyHash kh = hash_key<G>(d, key);
  uint32_t ev = 0, vt = 0;
  uint64_t vb = 0;
  const int r = evict_key<G, FW>(d, kh, ev, vt, vb, ec);
  if (r != EV_OK) log_victim(d, vt, vb);
  if (flags) st_flag(flags + i, uint8_t(r));
  if (evout) evout[i] = ev;
  ev_total += ev;
  return r;
}

// ---------------------------------------------------------------------------
// Single-filter kernels: a persistent grid walks the batch's tiles.
// ---------------------------------------------------------------------------
template <class G, int K, int MINB = CF_MINB_MUT, bool RT = false>
__global__ void __launch_bounds__(kBlock, MINB)
k_insert_direct(DevFilter d, const uint64_t* __restrict__ keys, uint32_t n,
                uint8_t* __restrict__ flags, uint32_t* __restrict__ evout,
                uint32_t* __restrict__ queue) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gw = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  TileCounts c;
  const QueuePush push{&d.ctrl->queue_count, queue};
  for (uint64_t base = gw * (32u * K); base < n; base += nw * (32u * K))
    tile_insert<G, K, QueuePush, RT>(d, keys, n, base, lane, flags, evout, push, c);
  block_add(&d.ctrl->occupancy, c.ok);
  block_add(&d.ctrl->insert_ok, c.ok);
  block_add(&d.ctrl->insert_fail, c.cont);
  block_add(&d.ctrl->contention, c.cont);
  cas_count_block_add(d, c.cas);
  if (c.cont) atomicOr(&d.ctrl->error_word, 1u);
}

// Insert, phase 2: the eviction loop for every queued key.  Chains have
// very different lengths, so a lane does not run one chain to its end:
// every warp iteration runs ONE round of each lane's chain, and lanes whose
// chain ended take the next key of the warp's share of the queue.  Each
// warp owns a contiguous share (no shared cursor to contend on), and warps
// stay full until their share runs dry instead of waiting for their
// longest chain.  The queue length is read on the device, so no host round
// trip separates the two phases; the last block to finish resets the queue.
// FROM_HASH: keys[] holds the keys' 64-bit hashes instead of the keys (the
// slice-partitioned path queues positions of its hash records).
//
// A chain's start costs three dependent loads (queue entry, key, first
// bucket), about as long as a round or two.  So each lane prepares its next
// chain while the current one runs, one stage per iteration, every stage
// using what the previous iteration loaded: take and load the queue entry,
// load the key, load the first bucket.  When the chain ends, the next one
// starts from the prepared words at once.  (The words may be a few rounds
// old: a stale word only costs the CAS that detects it.)
//
// map / min_q: when map is given and at least min_q keys are queued, the
// BFS rounds ask the full-bucket map (built by k_fullmap just before, on the
// same rule) whether candidates' alternate buckets are open (bfs_round_map).
template <class G, bool FROM_HASH = false>
__global__ void __launch_bounds__(kBlock, CF_MINB_EVICT)
k_insert_evict(DevFilter d, const uint64_t* __restrict__ keys,
               uint8_t* __restrict__ flags, uint32_t* __restrict__ evout,
               const uint32_t* __restrict__ queue, uint32_t* map, uint32_t min_q,
               const uint32_t* levels_on) {
  // levels_on: nonzero when the slice-grouped eviction levels took this
  // queue (cf_levels.cuh); the kernel then only resets the queue.
  const uint32_t qn = levels_on && __ldcg(levels_on)
                          ? 0u
                          : *reinterpret_cast<volatile unsigned int*>(&d.ctrl->queue_count);
  const bool use_map = map != nullptr && qn >= min_q && d.eviction == 0;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t n_warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t next = uint32_t(uint64_t(qn) * warp / n_warps);
  const uint32_t end = uint32_t(uint64_t(qn) * (warp + 1) / n_warps);
  uint32_t n_ok = 0, n_fail = 0, n_ev = 0;
  EvictCounters ec;
  Chain<G> c{};
  uint32_t idx = 0;
  bool active = false;
  // The lane's next chain: stage 0 none, 1 queue entry pidx loading, 2 key
  // pkey loading, 3 its head pch computed and its first bucket pbk loading
  // (the head is computed once: its hashes serve the chain's start).
  uint32_t pst = 0, pidx = 0;
  uint64_t pkey = 0;
  ChainHead<G> pch{};
  Bucket<G> pbk{};
  auto key_h = [&](uint64_t k) { return FROM_HASH ? k : xxh64_u64(k); };
  for (;;) {
    if (CF_EVICT_PREP && pst == 2 && d.max_ev != 0) {
      pch = chain_head<G>(d, key_h(pkey));
      pbk = load_bucket_ev<G>(bucket_ptr<G>(d, pch.cur));
      pst = 3;
    } else if (CF_EVICT_PREP && pst == 1) {
      pkey = keys[pidx];
      pst = 2;
    }
    if (next < end) {
      const bool want = pst == 0 && (CF_EVICT_PREP || !active);
      const unsigned need = __ballot_sync(0xFFFFFFFFu, want);
      if (want) {
        const uint32_t e = next + __popc(need & ((1u << lane) - 1u));
        if (e < end) {
          pidx = queue[e];
          pst = 1;
        }
      }
      next += __popc(need);
    }
    if (!active && pst != 0) {
      if (pst == 1) pkey = keys[pidx];  // nothing to overlap these loads with
      const bool pst3 = pst == 3;
      idx = pidx;
      pst = 0;
      if (d.max_ev == 0) {
        const KeyHash kh = hash_from_h<G>(d, key_h(pkey));
        log_victim(d, kh.fp, kh.i1);
        if (flags) st_flag(flags + idx, EV_FAIL);
        if (evout) evout[idx] = 0;
        n_fail++;
      } else {
        if (!pst3) {
          pch = chain_head<G>(d, key_h(pkey));
          pbk = load_bucket_ev<G>(bucket_ptr<G>(d, pch.cur));
        }
        c = chain_start_loaded<G>(pch, pbk);
        active = true;
      }
    }
    if (!__any_sync(0xFFFFFFFFu, active)) {
      if (next >= end) break;
      continue;
    }
    if (active) {
      uint32_t vt = 0;
      uint64_t vb = 0;
      const int r = use_map ? evict_round_map<G>(d, c, map, vt, vb, ec)
                            : evict_round<G, EvictFW<G>::value>(d, c, vt, vb, ec);
      if (r != ROUND_CONTINUE) {
        if (r != EV_OK) log_victim(d, vt, vb);
        if (flags) st_flag(flags + idx, uint8_t(r));
        if (evout) evout[idx] = c.ev;
        n_ev += c.ev;
        if (r == EV_OK) n_ok++; else n_fail++;
        active = false;
      }
    }
  }
  block_add(&d.ctrl->occupancy, n_ok);
  block_add(&d.ctrl->insert_ok, n_ok);
  block_add(&d.ctrl->insert_fail, n_fail);
  block_add(&d.ctrl->evictions, n_ev);
  block_add(&d.ctrl->rollbacks, ec.rollbacks);
  block_add(&d.ctrl->rollback_lost, ec.rollback_lost);
  block_add(&d.ctrl->contention, ec.contention);
  cas_count_block_add(d, ec.cas);
  if (ec.contention) atomicOr(&d.ctrl->error_word, 1u);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&d.ctrl->done_blocks, 1u);
    if (prev == gridDim.x - 1) {
      d.ctrl->queue_count = 0;
      d.ctrl->done_blocks = 0;
      __threadfence();
    }
  }
}

// The full-bucket map of the eviction loop (see bfs_round_map): bit j set
// iff bucket j has no empty slot, from one pass over the table.  A warp
// reads 32 consecutive buckets (one per lane, coalesced) and writes their 32
// bits as one word.  Runs only when at least min_q keys are queued, the
// rule k_insert_evict applies to use the map.
template <class G>
__global__ void __launch_bounds__(kBlock)
k_fullmap(DevFilter d, uint32_t* __restrict__ map, uint32_t min_q) {
  const uint32_t qn = *reinterpret_cast<volatile unsigned int*>(&d.ctrl->queue_count);
  if (qn < min_q || d.eviction != 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&d.ctrl->map_builds, 1ull);
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gw = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const uint64_t groups = (d.m + 31) >> 5;
  for (uint64_t g = gw; g < groups; g += nw) {
    const uint64_t j = (g << 5) + lane;
    bool full = false;
    if (j < d.m) full = !has_empty<G>(load_bucket<G, true>(bucket_ptr<G>(d, j)));
    const unsigned bits = __ballot_sync(0xFFFFFFFFu, full);
    if (lane == 0) map_store(map + g, bits);
  }
}

// TryInsert that keeps an exact full-bucket map (one thread only).
template <class G>
__device__ __forceinline__ int try_insert_mapped(const DevFilter& d, uint64_t j,
                                                 uint32_t tag, uint32_t* map) {
  Bucket<G> bk = load_bucket<G, false>(bucket_ptr<G>(d, j));
  CasCount first;  // one thread: no CAS ever fails
  const int r = try_insert_loaded<G>(d, j, tag, bk, first);
  if (map && r == TI_OK && !has_empty<G>(bk)) map_set(d, map, j);
  return r;
}

// The whole insert of Alg. 1 + Sec. 4.6.1, one thread, keys in order
// (deterministic placement; used to compare with a sequential
// implementation bit for bit).  With a map (built from the table just
// before and kept exact here), the BFS rounds take their candidates'
// open / full answers from it (bfs_round_map).
template <class G>
__global__ void k_insert_serial(DevFilter d, const uint64_t* __restrict__ keys,
                                uint64_t n, uint8_t* __restrict__ flags,
                                uint32_t* __restrict__ evout, uint32_t* map) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  EvictCounters ec;
  unsigned long long n_ok = 0, n_fail = 0, n_ev = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const KeyHash kh = hash_key<G>(d, keys[i]);
    uint32_t ev = 0, vt = 0;
    uint64_t vb = 0;
    int r;
    const int a = try_insert_mapped<G>(d, kh.i1, kh.fp, map);
    if (a == TI_OK) {
      r = EV_OK;
    } else if (a == TI_CONTENTION) {
      r = EV_CONTENTION;
      vt = kh.fp;
      vb = kh.i1;
    } else {
      const int b = try_insert_mapped<G>(d, kh.i2, kh.fp | G::kChoice, map);
      if (b == TI_OK) {
        r = EV_OK;
      } else if (b == TI_CONTENTION) {
        r = EV_CONTENTION;
        vt = kh.fp | G::kChoice;
        vb = kh.i2;
      } else if (map && d.eviction == 0) {
        r = evict_key_map<G>(d, kh, map, ev, vt, vb, ec);
      } else {
        r = evict_key<G>(d, kh, ev, vt, vb, ec);
      }
    }
    if (r != EV_OK) log_victim(d, vt, vb);
    if (flags) flags[i] = uint8_t(r);
    if (evout) evout[i] = ev;
    n_ev += ev;
    if (r == EV_OK) n_ok++; else n_fail++;
  }
  atomicAdd(&d.ctrl->occupancy, n_ok);
  atomicAdd(&d.ctrl->insert_ok, n_ok);
  atomicAdd(&d.ctrl->insert_fail, n_fail);
  atomicAdd(&d.ctrl->evictions, n_ev);
  atomicAdd(&d.ctrl->rollbacks, (unsigned long long)ec.rollbacks);
  atomicAdd(&d.ctrl->rollback_lost, (unsigned long long)ec.rollback_lost);
  atomicAdd(&d.ctrl->contention, (unsigned long long)ec.contention);
}

template <class G, int K>
__global__ void __launch_bounds__(kBlock)
k_contains(DevFilter d, const uint64_t* __restrict__ keys, uint64_t n,
           uint8_t* __restrict__ flags) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gw = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t base = gw * (32u * K); base < n; base += nw * (32u * K))
    tile_contains<G, K>(d, keys, n, base, lane, flags);
}

template <class G, int K, int MINB = CF_MINB_MUT, bool RT = false>
__global__ void __launch_bounds__(kBlock, MINB)
k_remove(DevFilter d, const uint64_t* __restrict__ keys, uint64_t n,
         uint8_t* __restrict__ flags) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gw = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  TileCounts c;
  for (uint64_t base = gw * (32u * K); base < n; base += nw * (32u * K))
    tile_remove<G, K, RT>(d, keys, n, base, lane, flags, c);
  block_add(&d.ctrl->occupancy, c.ok, /*negate=*/true);
  block_add(&d.ctrl->remove_ok, c.ok);
  block_add(&d.ctrl->remove_fail, c.fail + c.cont);
  block_add(&d.ctrl->contention, c.cont);
  cas_count_block_add(d, c.cas);
  if (c.cont) atomicOr(&d.ctrl->error_word, 1u);
}

// Hash export for tests: fp, i1, i2 per key.
template <class G>
__global__ void k_hash(DevFilter d, const uint64_t* __restrict__ keys,
                       uint64_t n, uint32_t* fp, uint64_t* i1, uint64_t* i2) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n;
       i += uint64_t(gridDim.x) * blockDim.x) {
    const KeyHash kh = hash_key<G>(d, keys[i]);
    if (fp) fp[i] = kh.fp;
    if (i1) i1[i] = kh.i1;
    if (i2) i2[i] = kh.i2;
  }
}

// Test export: load bucket j through the (in bounds-checked builds,
// checked) bucket address and add its nonzero slot count to *out.
template <class G>
__global__ void k_touch(DevFilter d, uint64_t j, unsigned long long* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const Bucket<G> bk = load_bucket<G, false>(bucket_ptr<G>(d, j));
  uint32_t c = 0;
#pragma unroll
  for (int q = 0; q < G::kWpb; ++q) {
    if constexpr (G::kW32)
      c += G::kTpw - __popc(zero_lanes<G>(bk.w[q]));
    else
      c += G::kTpw - __popcll(zero_lanes<G>(bk.w[q]));
  }
  atomicAdd(out, (unsigned long long)c);
}

// Number of nonzero slots, added to *out.
template <class G>
__global__ void __launch_bounds__(kBlock)
k_count(DevFilter d, unsigned long long* out) {
  using W = typename G::Word;
  const W* t = reinterpret_cast<const W*>(d.table);
  const uint64_t words = d.m * G::kWpb;
  uint32_t c = 0;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < words;
       i += uint64_t(gridDim.x) * blockDim.x) {
    const W w = t[i];
    if constexpr (G::kW32)
      c += G::kTpw - __popc(zero_lanes<G>(w));
    else
      c += G::kTpw - __popcll(zero_lanes<G>(w));
  }
  block_add(out, c);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
int device_sm_count();
int cached_occupancy(const void* fn, int block);

template <class F>
inline unsigned persistent_grid(F* fn, uint64_t work_items, int per_block,
                                int block = kBlock) {
  const int occ = cached_occupancy(reinterpret_cast<const void*>(fn), block);
  const uint64_t cap = uint64_t(device_sm_count()) * uint64_t(occ > 0 ? occ : 1);
  uint64_t need = (work_items + per_block - 1) / per_block;
  if (need < 1) need = 1;
  return unsigned(need < cap ? need : cap);
}

// Grid of the eviction kernel: CF_EVICT_BPSM blocks per SM (0: as many as
// fit).  Its chains are bound by dependent random accesses, and more chains
// in flight only add queueing (2^28-bucket workload, eviction ms per step
// at 1 / 2 / 3 / 4 / 6 blocks per SM: 58.0 / 46.2 / 48.3 / 48.8 / 48.7).
// With the full-bucket map a round loads one bucket from DRAM instead of
// b/2, and the loop becomes bound by the latency of its dependent round
// trips instead: more chains in flight pay (eviction ms per step at 2 / 3
// / 4 blocks per SM: 39.4 / 36.7 / 37.9 with the map, 46.0 / 48.0 / 48.3
// without), CF_EVICT_BPSM_MAP blocks per SM for launches that may use it.
#ifndef CF_EVICT_BPSM
#define CF_EVICT_BPSM 2
#endif
#ifndef CF_EVICT_BPSM_MAP
#define CF_EVICT_BPSM_MAP 3
#endif
inline unsigned evict_grid(const void* fn, bool map = false) {
  const int occ = cached_occupancy(fn, kBlock);
  const int want = map ? CF_EVICT_BPSM_MAP : CF_EVICT_BPSM;
  const int per = want > 0 && want < occ ? want : occ;
  return unsigned(device_sm_count() * (per > 0 ? per : 1));
}

// Optional per-launch timing: the host side records CUDA events around each
// kernel launch on the launching stream (cf_set_kernel_timing).
enum KernelKind : int {
  KK_INSERT_DIRECT = 0,
  KK_INSERT_EVICT = 1,
  KK_CONTAINS = 2,
  KK_REMOVE = 3,
  KK_SLICE_SPLIT = 4,   // slice-partitioned path: scatter
  KK_SLICE_PROBE1 = 5,  // ... bucket i1 pass
  KK_SLICE_PROBE2 = 6,  // ... bucket i2 pass
  KK_SLICE_MERGE = 7,   // ... merge + out (results back to key order)
  KK_EVICT_MAP = 8,     // full-bucket map of the eviction loop
  KK_H2D = 9,           // host-buffer calls: key copies to the device
  KK_D2H = 10,          // ... flag copies back to the host
  KK_EVICT_LEVEL = 11,  // slice-grouped eviction levels (seed + levels)
  KK_NUM = 12
};

// The full-bucket map of one insert call: bits (m/32 words, rounded up) or
// null, and the least number of queued keys for which it is built and used.
struct EvictMap {
  uint32_t* bits = nullptr;
  uint32_t min_q = 0;
  // The slice-grouped eviction levels (sliced passes only; lv.rec[0] null:
  // none).
  LevelBufs lv{};
};
struct KernelTimer {
  virtual void begin(int kind, cudaStream_t s) = 0;
  virtual void end(int kind, cudaStream_t s) = 0;
  virtual ~KernelTimer() = default;
};

template <class G>
struct Launch {
  static constexpr int KQ = Tiles<G, false>::K;
  static constexpr int KM = Tiles<G, true>::K;
  // Resident blocks of the mutating kernels for an L2-resident table.
  static constexpr int MINB_L2 = G::kBucketBytes == 16 ? CF_MINB_MUT : CF_MINB_MUT_L2;
  static bool l2_table(const DevFilter& d) { return d.m * G::kBucketBytes <= kL2TableBytes; }

  static cudaError_t contains(const DevFilter& d, const uint64_t* keys,
                              uint64_t n, uint8_t* flags, cudaStream_t s,
                              KernelTimer* t) {
    auto fn = k_contains<G, KQ>;
    if (t) t->begin(KK_CONTAINS, s);
    fn<<<persistent_grid(fn, n, kBlock * KQ), kBlock, 0, s>>>(d, keys, n, flags);
    if (t) t->end(KK_CONTAINS, s);
    return cudaGetLastError();
  }
  static cudaError_t remove(const DevFilter& d, const uint64_t* keys,
                            uint64_t n, uint8_t* flags, cudaStream_t s,
                            KernelTimer* t) {
    auto fn = d.max_cas != kMaxCas ? k_remove<G, KM, CF_MINB_MUT, true>
              : l2_table(d)        ? k_remove<G, KM, MINB_L2>
                                   : k_remove<G, KM>;
    if (t) t->begin(KK_REMOVE, s);
    fn<<<persistent_grid(fn, n, kBlock * KM), kBlock, 0, s>>>(d, keys, n, flags);
    if (t) t->end(KK_REMOVE, s);
    return cudaGetLastError();
  }
  // The full-bucket map before an eviction launch (a no-op launch unless
  // at least em.min_q keys are queued).
  static cudaError_t fullmap(const DevFilter& d, const EvictMap& em, cudaStream_t s,
                             KernelTimer* t) {
    if (!em.bits) return cudaSuccess;
    auto fm = k_fullmap<G>;
    if (t) t->begin(KK_EVICT_MAP, s);
    fm<<<persistent_grid(fm, d.m, kBlock), kBlock, 0, s>>>(d, em.bits, em.min_q);
    if (t) t->end(KK_EVICT_MAP, s);
    return cudaGetLastError();
  }
  static cudaError_t insert_chunk(const DevFilter& d, const uint64_t* keys,
                                  uint32_t n, uint8_t* flags, uint32_t* evout,
                                  uint32_t* queue, const EvictMap& em, cudaStream_t s,
                                  KernelTimer* t) {
    auto f1 = d.max_cas != kMaxCas ? k_insert_direct<G, KM, CF_MINB_MUT, true>
              : l2_table(d)        ? k_insert_direct<G, KM, MINB_L2>
                                   : k_insert_direct<G, KM>;
    if (t) t->begin(KK_INSERT_DIRECT, s);
    f1<<<persistent_grid(f1, n, kBlock * KM), kBlock, 0, s>>>(d, keys, n, flags,
                                                             evout, queue);
    if (t) t->end(KK_INSERT_DIRECT, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = fullmap(d, em, s, t);
    if (e != cudaSuccess) return e;
    auto f2 = k_insert_evict<G>;
    if (t) t->begin(KK_INSERT_EVICT, s);
    f2<<<evict_grid(reinterpret_cast<const void*>(f2), em.bits != nullptr), kBlock, 0, s>>>(
        d, keys, flags, evout, queue, em.bits, em.min_q, nullptr);
    if (t) t->end(KK_INSERT_EVICT, s);
    return cudaGetLastError();
  }
  // map: null, or a full-bucket map to build now and keep exact (BFS only).
  static cudaError_t insert_serial(const DevFilter& d, const uint64_t* keys,
                                   uint64_t n, uint8_t* flags, uint32_t* evout,
                                   uint32_t* map, cudaStream_t s) {
    if (map) {
      cudaError_t e = fullmap(d, EvictMap{map, 0}, s, nullptr);
      if (e != cudaSuccess) return e;
    }
    k_insert_serial<G><<<1, 32, 0, s>>>(d, keys, n, flags, evout, map);
    return cudaGetLastError();
  }
  static cudaError_t hash(const DevFilter& d, const uint64_t* keys, uint64_t n,
                          uint32_t* fp, uint64_t* i1, uint64_t* i2,
                          cudaStream_t s) {
    auto fn = k_hash<G>;
    fn<<<persistent_grid(fn, n, kBlock), kBlock, 0, s>>>(d, keys, n, fp, i1, i2);
    return cudaGetLastError();
  }
  static cudaError_t touch(const DevFilter& d, uint64_t j, unsigned long long* out,
                           cudaStream_t s) {
    k_touch<G><<<1, 32, 0, s>>>(d, j, out);
    return cudaGetLastError();
  }
  static cudaError_t count(const DevFilter& d, unsigned long long* out,
                           cudaStream_t s) {
    auto fn = k_count<G>;
    fn<<<persistent_grid(fn, d.m * G::kWpb, kBlock), kBlock, 0, s>>>(d, out);
    return cudaGetLastError();
  }
};

struct Ops {
  cudaError_t (*contains)(const DevFilter&, const uint64_t*, uint64_t,
                          uint8_t*, cudaStream_t, KernelTimer*);
  cudaError_t (*remove)(const DevFilter&, const uint64_t*, uint64_t, uint8_t*,
                        cudaStream_t, KernelTimer*);
  cudaError_t (*insert_chunk)(const DevFilter&, const uint64_t*, uint32_t,
                              uint8_t*, uint32_t*, uint32_t*, const EvictMap&,
                              cudaStream_t, KernelTimer*);
  cudaError_t (*insert_serial)(const DevFilter&, const uint64_t*, uint64_t,
                               uint8_t*, uint32_t*, uint32_t*, cudaStream_t);
  cudaError_t (*hash)(const DevFilter&, const uint64_t*, uint64_t, uint32_t*,
                      uint64_t*, uint64_t*, cudaStream_t);
  cudaError_t (*count)(const DevFilter&, unsigned long long*, cudaStream_t);
  // Slice-partitioned insert / contains / remove of one chunk (op: 0 / 1 / 2).
  cudaError_t (*sliced)(const DevFilter&, int, const uint64_t*, uint64_t,
                        uint8_t*, const SliceBufs&, uint32_t*, const EvictMap&,
                        cudaStream_t, KernelTimer*);
  // The same pass in parts: begin, scatter of keys [dst_off, dst_off + n)
  // (repeatable), finish (see SliceLaunch).
  cudaError_t (*sliced_begin)(const SliceBufs&, cudaStream_t);
  cudaError_t (*sliced_scatter)(const DevFilter&, const uint64_t*, uint64_t, uint64_t,
                                int, const SliceBufs&, cudaStream_t, KernelTimer*);
  cudaError_t (*sliced_finish)(const DevFilter&, int, uint64_t, uint8_t*,
                               const SliceBufs&, uint32_t*, const EvictMap&,
                               cudaStream_t, KernelTimer*);
  // Test export: one bucket loaded through the kernels' addressing.
  cudaError_t (*touch)(const DevFilter&, uint64_t, unsigned long long*, cudaStream_t);
};

// ops_for<G>() (the table of one geometry) is defined in cf_slice.cuh.

// One per translation unit (fingerprint width).
const Ops* ops_f8(int b, int policy);
const Ops* ops_f16(int b, int policy);
const Ops* ops_f32(int b, int policy);

inline const Ops* get_ops(int f, int b, int policy) {
  switch (f) {
    case 8: return ops_f8(b, policy);
    case 16: return ops_f16(b, policy);
    case 32: return ops_f32(b, policy);
    default: return nullptr;
  }
}

}  // namespace cfk
