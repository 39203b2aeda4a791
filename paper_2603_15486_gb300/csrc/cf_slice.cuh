// Slice-partitioned execution of query (Alg. 2), delete (Alg. 3) and the
// direct phase of the insert (Alg. 1), for tables much larger than L2.
//
// A random bucket access to a table far larger than L2 costs one DRAM round
// trip that delivers about four 32-byte sectors, and the plain kernels are
// bound by the rate of those round trips.  Here a batch is first grouped by
// the slice of its primary bucket (a slice = 2^shift consecutive buckets,
// sized to a fraction of L2), and the grouped records are then processed in
// order: all warps work inside one or two slices at a time, so a slice's
// buckets come from DRAM about once and every further access hits L2.
// Records left pending by their primary bucket (not found, not removed, or
// the bucket was full) are grouped again by the slice of their alternate
// bucket and processed the same way.  Results go back to the caller's key
// order through the two permutations; both are made of runs (one per block
// tile and slice), which keeps those gathers local.
//
// Bucket loads here use ld.global.cg (cached in L2 at normal priority): the
// non-coherent .nc form of the plain query kernel left the slice's lines
// to be evicted by the streams and re-fetched from DRAM.
//
// Every key still runs Alg. 1 / 2 / 3 on its own: bucket i1 first, bucket i2
// only if i1 did not settle it, the eviction loop only if both were full.
// Only the interleaving between keys changes, which the concurrent kernels
// leave open anyway.
//
// Passes over a chunk of n keys, S slices:
//   hist     keys -> per-slice counts of i1's slice
//   scan     exclusive prefix of the counts -> scatter cursors
//   scatter  keys -> rec1 (the 64-bit hash of each key, grouped by slice),
//            dst[j] = rec1 position of key j
//   probe1   rec1 in order (tiles staged in shared memory by TMA bulk
//            copies): the operation on bucket i1; pending records -> rec2
//            (grouped by i2's slice, cap2 records per slice, overflow in a
//            spill region after the slices), link[p] = rec2 position
//   probe2   rec2 in order: the operation on bucket i2; an insert whose two
//            buckets are full joins the eviction queue (by rec2 position)
//   evict    (insert) the eviction loop on the queued rec2 records
//   merge    f1[p] = f2[link[p]] wherever f1[p] is pending
//   out      flags[j] = f1[dst[j]]
// Without a flags array the passes that only carry results (dst, f1, link,
// f2, merge, out) are skipped.
#pragma once

#include "cf_kernels.cuh"

namespace cfk {

constexpr uint8_t kPending = 0xFF;
// Per-slice counters are spread one per 128-byte line (kCtrStride words
// apart): every block tile bumps one counter per slice, and counters packed
// into a few lines would serialise those atomics on a few L2 slices.
constexpr uint32_t kCtrStride = 32;
// fill2 holds S per-slice counters, then the spill count (index S) and the
// dynamic tile counters of probe2 (S + 1) and probe1 (S + 2): kFill2Extra.

enum : int { SOP_INSERT = 0, SOP_CONTAINS = 1, SOP_REMOVE = 2 };

// Tuning of the bucket passes (2^28-bucket workload, ms per step): three
// resident blocks per SM rather than two (136.4 vs 141.9), and four keys
// per round for the delete passes (delete phase 10.3 vs 11.6 ms; insert and
// query are faster with eight).  CF_SLICE_KMUT overrides the delete K (and
// caps the insert K when set), CF_SLICE_MINB the resident blocks.
#ifndef CF_SLICE_KMUT
#define CF_SLICE_KMUT 0
#endif
#ifndef CF_SLICE_MINB
#define CF_SLICE_MINB 3
#endif
#ifndef CF_SLICE2_MINB
#define CF_SLICE2_MINB CF_SLICE_MINB
#endif
// Minimum resident blocks per SM of the split kernels (hist, scatter): 4
// (64 registers) ran the split in 17.4 ms per step against 18.1 at the
// compiler's own choice.
#ifndef CF_SPLIT_MINB
#define CF_SPLIT_MINB 4
#endif

__device__ __forceinline__ void st_cs_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.global.cs.u32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ uint32_t ld_cs_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) from global to shared memory
// completing on an mbarrier, with bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One thread: expect `bytes` and start the copy of `bytes` (a multiple of 16,
// both addresses 16-byte aligned) from global src to shared dst.  bytes == 0
// only arrives, which completes the phase at once.
__device__ __forceinline__ void bulk_load(uint64_t* bar, void* dst, const void* src,
                                          uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  if (bytes)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Wait for the phase with the given parity to complete; false if it has not
// after a bounded number of polls (the caller reports the timeout).
constexpr uint32_t kMaxMbarPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kMaxMbarPolls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}
constexpr uint32_t kErrAsyncCopy = 4u;  // error_word bit: a bulk copy never completed

// ---------------------------------------------------------------------------
// hist: counts of i1's slice.  Each block bins its keys in shared memory and
// adds its bins to the global histogram once.
// ---------------------------------------------------------------------------
template <class G, int U>
__global__ void __launch_bounds__(kBlock, CF_SPLIT_MINB)
k_slice_hist(DevFilter d, const uint64_t* __restrict__ keys, uint64_t n,
             uint32_t shift, uint32_t S, uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t s_cnt[];
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) s_cnt[s] = 0;
  __syncthreads();
  const uint64_t tile = uint64_t(blockDim.x) * U;
  for (uint64_t t0 = blockIdx.x * tile; t0 < n; t0 += uint64_t(gridDim.x) * tile) {
    uint64_t v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      v[u] = i < n ? ld_stream_u64(keys + i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      if (i < n) atomicAdd(&s_cnt[hash_primary<G>(d, v[u]).i1 >> shift], 1u);
    }
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x)
    if (s_cnt[s]) atomicAdd(&hist[s * kCtrStride], s_cnt[s]);
}

// ---------------------------------------------------------------------------
// scan: exclusive prefix of the S counts in place (one block of 1024), and
// the rec2 fill counters and tile counters zeroed.
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(1024)
k_slice_scan(uint32_t* __restrict__ cursor, uint32_t S, uint32_t* __restrict__ fill2) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < S; base += blockDim.x) {
    const uint32_t s = base + threadIdx.x;
    const uint32_t v = s < S ? cursor[s * kCtrStride] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= uint32_t(o)) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = warp_sum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
        if (lane >= uint32_t(o)) t += y;
      }
      warp_sum[lane] = t;
    }
    __syncthreads();
    if (s < S) cursor[s * kCtrStride] = carry + (warp ? warp_sum[warp - 1] : 0u) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[31];
    __syncthreads();
  }
  for (uint32_t s = threadIdx.x; s < S + kFill2Extra; s += blockDim.x) fill2[s * kCtrStride] = 0;
}

// Exclusive prefix of in[0..S) into out[0..S) by the whole block (each
// thread sums a run of consecutive bins, one warp scans the run sums).
// Ends with a barrier; tmp is 32 words of shared memory.
__device__ __forceinline__ void block_scan_excl(const uint32_t* in, uint32_t* out,
                                                uint32_t S, uint32_t* tmp) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t per = (S + blockDim.x - 1) / blockDim.x;
  const uint32_t b0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t i = 0; i < per; ++i)
    if (b0 + i < S) sum += in[b0 + i];
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= uint32_t(o)) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (blockDim.x >> 5) ? tmp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= uint32_t(o)) t += y;
    }
    tmp[lane] = t;
  }
  __syncthreads();
  uint32_t run = (warp ? tmp[warp - 1] : 0u) + x - sum;
  for (uint32_t i = 0; i < per; ++i)
    if (b0 + i < S) {
      const uint32_t v = in[b0 + i];
      out[b0 + i] = run;
      run += v;
    }
  __syncthreads();
}

template <class G>
__device__ __forceinline__ uint32_t slice_of_h(const DevFilter& d, uint64_t h,
                                               uint32_t shift) {
  return hash_from_h<G>(d, h).i1 >> shift;
}

// ---------------------------------------------------------------------------
// scatter (a multi-split): each block tile of kBlock*U keys is binned by
// slice in shared memory (a rank per key), sorted by slice inside shared
// memory, and written out as one contiguous run per occupied slice (one
// global cursor bump per run), so consecutive threads store consecutive
// records.  dst[] is written in key order.
// Shared memory: 3*S counters + 8*kBlock*U bytes.
// ---------------------------------------------------------------------------
template <class G, int U>
__global__ void __launch_bounds__(kBlock, CF_SPLIT_MINB)
k_slice_scatter(DevFilter d, const uint64_t* __restrict__ keys, uint64_t n,
                uint32_t shift, uint32_t S, uint32_t* __restrict__ cursor,
                uint64_t* __restrict__ rec1, uint32_t* __restrict__ dst) {
  extern __shared__ uint64_t sm64[];
  constexpr uint32_t T = kBlock * U;
  uint64_t* stash = sm64;                                   // [T]
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(sm64 + T);  // [S]
  uint32_t* s_off = s_cnt + S;                              // [S]
  uint32_t* s_base = s_off + S;                             // [S]
  __shared__ uint32_t tmp[32];
  for (uint64_t t0 = blockIdx.x * uint64_t(T); t0 < n; t0 += uint64_t(gridDim.x) * T) {
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) s_cnt[s] = 0;
    __syncthreads();
    uint64_t h[U];
    uint32_t slrk[U];  // slice << 16 | rank
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      h[u] = i < n ? ld_stream_u64(keys + i) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      slrk[u] = 0;
      if (i < n) {
        h[u] = xxh64_u64(h[u]);
        const uint32_t sl = slice_of_h<G>(d, h[u], shift);
        slrk[u] = (sl << 16) | atomicAdd(&s_cnt[sl], 1u);
      }
    }
    __syncthreads();
    block_scan_excl(s_cnt, s_off, S, tmp);
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x)
      if (s_cnt[s]) s_base[s] = atomicAdd(&cursor[s * kCtrStride], s_cnt[s]);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      if (i < n) {
        const uint32_t sl = slrk[u] >> 16, rk = slrk[u] & 0xFFFFu;
        stash[s_off[sl] + rk] = h[u];
        if (dst) st_cs_u32(dst + i, s_base[sl] + rk);
      }
    }
    __syncthreads();
    const uint32_t cnt = uint32_t(n - t0 < T ? n - t0 : T);
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
      const uint64_t hv = stash[j];
      const uint32_t sl = slice_of_h<G>(d, hv, shift);
      rec1[s_base[sl] + (j - s_off[sl])] = hv;
    }
    __syncthreads();
  }
}

// rec2 position of the rk-th pending record of slice s in a block tile,
// from the tile's claim (base = fill2[s] before the claim, cnt records):
// the first cap2 - base go to the slice, the rest to the spill region.
__device__ __forceinline__ uint64_t rec2_pos(uint32_t s, uint32_t rk,
                                             uint32_t base, uint32_t cnt,
                                             uint32_t spill, uint64_t cap2,
                                             uint32_t S) {
  const uint64_t room = base >= cap2 ? 0 : cap2 - base;
  const uint32_t in = room < cnt ? uint32_t(room) : cnt;
  return rk < in ? uint64_t(s) * cap2 + base + rk
                 : uint64_t(S) * cap2 + spill + (rk - in);
}

// ---------------------------------------------------------------------------
// probe1: the operation on bucket i1 for rec1 records in order.  A block
// tile is kBlock*8 records (thread t takes records t, t + kBlock, ...),
// staged in shared memory by a TMA bulk copy issued while the block works
// on the previous tile.  Records left pending are stashed in shared memory,
// sorted by the slice of i2 once per tile, and written to rec2 as one run
// per occupied slice (one claim on fill2 per run).
// Shared memory: 20*T bytes + 4*S counters (T = kBlock*8 = 2048 records).
// ---------------------------------------------------------------------------

constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

template <class G, int OP, int K>
__global__ void __launch_bounds__(kBlock, CF_SLICE_MINB)
k_slice_probe1(DevFilter d, SliceBufs sb, uint32_t n, int want_flags) {
  // R rounds of K records per thread: every tile holds 8 records per thread
  // whatever the bucket size (K = 8 / 4 / 2 / 1 for 8 / 16 / 32 / 64-byte
  // buckets), so the per-tile work (barriers, prefix, claims) stays amortised.
  constexpr int R = 8 / K;
  constexpr int N = R * K;
  constexpr uint32_t T = kBlock * N;
  static_assert(K == 8 || K == 4 || K == 2 || K == 1, "records per thread");
  static_assert(T <= 2048, "shared entries pack an 11-bit tile index");
  extern __shared__ uint64_t sm64[];
  const uint32_t S = sb.n_slices;
  uint64_t* pref = sm64;                                            // [T] next tile's records
  uint64_t* stash_h = sm64 + T;                                     // [T] by tile index
  uint32_t* s_order = reinterpret_cast<uint32_t*>(sm64 + 2 * T);   // [T] index | slice << 11
  uint32_t* s_cnt = s_order + T;                                    // [S]
  uint32_t* s_off = s_cnt + S;                                      // [S]
  uint32_t* s_base = s_off + S;                                     // [S]
  uint32_t* s_spill = s_base + S;                                   // [S]
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_next;
  __shared__ __align__(8) uint64_t s_bar;
  TileCounts c;
  // Tiles are handed out in order by a counter, so the blocks at work stay
  // within a window of consecutive tiles (one or two slices) instead of
  // drifting apart as a static grid stride lets them.  One thread copies the
  // next tile's records into shared memory (TMA bulk copy) while the block
  // works on the current one.
  uint32_t* tile_ctr = sb.fill2 + (S + 2) * kCtrStride;
  auto tile_bytes = [&](uint32_t tile) -> uint32_t {
    const uint32_t t0 = tile * T;
    return t0 >= n ? 0u : ((n - t0 < T ? n - t0 : T) * 8u) & ~15u;
  };
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    s_next = atomicAdd(tile_ctr, 1u);
    if (s_next * T < n) bulk_load(&s_bar, pref, sb.rec1 + size_t(s_next) * T, tile_bytes(s_next));
  }
  __syncthreads();
  uint32_t tile = s_next;
  uint32_t parity = 0;
  for (;;) {
    const uint32_t t0 = tile * T;
    if (t0 >= n) break;
    if (!mbar_wait(&s_bar, parity)) {
      // The copy did not complete: report it and leave this tile (its
      // records stay unprocessed; the error bit tells the caller).
      if (threadIdx.x == 0) atomicOr(&d.ctrl->error_word, kErrAsyncCopy);
      mbar_wait(&s_bar, parity);  // once more (bounded) for the copy in flight
      break;
    }
    parity ^= 1u;
    // Record i of this thread: tile index loc(i) = i*kBlock + thread (lane-
    // strided: conflict-free reads of the staged tile, coalesced stores).
    const uint32_t copied = tile_bytes(tile) / 8u;  // records now in pref
    uint64_t hr[N];
    bool vr[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t loc = uint32_t(i) * kBlock + threadIdx.x;
      vr[i] = t0 + loc < n;
      hr[i] = loc < copied ? pref[loc] : (vr[i] ? ld_stream_u64(sb.rec1 + t0 + loc) : 0ull);
    }
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) s_cnt[s] = 0;
    __syncthreads();  // pref consumed, counters zeroed
    if (threadIdx.x == 0) {
      s_next = atomicAdd(tile_ctr, 1u);
      if (s_next * T < n)
        bulk_load(&s_bar, pref, sb.rec1 + size_t(s_next) * T, tile_bytes(s_next));
    }
    uint32_t slrk[N];  // slice << 16 | rank of a pending record, else kNoSlot
#pragma unroll
    for (int r = 0; r < R; ++r) {
      bool valid[K];
      uint32_t bkt[K], tag[K];
      int res[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        valid[k] = vr[r * K + k];
        const KeyHash kh = hash_from_h<G>(d, hr[r * K + k]);
        bkt[k] = kh.i1;
        tag[k] = kh.fp;
      }
      if constexpr (OP == SOP_CONTAINS) {
        Bucket<G> bk[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (valid[k]) bk[k] = load_bucket<G, false>(bucket_ptr<G>(d, bkt[k]));
#pragma unroll
        for (int k = 0; k < K; ++k)
          res[k] = valid[k] && bucket_has<G>(bk[k], tag[k]) ? TI_OK : TI_FULL;
      } else {
        cas_many<G, K, OP == SOP_INSERT>(d, bkt, tag, valid, res);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = r * K + k;
        const uint32_t loc = uint32_t(i) * kBlock + threadIdx.x;
        slrk[i] = kNoSlot;
        uint8_t v = 0;
        if (valid[k] && res[k] == TI_FULL) {
          const uint32_t sl = alt_index<G>(d, bkt[k], tag[k]) >> sb.shift;
          slrk[i] = (sl << 16) | atomicAdd(&s_cnt[sl], 1u);
          stash_h[loc] = hr[i];
          v = kPending;
        } else if (valid[k]) {
          if (res[k] == TI_OK) {
            v = 1;
            c.ok++;
          } else {
            v = 2;
            c.cont++;
            if (OP == SOP_INSERT) log_victim(d, tag[k], bkt[k]);
          }
        }
        if (want_flags && valid[k]) st_flag(sb.f1 + t0 + loc, v);
      }
    }
    __syncthreads();
    block_scan_excl(s_cnt, s_off, S, tmp);
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
      const uint32_t cnt = s_cnt[s];
      if (!cnt) continue;
      const uint32_t base = atomicAdd(&sb.fill2[s * kCtrStride], cnt);
      const uint64_t room = base >= sb.cap2 ? 0 : sb.cap2 - base;
      s_base[s] = base;
      s_spill[s] = room < cnt ? atomicAdd(&sb.fill2[S * kCtrStride], cnt - uint32_t(room))
                              : 0u;
    }
    const uint32_t np = s_off[S - 1] + s_cnt[S - 1];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t loc = uint32_t(i) * kBlock + threadIdx.x;
      uint32_t lk = 0;
      if (slrk[i] != kNoSlot) {
        const uint32_t sl = slrk[i] >> 16, rk = slrk[i] & 0xFFFFu;
        s_order[s_off[sl] + rk] = loc | (sl << 11);
        lk = uint32_t(rec2_pos(sl, rk, s_base[sl], s_cnt[sl], s_spill[sl], sb.cap2, S));
      }
      if (want_flags && vr[i]) sb.link[t0 + loc] = lk;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < np; j += blockDim.x) {
      const uint32_t e = s_order[j];
      const uint32_t sl = e >> 11;
      const uint64_t q = rec2_pos(sl, j - s_off[sl], s_base[sl], s_cnt[sl], s_spill[sl],
                                  sb.cap2, S);
      sb.rec2[q] = stash_h[e & 0x7FFu];
    }
    __syncthreads();
    tile = s_next;
  }
  if constexpr (OP == SOP_INSERT) {
    block_add(&d.ctrl->occupancy, c.ok);
    block_add(&d.ctrl->insert_ok, c.ok);
    block_add(&d.ctrl->insert_fail, c.cont);
    block_add(&d.ctrl->contention, c.cont);
  } else if constexpr (OP == SOP_REMOVE) {
    block_add(&d.ctrl->occupancy, c.ok, /*negate=*/true);
    block_add(&d.ctrl->remove_ok, c.ok);
    block_add(&d.ctrl->remove_fail, c.cont);
    block_add(&d.ctrl->contention, c.cont);
  }
}

// ---------------------------------------------------------------------------
// probe2: the operation on bucket i2 for the rec2 records, slice regions in
// order, then the spill region.  Warp tiles of 32*K positions; positions
// past a region's fill are skipped.
// ---------------------------------------------------------------------------
template <class G, int OP, int K>
__global__ void __launch_bounds__(kBlock, CF_SLICE2_MINB)
k_slice_probe2(DevFilter d, SliceBufs sb, uint64_t n, int want_flags,
               uint32_t* __restrict__ queue) {
  // The filled part of each region (S slices, then the spill region) and
  // its start in the compacted order, so that warps walk only records.
  extern __shared__ uint32_t s_reg[];
  __shared__ uint32_t tmp[32];
  const uint32_t S = sb.n_slices;
  const uint32_t NR = S + 1;
  uint32_t* s_len = s_reg;
  uint32_t* s_start = s_reg + NR;
  for (uint32_t r = threadIdx.x; r < NR; r += blockDim.x) {
    const uint32_t fill = __ldg(sb.fill2 + r * kCtrStride);
    s_len[r] = r < S ? (fill < sb.cap2 ? fill : uint32_t(sb.cap2)) : fill;
  }
  __syncthreads();
  block_scan_excl(s_len, s_start, NR, tmp);
  const uint64_t total = uint64_t(s_start[NR - 1]) + s_len[NR - 1];
  const uint32_t lane = threadIdx.x & 31;
  // R rounds of K positions per thread: tiles of 8 records per thread for
  // every bucket size (see probe1).
  constexpr int R = 8 / K;
  const uint32_t T = blockDim.x * K * R;
  __shared__ uint32_t s_tile;
  uint32_t* tile_ctr = sb.fill2 + (S + 1) * kCtrStride;
  TileCounts c;
  const QueuePush push{&d.ctrl->queue_count, queue};
  // The region (S slices, then the spill region) holding compacted
  // position x: the last one starting at or before x.
  auto region_of = [&](uint64_t x) {
    uint32_t lo = 0, hi = NR;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_start[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
  };
  // Block tiles of T compacted positions, handed out in order by a counter
  // (see probe1); lane-strided inside the tile.
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const uint64_t x0 = uint64_t(s_tile) * T;
    __syncthreads();
    if (x0 >= total) break;
    const uint64_t xl = (x0 + T < total ? x0 + T : total) - 1;
    const uint32_t r0 = region_of(x0), r1 = region_of(xl);
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      bool valid[K];
      uint64_t q[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint64_t x = x0 + uint64_t(rr * K + k) * blockDim.x + threadIdx.x;
        valid[k] = x < total;
        q[k] = 0;
        if (valid[k]) {
          const uint32_t r = r0 == r1 ? r0 : region_of(x);
          q[k] = uint64_t(r) * sb.cap2 + (x - s_start[r]);
        }
      }
      uint32_t bkt[K], tag[K];
      int res[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const KeyHash kh =
            hash_from_h<G>(d, valid[k] ? ld_stream_u64(sb.rec2 + q[k]) : 0ull);
        bkt[k] = alt_index<G>(d, kh.i1, kh.fp);
        tag[k] = kh.fp | G::kChoice;
      }
      if constexpr (OP == SOP_CONTAINS) {
        Bucket<G> bk[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (valid[k]) bk[k] = load_bucket<G, false>(bucket_ptr<G>(d, bkt[k]));
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (valid[k] && want_flags)
            st_flag(sb.f2 + q[k], bucket_has<G>(bk[k], tag[k]) ? 1 : 0);
      } else {
        cas_many<G, K, OP == SOP_INSERT>(d, bkt, tag, valid, res);
        bool to_queue[K];
        uint32_t qidx[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          to_queue[k] = false;
          qidx[k] = uint32_t(q[k]);
          if (valid[k]) {
            uint8_t v;
            if (res[k] == TI_OK) {
              v = 1;
              c.ok++;
            } else if (res[k] == TI_CONTENTION) {
              v = 2;
              c.cont++;
              if (OP == SOP_INSERT) log_victim(d, tag[k], bkt[k]);
            } else {
              v = 0;
              if (OP == SOP_INSERT) to_queue[k] = true;
              else c.fail++;
            }
            if (want_flags && !to_queue[k]) st_flag(sb.f2 + q[k], v);
          }
        }
        if constexpr (OP == SOP_INSERT) push.push_all(to_queue, qidx, lane);
      }
    }
  }
  if constexpr (OP == SOP_INSERT) {
    block_add(&d.ctrl->occupancy, c.ok);
    block_add(&d.ctrl->insert_ok, c.ok);
    block_add(&d.ctrl->insert_fail, c.cont);
    block_add(&d.ctrl->contention, c.cont);
  } else if constexpr (OP == SOP_REMOVE) {
    block_add(&d.ctrl->occupancy, c.ok, /*negate=*/true);
    block_add(&d.ctrl->remove_ok, c.ok);
    block_add(&d.ctrl->remove_fail, c.fail + c.cont);
    block_add(&d.ctrl->contention, c.cont);
  }
}

// ---------------------------------------------------------------------------
// merge: f1[p] = f2[link[p]] for pending records.  A thread takes V groups of
// four records per iteration (V grid strides apart), so that up to 4*V of
// its gathers are in flight together.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pending_mask(uint32_t w) {
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (((w >> (8 * j)) & 0xFFu) == kPending) m |= 1u << j;
  return m;
}

#ifndef CF_MERGE_V
#define CF_MERGE_V 4
#endif
// Minimum resident blocks per SM of merge / out (latency-bound gathers):
// 6 (40 registers) ran them in 8.3 ms per step against 8.6 at 4 and 9.1 at
// the compiler's own choice.
#ifndef CF_MERGE_MINB
#define CF_MERGE_MINB 6
#endif
static __global__ void __launch_bounds__(kBlock, CF_MERGE_MINB)
k_slice_merge(uint8_t* __restrict__ f1, const uint32_t* __restrict__ link,
              const uint8_t* __restrict__ f2, uint64_t n) {
  constexpr int V = CF_MERGE_V;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t n4 = n / 4;
  uint32_t* f1w = reinterpret_cast<uint32_t*>(f1);
  const uint4* link4 = reinterpret_cast<const uint4*>(link);
  for (uint64_t v0 = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v0 < n4;
       v0 += stride * V) {
    uint32_t w[V], pend[V];
    uint4 l[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const uint64_t v = v0 + u * stride;
      w[u] = v < n4 ? ld_cs_u32(f1w + v) : 0u;
      pend[u] = v < n4 ? pending_mask(w[u]) : 0u;
    }
#pragma unroll
    for (int u = 0; u < V; ++u)
      if (pend[u]) l[u] = link4[v0 + u * stride];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      if (!pend[u]) continue;
      const uint32_t ls[4] = {l[u].x, l[u].y, l[u].z, l[u].w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (pend[u] & (1u << j))
          w[u] = (w[u] & ~(0xFFu << (8 * j))) | (uint32_t(f2[ls[j]]) << (8 * j));
      f1w[v0 + u * stride] = w[u];
    }
  }
  for (uint64_t p = n4 * 4 + blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; p < n;
       p += stride)
    if (f1[p] == kPending) f1[p] = f2[link[p]];
}

// ---------------------------------------------------------------------------
// out: flags[j] = f1[dst[j]], V groups of four keys per thread and iteration
// (byte stores when the caller's flags are not 4-byte aligned).
// ---------------------------------------------------------------------------
static __global__ void __launch_bounds__(kBlock, CF_MERGE_MINB)
k_slice_out(const uint32_t* __restrict__ dst, const uint8_t* __restrict__ f1,
            uint8_t* __restrict__ out, uint64_t n) {
  constexpr int V = CF_MERGE_V;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t n4 = n / 4;
  const bool aligned = (reinterpret_cast<uintptr_t>(out) & 3u) == 0;
  const uint4* dst4 = reinterpret_cast<const uint4*>(dst);
  for (uint64_t v0 = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; v0 < n4;
       v0 += stride * V) {
    uint4 p[V];
#pragma unroll
    for (int u = 0; u < V; ++u)
      if (v0 + u * stride < n4) p[u] = dst4[v0 + u * stride];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const uint64_t v = v0 + u * stride;
      if (v >= n4) continue;
      const uint32_t b0 = f1[p[u].x], b1 = f1[p[u].y], b2 = f1[p[u].z], b3 = f1[p[u].w];
      if (aligned) {
        reinterpret_cast<uint32_t*>(out)[v] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
      } else {
        out[4 * v] = uint8_t(b0);
        out[4 * v + 1] = uint8_t(b1);
        out[4 * v + 2] = uint8_t(b2);
        out[4 * v + 3] = uint8_t(b3);
      }
    }
  }
  for (uint64_t j = n4 * 4 + blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < n;
       j += stride)
    out[j] = f1[dst[j]];
}

// ---------------------------------------------------------------------------
// Launch sequence of one chunk.
// ---------------------------------------------------------------------------
template <class G>
struct SliceLaunch {
  static constexpr int KQ = Tiles<G, false>::K;
  // Keys per round: the query's K for insert (unless CF_SLICE_KMUT caps
  // it), half of it (at most 4) for delete.
  static constexpr int KMS = (CF_SLICE_KMUT > 0 && CF_SLICE_KMUT < KQ) ? CF_SLICE_KMUT : KQ;
  static constexpr int KRM = CF_SLICE_KMUT > 0 ? KMS : (KQ >= 8 ? 4 : KQ);
  static constexpr int U = 16;  // keys per thread of a scatter tile

  template <int OP, int K>
  static cudaError_t probes(const DevFilter& d, const SliceBufs& sb, uint64_t n,
                            int want, uint32_t* queue, cudaStream_t s,
                            KernelTimer* t) {
    constexpr uint32_t T = kBlock * 8;
    const size_t smem = size_t(20) * T + size_t(16) * sb.n_slices;
    auto p1 = k_slice_probe1<G, OP, K>;
    if (smem > 48 * 1024) {
      const cudaError_t ea =
          cudaFuncSetAttribute(p1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (ea != cudaSuccess) return ea;
    }
    if (t) t->begin(KK_SLICE_PROBE1, s);
    p1<<<persistent_grid(p1, n, T), kBlock, smem, s>>>(d, sb, uint32_t(n), want);
    if (t) t->end(KK_SLICE_PROBE1, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto p2 = k_slice_probe2<G, OP, K>;
    const size_t smem2 = size_t(2) * (sb.n_slices + 1) * sizeof(uint32_t);
    if (t) t->begin(KK_SLICE_PROBE2, s);
    p2<<<persistent_grid(p2, n, kBlock * 8), kBlock, smem2, s>>>(d, sb, n, want, queue);
    if (t) t->end(KK_SLICE_PROBE2, s);
    return cudaGetLastError();
  }

  static cudaError_t run(const DevFilter& d, int op, const uint64_t* keys,
                         uint64_t n, uint8_t* flags, const SliceBufs& sb,
                         uint32_t* queue, cudaStream_t s, KernelTimer* t) {
    const int want = flags != nullptr;
    const uint32_t S = sb.n_slices;
    if (t) t->begin(KK_SLICE_SPLIT, s);
    cudaError_t e =
        cudaMemsetAsync(sb.cursor, 0, size_t(S) * kCtrStride * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    auto fh = k_slice_hist<G, U>;
    fh<<<persistent_grid(fh, n, kBlock * U), kBlock, S * sizeof(uint32_t), s>>>(
        d, keys, n, sb.shift, S, sb.cursor);
    k_slice_scan<<<1, 1024, 0, s>>>(sb.cursor, S, sb.fill2);
    auto fs = k_slice_scatter<G, U>;
    const size_t smem = size_t(8) * kBlock * U + size_t(12) * S;
    fs<<<persistent_grid(fs, n, kBlock * U), kBlock, smem, s>>>(
        d, keys, n, sb.shift, S, sb.cursor, sb.rec1, want ? sb.dst : nullptr);
    if (t) t->end(KK_SLICE_SPLIT, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // All three operations take the query's K (8 for 8-byte buckets): the
    // bucket accesses hit L2 here, so the mutating passes are latency-bound
    // and want every key's load and CAS of a tile in flight together.
    if (op == SOP_CONTAINS)
      e = probes<SOP_CONTAINS, KQ>(d, sb, n, want, queue, s, t);
    else if (op == SOP_REMOVE)
      e = probes<SOP_REMOVE, KRM>(d, sb, n, want, queue, s, t);
    else
      e = probes<SOP_INSERT, KMS>(d, sb, n, want, queue, s, t);
    if (e != cudaSuccess) return e;
    if (op == SOP_INSERT) {
      auto fe = k_insert_evict<G, true>;
      if (t) t->begin(KK_INSERT_EVICT, s);
      fe<<<evict_grid(reinterpret_cast<const void*>(fe)), kBlock, 0, s>>>(
          d, sb.rec2, want ? sb.f2 : nullptr, nullptr, queue);
      if (t) t->end(KK_INSERT_EVICT, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (!want) return cudaSuccess;
    if (t) t->begin(KK_SLICE_MERGE, s);
    k_slice_merge<<<persistent_grid(k_slice_merge, n, kBlock * 4 * CF_MERGE_V), kBlock, 0,
                    s>>>(sb.f1, sb.link, sb.f2, n);
    k_slice_out<<<persistent_grid(k_slice_out, n, kBlock * 4 * CF_MERGE_V), kBlock, 0, s>>>(
        sb.dst, sb.f1, flags, n);
    if (t) t->end(KK_SLICE_MERGE, s);
    return cudaGetLastError();
  }
};

template <class G>
const Ops* ops_for() {
  static const Ops o = {&Launch<G>::contains, &Launch<G>::remove,
                        &Launch<G>::insert_chunk, &Launch<G>::insert_serial,
                        &Launch<G>::hash, &Launch<G>::count, &SliceLaunch<G>::run};
  return &o;
}

}  // namespace cfk
