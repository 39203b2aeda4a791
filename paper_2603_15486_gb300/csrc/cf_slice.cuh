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
//   scatter  keys -> rec1 (the 64-bit hash of each key, grouped by i1's
//            slice: cap1 records per slice, overflow in a spill region
//            after the slices), dst[j] = rec1 position of key j
//   probe1   rec1 regions in order (tiles staged in shared memory by TMA
//            bulk copies): the operation on bucket i1; pending records ->
//            rec2 (grouped by i2's slice the same way, cap2 records per
//            slice and a spill region); link[p] = the rec2 position of a
//            pending record, else its flag (tagged kSettled)
//   probe2   rec2 regions in order: the operation on bucket i2; an insert
//            whose two buckets are full joins the eviction queue (by rec2
//            position)
//   evict    (insert) the eviction loop on the queued rec2 records
//   merge    f1[p] = the flag in link[p], or f2 at the rec2 position it
//            holds
//   out      flags[j] = f1[dst[j]]
// The region capacities (the expected count plus six standard deviations)
// hold a batch of distinct uniform hashes, so no counting pass precedes the
// scatter; repeated keys or skewed batches only move records to the spill
// region.  Without a flags array the passes that only carry results (dst,
// f1, link, f2, merge, out) are skipped.
#pragma once

#include "cf_kernels.cuh"

namespace cfk {

// link[p] of a rec1 record: its rec2 position while pending, else
// kSettled | flag (every rec2 position lies below kSettled).
constexpr uint32_t kSettled = 0xFFFFFF00u;
// Per-slice counters are spread one per 128-byte line (kCtrStride words
// apart): every block tile bumps one counter per slice, and counters packed
// into a few lines would serialise those atomics on a few L2 slices.
constexpr uint32_t kCtrStride = 32;
// fill1 holds S per-slice counters and the spill count (index S); fill2
// the same for rec2, then the dynamic tile counters of probe2 (S + 1) and
// probe1 (S + 2): kFill2Extra.  The two arrays are zeroed together before
// the scatter.

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
// Threads per block of the bucket passes (probe1 / probe2).
#ifndef CF_SLICE_BLOCK
#define CF_SLICE_BLOCK 256
#endif
constexpr int kSliceBlock = CF_SLICE_BLOCK;
// Minimum resident blocks per SM of the scatter: 4 (64 registers) ran the
// split in 17.4 ms per step against 18.1 at the compiler's own choice.
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

// Position of the rk-th record of slice s in a block tile's run, from the
// tile's claim (base = fill[s] before the claim, cnt records): the first
// cap - base go to the slice's region, the rest to the spill region after
// the S regions.
__device__ __forceinline__ uint64_t region_pos(uint32_t s, uint32_t rk,
                                               uint32_t base, uint32_t cnt,
                                               uint32_t spill, uint64_t cap,
                                               uint32_t S) {
  const uint64_t room = base >= cap ? 0 : cap - base;
  const uint32_t in = room < cnt ? uint32_t(room) : cnt;
  return rk < in ? uint64_t(s) * cap + base + rk
                 : uint64_t(S) * cap + spill + (rk - in);
}

// A block tile's claims: for every slice with s_cnt[s] records, s_base[s] =
// fill[s] before adding them, and s_spill[s] = the spill count before
// adding the part that does not fit the region (fill[S] counts the spill).
// *spilled becomes nonzero if any run of the tile reaches the spill region;
// while it stays zero, the rk-th record of slice s goes to s*cap + s_base[s]
// + rk (all positions fit 32 bits).
__device__ __forceinline__ void claim_runs(const uint32_t* s_cnt, uint32_t* s_base,
                                           uint32_t* s_spill, uint32_t S,
                                           uint32_t* fill, uint64_t cap,
                                           uint32_t* spilled) {
  for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
    const uint32_t cnt = s_cnt[s];
    if (!cnt) continue;
    const uint32_t base = atomicAdd(&fill[s * kCtrStride], cnt);
    const uint64_t room = base >= cap ? 0 : cap - base;
    s_base[s] = base;
    s_spill[s] = 0;
    if (room < cnt) {
      s_spill[s] = atomicAdd(&fill[S * kCtrStride], cnt - uint32_t(room));
      *spilled = 1;
    }
  }
}

// Records in region r of a split (S slice regions of cap, then the spill).
__device__ __forceinline__ uint32_t region_len(const uint32_t* fill, uint32_t r,
                                               uint32_t S, uint64_t cap) {
  const uint32_t f = __ldcg(fill + r * kCtrStride);
  return r < S && f > cap ? uint32_t(cap) : f;
}

// ---------------------------------------------------------------------------
// scatter (a multi-split): each block tile of kBlock*U keys is binned by
// slice in shared memory (a rank per key), sorted by slice inside shared
// memory, and written out as one contiguous run per occupied slice (one
// claim on fill1 per run), so consecutive threads store consecutive
// records.  dst[] is written in key order.
// Shared memory: 4*S counters + 8*kBlock*U bytes.
// ---------------------------------------------------------------------------
template <class G, int U>
__global__ void __launch_bounds__(kBlock, CF_SPLIT_MINB)
k_slice_scatter(DevFilter d, const uint64_t* __restrict__ keys, uint64_t n,
                SliceBufs sb, uint32_t* __restrict__ dst) {
  extern __shared__ uint64_t sm64[];
  constexpr uint32_t T = kBlock * U;
  const uint32_t S = sb.n_slices, shift = sb.shift;
  uint64_t* stash = sm64;                                   // [T]
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(sm64 + T);  // [S]
  uint32_t* s_off = s_cnt + S;                              // [S]
  uint32_t* s_base = s_off + S;                             // [S]
  uint32_t* s_spill = s_base + S;                           // [S]
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_spilled;
  const uint32_t cap = uint32_t(sb.cap1);
  for (uint64_t t0 = blockIdx.x * uint64_t(T); t0 < n; t0 += uint64_t(gridDim.x) * T) {
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) s_cnt[s] = 0;
    if (threadIdx.x == 0) s_spilled = 0;
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
    claim_runs(s_cnt, s_base, s_spill, S, sb.fill1, sb.cap1, &s_spilled);
    __syncthreads();
    const bool spilled = s_spilled != 0;
    auto pos = [&](uint32_t sl, uint32_t rk) -> uint32_t {
      return spilled ? uint32_t(region_pos(sl, rk, s_base[sl], s_cnt[sl], s_spill[sl],
                                           sb.cap1, S))
                     : sl * cap + s_base[sl] + rk;
    };
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = t0 + uint64_t(u) * blockDim.x + threadIdx.x;
      if (i < n) {
        const uint32_t sl = slrk[u] >> 16, rk = slrk[u] & 0xFFFFu;
        stash[s_off[sl] + rk] = h[u];
        if (dst) st_cs_u32(dst + i, pos(sl, rk));
      }
    }
    __syncthreads();
    const uint32_t cnt = uint32_t(n - t0 < T ? n - t0 : T);
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
      const uint64_t hv = stash[j];
      const uint32_t sl = slice_of_h<G>(d, hv, shift);
      sb.rec1[pos(sl, j - s_off[sl])] = hv;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// probe1: the operation on bucket i1 for rec1 records, regions in order.  A
// block tile is up to kSliceBlock*8 records of one region (thread t takes
// records t, t + kSliceBlock, ...), staged in shared memory by a TMA bulk copy
// issued while the block works on the previous tile.  Records left pending
// are stashed in shared memory, sorted by the slice of i2 once per tile,
// and written to rec2 as one run per occupied slice (one claim on fill2 per
// run).
// Shared memory: 20*T bytes + 4*S counters + 4*(S + 2) tile starts +
// 4*(S + 1) region lengths (T = kSliceBlock*8 records).
// ---------------------------------------------------------------------------

template <class G, int OP, int K, bool RT = false>
__global__ void __launch_bounds__(kSliceBlock, CF_SLICE_MINB)
k_slice_probe1(DevFilter d, SliceBufs sb, int want_flags) {
  // R rounds of K records per thread: every tile holds 8 records per thread
  // whatever the bucket size (K = 8 / 4 / 2 / 1 for 8 / 16 / 32 / 64-byte
  // buckets), so the per-tile work (barriers, prefix, claims) stays amortised.
  constexpr int R = 8 / K;
  constexpr int N = R * K;
  constexpr uint32_t T = kSliceBlock * N;
  static_assert(K == 8 || K == 4 || K == 2 || K == 1, "records per thread");
  static_assert(T <= 2048, "shared entries pack an 11-bit tile index");
  extern __shared__ uint64_t sm64[];
  const uint32_t S = sb.n_slices;
  const uint32_t NR = S + 1;  // rec1 regions: S slices, then the spill
  uint64_t* pref = sm64;                                            // [T] next tile's records
  uint64_t* stash_h = sm64 + T;                                     // [T] by tile index
  uint32_t* s_order = reinterpret_cast<uint32_t*>(sm64 + 2 * T);   // [T] index | slice << 11
  uint32_t* s_cnt = s_order + T;                                    // [S + 1]
  uint32_t* s_off = s_cnt + NR;                                     // [S]
  uint32_t* s_base = s_off + S;                                     // [S]
  uint32_t* s_spill = s_base + S;                                   // [S]
  uint32_t* s_tstart = s_spill + S;                                 // [S + 2]
  uint32_t* s_len = s_tstart + NR + 1;                              // [S + 1]
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_next_p, s_next_cnt, s_spilled;
  __shared__ __align__(8) uint64_t s_bar;
  TileCounts c;
  // Records and first tile of every region (tiles never straddle two
  // regions), and the number of tiles after the last one.
  for (uint32_t r = threadIdx.x; r < NR; r += blockDim.x) {
    s_len[r] = region_len(sb.fill1, r, S, sb.cap1);
    s_cnt[r] = (s_len[r] + T - 1) / T;
  }
  __syncthreads();
  block_scan_excl(s_cnt, s_tstart, NR, tmp);
  if (threadIdx.x == 0) s_tstart[NR] = s_tstart[NR - 1] + s_cnt[NR - 1];
  // Tiles are handed out in order by a counter, so the blocks at work stay
  // within a window of consecutive tiles (one or two slices) instead of
  // drifting apart as a static grid stride lets them.  One thread copies the
  // next tile's records into shared memory (TMA bulk copy) while the block
  // works on the current one; a tile of cnt records copies cnt & ~1 of
  // them (16-byte multiples; region starts are multiples of 256 records)
  // and the block loads an odd last one itself.
  uint32_t* tile_ctr = sb.fill2 + (S + 2) * kCtrStride;
  uint32_t reg = 0;  // thread 0: region of the block's latest tile (its tiles only grow)
  auto fetch = [&]() {  // thread 0
    const uint32_t t = atomicAdd(tile_ctr, 1u);
    if (t >= s_tstart[NR]) {
      s_next_cnt = 0;
      return;
    }
    while (s_tstart[reg + 1] <= t) ++reg;  // stops at a nonempty region: t < tiles
    const uint32_t k0 = (t - s_tstart[reg]) * T;
    const uint32_t len = s_len[reg];
    const uint32_t cnt = len - k0 < T ? len - k0 : T;
    const uint32_t p = reg * uint32_t(sb.cap1) + k0;
    s_next_p = p;
    s_next_cnt = cnt;
    bulk_load(&s_bar, pref, sb.rec1 + p, (cnt & ~1u) * 8u);
  };
  __syncthreads();  // tile starts in place
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fetch();
  }
  __syncthreads();
  uint32_t t0 = s_next_p, tcnt = s_next_cnt;
  uint32_t parity = 0;
  while (tcnt) {
    const bool copy_ok = mbar_wait(&s_bar, parity);
    parity ^= 1u;
    // Record i of this thread: tile index loc(i) = i*kSliceBlock + thread (lane-
    // strided: conflict-free reads of the staged tile, coalesced stores),
    // at rec1 position t0 + loc.
    const uint32_t copied = tcnt & ~1u;  // records now in pref
    uint64_t hr[N];
    bool vr[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t loc = uint32_t(i) * kSliceBlock + threadIdx.x;
      vr[i] = loc < tcnt;
      hr[i] = loc < copied ? pref[loc] : (vr[i] ? ld_stream_u64(sb.rec1 + t0 + loc) : 0ull);
    }
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) s_cnt[s] = 0;
    if (threadIdx.x == 32) s_spilled = 0;
    // pref consumed, counters zeroed; the block leaves together if any of
    // its threads gave up on the copy.
    if (!__syncthreads_and(copy_ok)) {
      // The copy did not complete: report it and leave this tile (its
      // records stay unprocessed; the error bit tells the caller).
      if (threadIdx.x == 0) atomicOr(&d.ctrl->error_word, kErrAsyncCopy);
      mbar_wait(&s_bar, parity ^ 1u);  // once more (bounded) for the copy in flight
      break;
    }
    if (threadIdx.x == 0) fetch();
    uint32_t slrk[N];  // slice << 16 | rank of a pending record, else kSettled | flag
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
        cas_many<G, K, OP == SOP_INSERT, RT>(d, bkt, tag, valid, res, c.cas);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = r * K + k;
        const uint32_t loc = uint32_t(i) * kSliceBlock + threadIdx.x;
        slrk[i] = kSettled;  // settled with flag 0 (or not a record)
        if (valid[k] && res[k] == TI_FULL) {
          const uint32_t sl = alt_index<G>(d, bkt[k], tag[k]) >> sb.shift;
          slrk[i] = (sl << 16) | atomicAdd(&s_cnt[sl], 1u);
          stash_h[loc] = hr[i];
        } else if (valid[k]) {
          if (res[k] == TI_OK) {
            slrk[i] = kSettled | 1u;
            c.ok++;
          } else {
            slrk[i] = kSettled | 2u;
            c.cont++;
            if (OP == SOP_INSERT) log_victim(d, tag[k], bkt[k]);
          }
        }
      }
    }
    __syncthreads();
    block_scan_excl(s_cnt, s_off, S, tmp);
    claim_runs(s_cnt, s_base, s_spill, S, sb.fill2, sb.cap2, &s_spilled);
    const uint32_t np = s_off[S - 1] + s_cnt[S - 1];
    __syncthreads();
    const bool spilled = s_spilled != 0;
    const uint32_t cap2 = uint32_t(sb.cap2);
    auto pos = [&](uint32_t sl, uint32_t rk) -> uint32_t {
      return spilled ? uint32_t(region_pos(sl, rk, s_base[sl], s_cnt[sl], s_spill[sl],
                                           sb.cap2, S))
                     : sl * cap2 + s_base[sl] + rk;
    };
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t loc = uint32_t(i) * kSliceBlock + threadIdx.x;
      uint32_t lk = slrk[i];
      if (lk < kSettled) {
        const uint32_t sl = lk >> 16, rk = lk & 0xFFFFu;
        s_order[s_off[sl] + rk] = loc | (sl << 11);
        lk = pos(sl, rk);
      }
      if (want_flags && vr[i]) sb.link[t0 + loc] = lk;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < np; j += blockDim.x) {
      const uint32_t e = s_order[j];
      const uint32_t sl = e >> 11;
      sb.rec2[pos(sl, j - s_off[sl])] = stash_h[e & 0x7FFu];
    }
    __syncthreads();
    t0 = s_next_p;
    tcnt = s_next_cnt;
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
  if constexpr (OP != SOP_CONTAINS) cas_count_block_add(d, c.cas);
  if (c.cont) atomicOr(&d.ctrl->error_word, 1u);
}

// ---------------------------------------------------------------------------
// probe2: the operation on bucket i2 for the rec2 records, slice regions in
// order, then the spill region.  The filled parts of the regions are
// numbered consecutively (a prefix of their fills in shared memory), and
// block tiles of kSliceBlock*8 of those numbers are handed out in order by a
// counter, so that only records are visited.
// ---------------------------------------------------------------------------
template <class G, int OP, int K, bool RT = false>
__global__ void __launch_bounds__(kSliceBlock, CF_SLICE2_MINB)
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
        cas_many<G, K, OP == SOP_INSERT, RT>(d, bkt, tag, valid, res, c.cas);
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
  if constexpr (OP != SOP_CONTAINS) cas_count_block_add(d, c.cas);
  if (c.cont) atomicOr(&d.ctrl->error_word, 1u);
}

// ---------------------------------------------------------------------------
// merge: f1[p] = the flag of rec1 record p: link[p] when probe1 settled it,
// else f2 at the rec2 position link[p] holds.  Records are walked in rec1
// order, the order in which probe1 wrote rec2, so the f2 gathers stay
// within a window that L2 holds.  A thread takes V groups of four rec1
// positions per iteration (V grid strides apart), so that up to 4*V of its
// gathers are in flight together.
// ---------------------------------------------------------------------------
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
k_slice_merge(SliceBufs sb) {
  constexpr int V = CF_MERGE_V;
  // Groups of four rec1 positions (cap1 is a multiple of four, so a group
  // never straddles two regions): the records of every region, its number
  // of groups and its first group in the order the threads walk them.
  extern __shared__ uint32_t s_reg[];
  __shared__ uint32_t tmp[32];
  const uint32_t S = sb.n_slices, NR = S + 1;
  uint32_t* s_len = s_reg;            // [S + 1]
  uint32_t* s_gcnt = s_len + NR;      // [S + 1]
  uint32_t* s_gstart = s_gcnt + NR;   // [S + 2]
  for (uint32_t r = threadIdx.x; r < NR; r += blockDim.x) {
    s_len[r] = region_len(sb.fill1, r, S, sb.cap1);
    s_gcnt[r] = (s_len[r] + 3) / 4;
  }
  __syncthreads();
  block_scan_excl(s_gcnt, s_gstart, NR, tmp);
  if (threadIdx.x == 0) s_gstart[NR] = s_gstart[NR - 1] + s_gcnt[NR - 1];
  __syncthreads();
  const uint32_t total = s_gstart[NR];
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t* f1w = reinterpret_cast<uint32_t*>(sb.f1);
  const uint4* link4 = reinterpret_cast<const uint4*>(sb.link);
  const uint32_t cap = uint32_t(sb.cap1);
  uint32_t r = 0;  // region of the thread's latest group (its groups only grow)
  for (uint32_t g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < total; g0 += stride * V) {
    uint32_t q[V], vc[V];
    uint4 l[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const uint32_t g = g0 + u * stride;
      vc[u] = 0;
      if (g < total) {
        while (s_gstart[r + 1] <= g) ++r;
        const uint32_t off = (g - s_gstart[r]) * 4;
        vc[u] = s_len[r] - off;  // records in the group: 1, 2, 3 or >= 4
        q[u] = (r * cap + off) / 4;
        l[u] = __ldcs(link4 + q[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      if (!vc[u]) continue;
      const uint32_t ls[4] = {l[u].x, l[u].y, l[u].z, l[u].w};
      uint32_t w = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // (A position past rec2 can only come from a tile that probe1 left
        // unprocessed after a copy timeout, which sets the error word.)
        const uint32_t b = uint32_t(j) >= vc[u]       ? 0u
                           : ls[j] >= kSettled        ? (ls[j] & 0xFFu)
                           : ls[j] < sb.rec2_len      ? uint32_t(sb.f2[ls[j]])
                                                      : 0u;
        w |= b << (8 * j);
      }
      f1w[q[u]] = w;
    }
  }
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

}  // namespace cfk
