// Slice-grouped eviction levels: phase 2 of Alg. 1 (the BFS eviction of
// Sec. 4.6.1) for the keys of a slice-partitioned insert pass whose two
// buckets were full, run level by level instead of chain by chain.
//
// The eviction loop (k_insert_evict) walks every chain on its own: each
// round touches a bucket in an unrelated part of the table, so for a table
// far larger than L2 every round is a DRAM round trip, and the loop runs at
// the rate of random sector accesses.  Here the chains advance one step per
// level, and a level's steps are grouped by the table slice of the bucket
// they touch, the way the bucket passes group the keys: all warps work in
// one or two slices at a time, so each slice's buckets come from DRAM about
// once per level and every further access hits L2.
//
// A chain between two levels is a record: the tag in hand, the bucket it is
// destined for, the key's random stream, the overwrites so far, the key's
// position (for its flag) and whether the bucket's map bit may be clear.
// One step of a chain at bucket j (words loaded):
//   place  the tag into j if j has an empty slot (Alg. 1's TryInsert): the
//          chain ends;
//   give up if the chain has used max_evictions overwrites (the tag in
//          hand is the victim);
//   swap   the BFS choice among b/2 consecutive slots from a random start,
//          asked of the full-bucket map (bfs_swap_map), and the swap of the
//          tag into the chosen slot; the evicted tag goes on to its
//          alternate bucket, which the next level's step places it in.
// This is the order of the loop's rounds (a round swaps, then tries the
// evicted tag's bucket), cut between the swap and the place: every chain
// takes the same steps and random draws as in the loop, only the
// interleaving of chains differs, which the concurrent loop leaves open
// anyway.
//
// Launches of one eviction (after the bucket passes and the map):
//   seed     the queued keys' chain heads (the first random draw picks i1
//            or i2), grouped by that bucket's slice: level 0's records
//   level k  (k = 0 .. L-1) one step of each record of level k, records
//            grouped by slice in order (block tiles handed out by a
//            counter); the chains that go on are grouped again by the
//            slice of their next bucket: level k + 1's records
//   resume   the records left when a level had fewer than stop_q records
//            (or after L levels) run to their end in the eviction loop's
//            manner (one step per lane and iteration, lanes refilled)
// The seed decides on the device whether the levels run (enough keys
// queued, a map built, room for the records); otherwise every level and
// the resume return at once and k_insert_evict takes the queue as before.
// A record that finds no room in the next level's buffer (its slice region
// and the spill region full, which only skewed batches reach) is run to its
// end at once by the thread that holds it.
#pragma once

#include "cf_slice.cuh"

namespace cfk {

// Records per thread of a level tile and resident blocks per SM of the
// level kernels, for buckets of up to 8 bytes (CF_LEVEL_N, CF_LEVEL_MINB)
// and for wider ones (one record per thread, CF_LEVEL_MINB_WIDE).  Large
// workload, eviction ms per step (records per thread x blocks per SM):
// 4 x 3: 35.5, 8 x 2: 41.4, 2 x 4: 32.6, 2 x 5: 30.9, 2 x 6: 31.1, 2 x 8
// (spilling): 34.6, 1 x 6: 32.6.  The steps are bound by random sector
// reads: more warps with fewer records each keep more of them in flight.
// Wider buckets spill above 3 blocks per SM.
#ifndef CF_LEVEL_N
#define CF_LEVEL_N 2
#endif
#ifndef CF_LEVEL_MINB
#define CF_LEVEL_MINB 5
#endif
#ifndef CF_LEVEL_MINB_WIDE
#define CF_LEVEL_MINB_WIDE 3
#endif
// Resident blocks per SM of the seed (four records per thread).
#ifndef CF_SEED_MINB
#define CF_SEED_MINB 3
#endif

// A chain record: 3 words (rng; cur | tag << 32; idx | (ev | mark << 31) << 32).
struct LvRec {
  uint64_t rng;
  uint32_t cur, tag, idx, evm;
};
__device__ __forceinline__ LvRec lv_load(const uint64_t* buf, uint64_t p) {
  const uint64_t* q = buf + 3 * p;
  const uint64_t w0 = __ldcs(q), w1 = __ldcs(q + 1), w2 = __ldcs(q + 2);
  return LvRec{w0, uint32_t(w1), uint32_t(w1 >> 32), uint32_t(w2), uint32_t(w2 >> 32)};
}
__device__ __forceinline__ void lv_store(uint64_t* buf, uint64_t p, const LvRec& r) {
  uint64_t* q = buf + 3 * p;
  __stcs(q, r.rng);
  __stcs(q + 1, uint64_t(r.cur) | (uint64_t(r.tag) << 32));
  __stcs(q + 2, uint64_t(r.idx) | (uint64_t(r.evm) << 32));
}
constexpr uint32_t kLvMark = 0x80000000u;

// Counters of level k (k = 0..L): S slice fills, the spill fill, the tile
// counter, one per 128-byte line.
__device__ __forceinline__ uint32_t* lv_fill(const LevelBufs& lb, uint32_t S, uint32_t k) {
  return lb.fill + size_t(k) * (S + 2) * kCtrStride;
}
// Records of region r (S slices, then the spill) of a level's buffer.
__device__ __forceinline__ uint32_t lv_region_len(const uint32_t* fill, uint32_t r, uint32_t S,
                                                  const LevelBufs& lb) {
  const uint32_t f = __ldcg(fill + r * kCtrStride);
  const uint64_t c = r < S ? lb.cap : lb.spill;
  return f > c ? uint32_t(c) : f;
}
// Position of the rk-th record of slice s in a tile's run (claims as in
// claim_runs): the slice's region, then the spill region; ~0 when both
// are full.
constexpr uint64_t kLvNoRoom = ~0ull;
__device__ __forceinline__ uint64_t lv_pos(uint32_t s, uint32_t rk, uint32_t base,
                                           uint32_t cnt, uint32_t spill_base,
                                           const LevelBufs& lb, uint32_t S) {
  const uint64_t room = base >= lb.cap ? 0 : lb.cap - base;
  const uint32_t in = room < cnt ? uint32_t(room) : cnt;
  if (rk < in) return uint64_t(s) * lb.cap + base + rk;
  const uint64_t sp = uint64_t(spill_base) + (rk - in);
  return sp < lb.spill ? uint64_t(S) * lb.cap + sp : kLvNoRoom;
}

// Does level k (k = 0..L-1) run: the seed switched the levels on, and
// level k >= 1 has at least stop_q records (a level that did not run
// leaves the next one none).
__device__ __forceinline__ bool lv_runs(const LevelBufs& lb, uint32_t k) {
  if (!__ldcg(lb.ctl)) return false;
  return k == 0 || __ldcg(lb.ctl + 1 + k) >= lb.stop_q;
}

// The place part of a step: EV_OK or EV_CONTENTION (vt/vb the victim) if
// the chain ended, else ROUND_CONTINUE with c.cur full (and its map bit set
// when mark).
template <class G>
__device__ __forceinline__ int lv_place(const DevFilter& d, uint32_t* map, Chain<G>& c,
                                        bool mark, uint32_t& vt, uint64_t& vb,
                                        EvictCounters& ec) {
  if (has_empty<G>(c.bk)) {
    const int r = try_insert_loaded<G>(d, c.cur, c.tag, c.bk, ec.cas);
    if (r == TI_OK) {
      if (!has_empty<G>(c.bk)) map_set(d, map, c.cur);
      return EV_OK;
    }
    if (r == TI_CONTENTION) {
      ec.contention++;
      vt = c.tag;
      vb = c.cur;
      return EV_CONTENTION;
    }
  }
  if (mark) map_set(d, map, c.cur);
  return ROUND_CONTINUE;
}

// One step of a chain at bucket c.cur (words c.bk), see the file comment.
// mark: c.cur's map bit may be clear.  Returns EV_OK, EV_FAIL or
// EV_CONTENTION (vt/vb the victim), or ROUND_CONTINUE with c at the
// evicted tag's bucket and mark_out for that bucket.
template <class G>
__device__ __forceinline__ int lv_step(const DevFilter& d, uint32_t* map, Chain<G>& c,
                                       bool mark, uint32_t& vt, uint64_t& vb,
                                       EvictCounters& ec, bool& mark_out) {
  const int p = lv_place<G>(d, map, c, mark, vt, vb, ec);
  if (p != ROUND_CONTINUE) return p;
  if (c.ev >= d.max_ev) {
    vt = c.tag;
    vb = c.cur;
    return EV_FAIL;
  }
  const uint32_t start = uint32_t(rng_next(c.rng) & (G::B - 1));
  Bucket<G> nb{};
  bool have_nb = false;
  return bfs_swap_map<G, false>(d, c, start, map, vt, vb, ec, mark_out, nb, have_nb);
}

// Per-thread tallies of the chains that ended.
struct LvCounts {
  uint32_t ok = 0, fail = 0, ev = 0;
  EvictCounters ec;
};
__device__ __forceinline__ void lv_end(const DevFilter& d, uint8_t* f2, uint32_t idx, int r,
                                       uint32_t ev, uint32_t vt, uint64_t vb, LvCounts& n) {
  if (r != EV_OK) log_victim(d, vt, vb);
  if (f2) st_flag(f2 + idx, uint8_t(r));
  n.ev += ev;
  if (r == EV_OK) n.ok++; else n.fail++;
}
// A chain run to its end by the calling thread (a record with no room in
// the next level's buffer).
template <class G>
__device__ void lv_run_out(const DevFilter& d, uint32_t* map, uint8_t* f2, const LvRec& rec,
                           LvCounts& n) {
  Chain<G> c{};
  c.rng = rec.rng;
  c.cur = rec.cur;
  c.tag = rec.tag;
  c.ev = rec.evm & ~kLvMark;
  bool mark = (rec.evm & kLvMark) != 0;
  uint32_t vt = 0;
  uint64_t vb = 0;
  int r;
  for (;;) {
    c.bk = load_bucket_ev<G>(bucket_ptr<G>(d, c.cur));
    bool mo = false;
    r = lv_step<G>(d, map, c, mark, vt, vb, n.ec, mo);
    if (r != ROUND_CONTINUE) break;
    mark = mo;
  }
  lv_end(d, f2, rec.idx, r, c.ev, vt, vb, n);
}
__device__ __forceinline__ void lv_counts_flush(const DevFilter& d, const LvCounts& n) {
  block_add(&d.ctrl->occupancy, n.ok);
  block_add(&d.ctrl->insert_ok, n.ok);
  block_add(&d.ctrl->insert_fail, n.fail);
  block_add(&d.ctrl->evictions, n.ev);
  block_add(&d.ctrl->contention, n.ec.contention);
  cas_count_block_add(d, n.ec.cas);
  if (n.ec.contention) atomicOr(&d.ctrl->error_word, 1u);
}

// Shared-memory layout of a tile's multi-split of records (T records).
struct LvSplit {
  uint64_t* stash;    // [3T] records by tile index
  uint32_t* order;    // [T]  tile index | slice << 11, in slice order
  uint32_t* cnt;      // [S]
  uint32_t* off;      // [S]
  uint32_t* base;     // [S]
  uint32_t* spill;    // [S]
};
template <int T>
__device__ __forceinline__ LvSplit lv_split_smem(uint64_t* sm, uint32_t S) {
  LvSplit p;
  p.stash = sm;
  p.order = reinterpret_cast<uint32_t*>(sm + 3 * T);
  p.cnt = p.order + T;
  p.off = p.cnt + S;
  p.base = p.off + S;
  p.spill = p.base + S;
  return p;
}
template <int T>
constexpr size_t lv_split_bytes(uint32_t S) {
  return size_t(28) * T + size_t(16) * S;
}
__device__ __forceinline__ void lv_stash(const LvSplit& sp, uint32_t loc, const LvRec& r) {
  sp.stash[3 * loc] = r.rng;
  sp.stash[3 * loc + 1] = uint64_t(r.cur) | (uint64_t(r.tag) << 32);
  sp.stash[3 * loc + 2] = uint64_t(r.idx) | (uint64_t(r.evm) << 32);
}
__device__ __forceinline__ LvRec lv_unstash(const LvSplit& sp, uint32_t loc) {
  const uint64_t w1 = sp.stash[3 * loc + 1], w2 = sp.stash[3 * loc + 2];
  return LvRec{sp.stash[3 * loc], uint32_t(w1), uint32_t(w1 >> 32), uint32_t(w2),
               uint32_t(w2 >> 32)};
}

// The second half of a tile's multi-split: every thread has recorded its
// pending records' slice << 16 | rank in slrk (kSettled when none) and
// stashed them; all threads call this.  The runs are claimed on fill, the
// records written to out (or run to their end when there is no room), and
// the number written added to *total.
template <class G, int N>
__device__ void lv_split_out(const DevFilter& d, uint32_t* map, uint8_t* f2, const LvSplit& sp,
                             const uint32_t (&slrk)[N], uint32_t S, uint32_t* fill,
                             const LevelBufs& lb, uint64_t* out, uint32_t* total,
                             LvCounts& n, uint32_t* tmp) {
  __shared__ uint32_t s_spilled, s_lost;
  if (threadIdx.x == 0) s_lost = 0;
  __syncthreads();
  block_scan_excl(sp.cnt, sp.off, S, tmp);
  claim_runs(sp.cnt, sp.base, sp.spill, S, fill, lb.cap, &s_spilled);
  const uint32_t np = sp.off[S - 1] + sp.cnt[S - 1];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const uint32_t lk = slrk[i];
    if (lk < kSettled) {
      const uint32_t sl = lk >> 16, rk = lk & 0xFFFFu;
      const uint32_t loc = uint32_t(i) * kBlock + threadIdx.x;
      sp.order[sp.off[sl] + rk] = loc | (sl << 11);
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < np; j += blockDim.x) {
    const uint32_t e = sp.order[j];
    const uint32_t sl = e >> 11;
    const LvRec r = lv_unstash(sp, e & 0x7FFu);
    // Claims that never reached the spill region keep their run whole.
    const uint64_t p = lv_pos(sl, j - sp.off[sl], sp.base[sl], sp.cnt[sl], sp.spill[sl], lb, S);
    if (p != kLvNoRoom) {
      lv_store(out, p, r);
    } else {
      atomicAdd(&s_lost, 1u);
      lv_run_out<G>(d, map, f2, r, n);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (np > s_lost) atomicAdd(total, np - s_lost);
    if (s_lost) atomicAdd(&d.ctrl->level_runout, (unsigned long long)s_lost);
  }
}

// ---------------------------------------------------------------------------
// seed: level 0's records from the eviction queue (rec2 positions of keys
// whose two buckets were full), grouped by the slice of the chain's first
// bucket.  Decides whether the levels run: BFS with the map built for this
// launch (at least map_q keys queued), at least min_q keys, and no more
// than the buffer's slice regions hold.
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(kBlock, CF_SEED_MINB)
k_evict_seed(DevFilter d, const uint64_t* __restrict__ rec2, const uint32_t* __restrict__ queue,
             uint32_t* map, uint32_t map_q, LevelBufs lb, uint32_t S, uint32_t shift,
             uint8_t* f2) {
  constexpr int N = 4;
  constexpr uint32_t T = kBlock * N;
  extern __shared__ uint64_t sm64[];
  __shared__ uint32_t tmp[32];
  const uint32_t qn = *reinterpret_cast<volatile unsigned int*>(&d.ctrl->queue_count);
  const bool on = map != nullptr && d.eviction == 0 && d.max_ev > 0 && qn >= map_q &&
                  qn >= lb.min_q && qn <= uint64_t(S) * lb.cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) lb.ctl[0] = on ? 1u : 0u;
  if (!on) return;
  const LvSplit sp = lv_split_smem<T>(sm64, S);
  LvCounts n;
  uint32_t* fill = lv_fill(lb, S, 0);
  for (uint64_t t0 = blockIdx.x * uint64_t(T); t0 < qn; t0 += uint64_t(gridDim.x) * T) {
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) sp.cnt[s] = 0;
    __syncthreads();
    uint32_t slrk[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint64_t e = t0 + uint64_t(i) * kBlock + threadIdx.x;
      slrk[i] = kSettled;
      if (e < qn) {
        const uint32_t pos = queue[e];
        const ChainHead<G> ch = chain_head<G>(d, rec2[pos]);
        const uint32_t cur = uint32_t(ch.cur), sl = cur >> shift;
        lv_stash(sp, uint32_t(i) * kBlock + threadIdx.x, LvRec{ch.rng, cur, ch.tag, pos, 0u});
        slrk[i] = (sl << 16) | atomicAdd(&sp.cnt[sl], 1u);
      }
    }
    __syncthreads();
    lv_split_out<G, N>(d, map, f2, sp, slrk, S, fill, lb, lb.rec[0], lb.ctl + 1, n, tmp);
  }
  lv_counts_flush(d, n);
}

// ---------------------------------------------------------------------------
// level k: one step of every record of level k.  Block tiles of T records
// of one region, handed out in order by a counter (see k_slice_probe1);
// each thread loads its N records and their buckets, then steps them one
// by one; the records that go on are multi-split into level k + 1's
// buffer.
// ---------------------------------------------------------------------------
template <class G>
struct LvTile {
  static constexpr int N = G::kBucketBytes <= 8 ? CF_LEVEL_N : 1;
  static constexpr int kMinB = G::kBucketBytes <= 8 ? CF_LEVEL_MINB : CF_LEVEL_MINB_WIDE;
  static constexpr uint32_t T = kBlock * N;
};

template <class G>
__global__ void __launch_bounds__(kBlock, LvTile<G>::kMinB)
k_evict_level(DevFilter d, uint32_t* map, LevelBufs lb, uint32_t S, uint32_t shift,
              uint32_t k, uint8_t* f2) {
  constexpr int N = LvTile<G>::N;
  constexpr uint32_t T = LvTile<G>::T;
  static_assert(T <= 2048, "tile index fits 11 bits");
  if (!lv_runs(lb, k)) return;
  extern __shared__ uint64_t sm64[];
  __shared__ uint32_t tmp[32];
  __shared__ uint32_t s_p0, s_cnt;
  const LvSplit sp = lv_split_smem<T>(sm64, S);
  const uint32_t NR = S + 1;
  // Region lengths and first tiles, after the split's arrays.
  uint32_t* s_len = sp.spill + S;       // [S + 1]
  uint32_t* s_tiles = s_len + NR;       // [S + 1]
  uint32_t* s_tstart = s_tiles + NR;    // [S + 2]
  const uint32_t* fin = lv_fill(lb, S, k);
  uint32_t* fout = lv_fill(lb, S, k + 1);
  const uint64_t* in = lb.rec[k & 1];
  uint64_t* out = lb.rec[(k + 1) & 1];
  for (uint32_t r = threadIdx.x; r < NR; r += blockDim.x) {
    s_len[r] = lv_region_len(fin, r, S, lb);
    s_tiles[r] = (s_len[r] + T - 1) / T;
  }
  __syncthreads();
  block_scan_excl(s_tiles, s_tstart, NR, tmp);
  if (threadIdx.x == 0) {
    s_tstart[NR] = s_tstart[NR - 1] + s_tiles[NR - 1];
    if (blockIdx.x == 0) {
      atomicAdd(&d.ctrl->level_passes, 1ull);
      atomicAdd(&d.ctrl->level_steps, (unsigned long long)__ldcg(lb.ctl + 1 + k));
    }
  }
  uint32_t* tile_ctr = const_cast<uint32_t*>(fin) + (S + 1) * kCtrStride;
  uint32_t reg = 0;  // thread 0: region of the block's latest tile
  LvCounts n;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t t = atomicAdd(tile_ctr, 1u);
      s_cnt = 0;
      if (t < s_tstart[NR]) {
        while (s_tstart[reg + 1] <= t) ++reg;
        const uint32_t k0 = (t - s_tstart[reg]) * T;
        const uint32_t len = s_len[reg];
        s_cnt = len - k0 < T ? len - k0 : T;
        s_p0 = uint32_t(reg * lb.cap + k0);
      }
    }
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) sp.cnt[s] = 0;
    __syncthreads();
    const uint32_t tcnt = s_cnt;
    if (!tcnt) break;
    const uint64_t p0 = s_p0;
    LvRec rec[N];
    Bucket<G> bk[N];
    bool valid[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint32_t loc = uint32_t(i) * kBlock + threadIdx.x;
      valid[i] = loc < tcnt;
      rec[i] = valid[i] ? lv_load(in, p0 + loc) : LvRec{};
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (valid[i]) bk[i] = load_bucket<G, false>(bucket_ptr<G>(d, rec[i].cur));
    // The records' steps one after the other: their bucket loads above are
    // in flight together, and overlapping their map loads and CASes as well
    // measured slower (the steps are bound by random DRAM sector reads, and
    // more records in flight only cost registers and collisions).
    uint32_t slrk[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      slrk[i] = kSettled;
      if (!valid[i]) continue;
      Chain<G> c;
      c.rng = rec[i].rng;
      c.cur = rec[i].cur;
      c.tag = rec[i].tag;
      c.ev = rec[i].evm & ~kLvMark;
      c.bk = bk[i];
      uint32_t vt = 0;
      uint64_t vb = 0;
      bool mo = false;
      const int r = lv_step<G>(d, map, c, (rec[i].evm & kLvMark) != 0, vt, vb, n.ec, mo);
      if (r == ROUND_CONTINUE) {
        const uint32_t cur = uint32_t(c.cur), sl = cur >> shift;
        lv_stash(sp, uint32_t(i) * kBlock + threadIdx.x,
                 LvRec{c.rng, cur, c.tag, rec[i].idx, c.ev | (mo ? kLvMark : 0u)});
        slrk[i] = (sl << 16) | atomicAdd(&sp.cnt[sl], 1u);
      } else {
        lv_end(d, f2, rec[i].idx, r, c.ev, vt, vb, n);
      }
    }
    __syncthreads();
    lv_split_out<G, N>(d, map, f2, sp, slrk, S, fout, lb, out, lb.ctl + 2 + k, n, tmp);
  }
  lv_counts_flush(d, n);
}

// ---------------------------------------------------------------------------
// resume: the records of the first level that did not run (or of level L)
// run to their end in the eviction loop's manner: after its place step, a
// chain takes the loop's rounds (evict_round_map: a round swaps and then
// tries the evicted tag's bucket, loaded while the swap's CAS runs), one
// round per lane and iteration; a lane whose chain ended takes the next
// record of its warp's share, which it has prepared meanwhile (stage 1:
// the record's words loading, 2: its bucket's words loading).
// ---------------------------------------------------------------------------
template <class G>
__global__ void __launch_bounds__(kBlock, CF_MINB_EVICT)
k_evict_resume(DevFilter d, uint32_t* map, LevelBufs lb, uint32_t S, uint8_t* f2) {
  if (!__ldcg(lb.ctl)) return;
  uint32_t ks = 1;
  while (ks < lb.n_levels && __ldcg(lb.ctl + 1 + ks) >= lb.stop_q) ++ks;
  const uint32_t total = __ldcg(lb.ctl + 1 + ks);
  const uint32_t NR = S + 1;
  extern __shared__ uint32_t s_reg[];
  __shared__ uint32_t tmp[32];
  uint32_t* s_len = s_reg;         // [S + 1]
  uint32_t* s_start = s_reg + NR;  // [S + 1]
  const uint32_t* fill = lv_fill(lb, S, ks);
  for (uint32_t r = threadIdx.x; r < NR; r += blockDim.x) s_len[r] = lv_region_len(fill, r, S, lb);
  __syncthreads();
  block_scan_excl(s_len, s_start, NR, tmp);
  const uint64_t* buf = lb.rec[ks & 1];
  // Buffer position of compacted record x.
  auto pos_of = [&](uint32_t x) {
    uint32_t lo = 0, hi = NR;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_start[mid] <= x) lo = mid; else hi = mid;
    }
    return uint64_t(lo) * lb.cap + (x - s_start[lo]);
  };
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t n_warps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  uint32_t next = uint32_t(uint64_t(total) * warp / n_warps);
  const uint32_t end = uint32_t(uint64_t(total) * (warp + 1) / n_warps);
  LvCounts n;
  Chain<G> c{};
  uint32_t idx = 0;
  bool active = false;
  uint32_t pst = 0;
  LvRec prec{};
  Bucket<G> pbk{};
  for (;;) {
    if (pst == 1) {
      pbk = load_bucket_ev<G>(bucket_ptr<G>(d, prec.cur));
      pst = 2;
    }
    if (next < end) {
      const bool want = pst == 0;
      const unsigned need = __ballot_sync(0xFFFFFFFFu, want);
      if (want) {
        const uint32_t e = next + __popc(need & ((1u << lane) - 1u));
        if (e < end) {
          prec = lv_load(buf, pos_of(e));
          pst = 1;
        }
      }
      next += __popc(need);
    }
    if (!active && pst != 0) {
      if (pst == 1) pbk = load_bucket_ev<G>(bucket_ptr<G>(d, prec.cur));
      pst = 0;
      c.rng = prec.rng;
      c.cur = prec.cur;
      c.tag = prec.tag;
      c.ev = prec.evm & ~kLvMark;
      c.bk = pbk;
      idx = prec.idx;
      uint32_t vt = 0;
      uint64_t vb = 0;
      const int r = lv_place<G>(d, map, c, (prec.evm & kLvMark) != 0, vt, vb, n.ec);
      if (r == ROUND_CONTINUE) active = true;
      else lv_end(d, f2, idx, r, c.ev, vt, vb, n);
    }
    if (!__any_sync(0xFFFFFFFFu, active)) {
      if (next >= end) break;
      continue;
    }
    if (active) {
      uint32_t vt = 0;
      uint64_t vb = 0;
      const int r = evict_round_map<G>(d, c, map, vt, vb, n.ec);
      if (r != ROUND_CONTINUE) {
        lv_end(d, f2, idx, r, c.ev, vt, vb, n);
        active = false;
      }
    }
  }
  lv_counts_flush(d, n);
}

}  // namespace cfk
