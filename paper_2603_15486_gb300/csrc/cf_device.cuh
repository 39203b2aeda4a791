// Device primitives and per-key algorithms of the cuckoo filter (sm_103a).
//
// Paper: "Cuckoo-GPU: Accelerating Cuckoo Filters on Modern GPUs" (Dortmann,
// Vieth, Schmidt, 2026).  Hashing: Sec. 2.1 Eq. 1-3 and Sec. 4.3 step 1.
// Layout: Sec. 4.2 / Fig. 2.  TryInsert: Alg. 1.  Find: Alg. 2.  TryRemove:
// Alg. 3.  BFS eviction: Sec. 4.6.1.  DFS chain: Alg. 1 phase 2.  Offset
// policy: Sec. 4.6.2.
//
// Every loop that waits on another thread's progress (CAS retry loops) has a
// fixed iteration bound; running out of it is reported as contention in the
// key's flag and in the control block, never by trapping.
#pragma once

#include <cstdint>
#include <type_traits>

#include "cf_types.h"

namespace cfk {

// Default bound of every CAS retry loop on one word (DevFilter::max_cas;
// tests lower it to make the loops run out).
constexpr uint32_t kMaxCas = 1u << 12;

// The bound of a CAS retry loop: the filter's (RT) or the default as a
// compile-time constant.  The hot multi-key CAS rounds of the direct insert,
// the delete and the bucket passes are compiled both ways and the host
// launches the RT instance only for a filter whose bound was lowered: the
// runtime bound cost those kernels about 5 ms per step of the large
// workload (113.1 vs 108.3 ms).
template <bool RT = true>
__device__ __forceinline__ uint32_t cas_bound(const DevFilter& d) {
  return RT ? d.max_cas : kMaxCas;
}

// CF_CAS_HIST=0 builds without the CAS-retry histogram (0.5 ms of the
// 106 ms step of the large workload).
#ifndef CF_CAS_HIST
#define CF_CAS_HIST 1
#endif

// ---------------------------------------------------------------------------
// Geometry: F-bit tags, B slots per bucket, bucket policy.
// ---------------------------------------------------------------------------
template <int F_, int B_, int POLICY_>
struct Geo {
  static constexpr int F = F_;
  static constexpr int B = B_;
  static constexpr int POLICY = POLICY_;
  static constexpr bool kW32 = (F * B == 32);
  using Word = std::conditional_t<kW32, unsigned int, unsigned long long>;
  static constexpr int kWordBits = kW32 ? 32 : 64;
  static constexpr int kTpw = kWordBits / F;          // tags per word
  static constexpr int kWpb = (F * B) / kWordBits;    // words per bucket
  static constexpr int kBucketBytes = F * B / 8;
  static constexpr Word kLaneMask =
      F == 32 ? Word(0xFFFFFFFFu) : Word((Word(1) << F) - 1);
  static constexpr Word ones() {
    Word w = 0;
    for (int l = 0; l < kTpw; ++l) w |= Word(1) << (l * F);
    return w;
  }
  static constexpr Word kOnes = ones();                 // 1 in every lane
  static constexpr Word kLow = kOnes * (kLaneMask >> 1);  // 0x7F.. per lane
  static constexpr uint32_t kChoice = POLICY == 1 ? (1u << (F - 1)) : 0u;
  static constexpr uint32_t kFpMask =
      POLICY == 1 ? kChoice - 1u : uint32_t(kLaneMask);
  static_assert(kWpb >= 1 && (kWpb & (kWpb - 1)) == 0, "words per bucket");
};

template <class G>
struct Bucket {
  typename G::Word w[G::kWpb];
};

// ---------------------------------------------------------------------------
// Loads.  Queries use non-coherent, L1-bypassing loads (the table is
// read-only while a query runs).  Mutating kernels use .cg loads (L2, which
// is coherent with the atomics) so that a thread never reads a stale L1 copy
// of a word it or another thread has just changed by CAS.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_nc_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned long long ld_nc_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void ld_nc_v2(const unsigned long long* p,
                                         unsigned long long& a,
                                         unsigned long long& b) {
  asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0,%1}, [%2];"
               : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ void ld_nc_v4(const unsigned long long* p,
                                         unsigned long long& a,
                                         unsigned long long& b,
                                         unsigned long long& c,
                                         unsigned long long& d) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
__device__ __forceinline__ unsigned int ld_cg_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void ld_cg_v2(const unsigned long long* p,
                                         unsigned long long& a,
                                         unsigned long long& b) {
  asm volatile("ld.global.cg.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ void ld_cg_v4(const unsigned long long* p,
                                         unsigned long long& a,
                                         unsigned long long& b,
                                         unsigned long long& c,
                                         unsigned long long& d) {
  asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
// Streaming loads of the key array (read once).
__device__ __forceinline__ unsigned long long ld_stream_u64(const uint64_t* p) {
  unsigned long long v;
  asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

template <class G, bool NC>
__device__ __forceinline__ Bucket<G> load_bucket(const typename G::Word* p) {
  Bucket<G> b;
  if constexpr (G::kW32) {
    b.w[0] = NC ? ld_nc_u32(p) : ld_cg_u32(p);
  } else if constexpr (G::kWpb == 1) {
    b.w[0] = NC ? ld_nc_u64(p) : ld_cg_u64(p);
  } else if constexpr (G::kWpb == 2) {
    if (NC) ld_nc_v2(p, b.w[0], b.w[1]); else ld_cg_v2(p, b.w[0], b.w[1]);
  } else {
#pragma unroll
    for (int q = 0; q < G::kWpb; q += 4) {
      if (NC)
        ld_nc_v4(p + q, b.w[q], b.w[q + 1], b.w[q + 2], b.w[q + 3]);
      else
        ld_cg_v4(p + q, b.w[q], b.w[q + 1], b.w[q + 2], b.w[q + 3]);
    }
  }
  return b;
}

// Bucket loads of the eviction chains: random, one use each, so with
// CF_EVICT_L2_64B the L2 fetch of a miss is limited to 64 bytes (two
// sectors) instead of the default 128 (one-word buckets only).
#ifndef CF_EVICT_L2_64B
#define CF_EVICT_L2_64B 0
#endif

template <class G>
__device__ __forceinline__ Bucket<G> load_bucket_ev(const typename G::Word* p) {
  if constexpr (CF_EVICT_L2_64B && G::kWpb == 1) {
    Bucket<G> b;
    if constexpr (G::kW32) {
      unsigned int v;
      asm volatile("ld.global.cg.L2::64B.u32 %0, [%1];" : "=r"(v) : "l"(p));
      b.w[0] = v;
    } else {
      unsigned long long v;
      asm volatile("ld.global.cg.L2::64B.u64 %0, [%1];" : "=l"(v) : "l"(p));
      b.w[0] = v;
    }
    return b;
  } else {
    return load_bucket<G, false>(p);
  }
}

template <class G>
__device__ __forceinline__ typename G::Word select_word(const Bucket<G>& b,
                                                        int wi) {
  typename G::Word w = b.w[0];
#pragma unroll
  for (int q = 1; q < G::kWpb; ++q)
    if (q == wi) w = b.w[q];
  return w;
}

template <class G>
__device__ __forceinline__ void set_word(Bucket<G>& b, int wi,
                                         typename G::Word v) {
#pragma unroll
  for (int q = 0; q < G::kWpb; ++q)
    if (q == wi) b.w[q] = v;
}

// ---------------------------------------------------------------------------
// SWAR on one word (Alg. 1-3 "ZeroMask", "HasZeroSegment", "BroadcastTag").
// zero_lanes sets the top bit of exactly the lanes that are zero: adding
// 0x7F..F to the low bits of a lane cannot carry into the next lane, so the
// mask is exact per lane (needed to pick a lane to CAS, not only to test).
// ---------------------------------------------------------------------------
template <class G>
__device__ __forceinline__ typename G::Word zero_lanes(typename G::Word x) {
  return ~(((x & G::kLow) + G::kLow) | x | G::kLow);
}
template <class G>
__device__ __forceinline__ typename G::Word broadcast(uint32_t tag) {
  return typename G::Word(tag) * G::kOnes;
}
template <class G>
__device__ __forceinline__ int first_lane(typename G::Word mask) {
  int bit;
  if constexpr (G::kW32)
    bit = __ffs(mask) - 1;
  else
    bit = __ffsll((long long)mask) - 1;
  return bit / G::F;
}
template <class G>
__device__ __forceinline__ uint32_t get_lane(typename G::Word w, int lane) {
  return uint32_t((w >> (lane * G::F)) & G::kLaneMask);
}
template <class G>
__device__ __forceinline__ typename G::Word replace_lane(typename G::Word w,
                                                         int lane,
                                                         uint32_t tag) {
  using W = typename G::Word;
  const int sh = lane * G::F;
  return (w & ~(G::kLaneMask << sh)) | (W(tag) << sh);
}
template <class G>
__device__ __forceinline__ uint32_t get_slot(const Bucket<G>& b, uint32_t s) {
  return get_lane<G>(select_word<G>(b, int(s / G::kTpw)), int(s % G::kTpw));
}
template <class G>
__device__ __forceinline__ bool has_empty(const Bucket<G>& b) {
  typename G::Word acc = 0;
#pragma unroll
  for (int q = 0; q < G::kWpb; ++q) acc |= zero_lanes<G>(b.w[q]);
  return acc != 0;
}
template <class G>
__device__ __forceinline__ bool bucket_has(const Bucket<G>& b, uint32_t tag) {
  const typename G::Word pat = broadcast<G>(tag);
  typename G::Word acc = 0;
#pragma unroll
  for (int q = 0; q < G::kWpb; ++q) acc |= zero_lanes<G>(b.w[q] ^ pat);
  return acc != 0;
}

// ---------------------------------------------------------------------------
// Hashing (Eq. 1-3, Sec. 4.3): XXH64 of the key's 8 little-endian bytes,
// seed 0, written from the public XXH64 specification.
// ---------------------------------------------------------------------------
constexpr uint64_t kP1 = 0x9E3779B185EBCA87ull;
constexpr uint64_t kP2 = 0xC2B2AE3D27D4EB4Full;
constexpr uint64_t kP3 = 0x165667B19E3779F9ull;
constexpr uint64_t kP4 = 0x85EBCA77C2B2AE63ull;
constexpr uint64_t kP5 = 0x27D4EB2F165667C5ull;

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) {
  return (x << r) | (x >> (64 - r));
}

__device__ __forceinline__ uint64_t xxh64_u64(uint64_t key) {
  uint64_t acc = kP5 + 8u;
  acc ^= rotl64(key * kP2, 31) * kP1;
  acc = rotl64(acc, 27) * kP1 + kP4;
  acc ^= acc >> 33;
  acc *= kP2;
  acc ^= acc >> 29;
  acc *= kP3;
  acc ^= acc >> 32;
  return acc;
}

// H(fp) of Eq. 3: XXH64 of the fingerprint, low 32 bits.
__device__ __forceinline__ uint32_t fp_hash(uint32_t fp) {
  return uint32_t(xxh64_u64(uint64_t(fp)));
}

// x mod d for 32-bit x and 1 <= d < 2^32, with M = floor((2^64-1)/d) + 1
// precomputed on the host (Lemire, Kaser, Kurz, "Faster remainder by direct
// computation", 2019).
__device__ __forceinline__ uint64_t fastmod32(uint32_t x, uint64_t M,
                                              uint64_t d) {
  return __umul64hi(M * uint64_t(x), d);
}

// Bucket indices fit in 32 bits (m <= 2^32), which halves the registers a
// thread needs per key in flight.
struct KeyHash {
  uint64_t h;
  uint32_t i1, i2;
  uint32_t fp;  // fingerprint proper (without the choice bit)
};

template <class G>
__device__ __forceinline__ uint64_t offset_of(const DevFilter& d, uint32_t fp) {
  return 1u + fastmod32(fp_hash(fp), d.fm_m1, d.m - 1);
}

// The alternate bucket of a key (Eq. 3 / Sec. 4.6.2) from its primary
// bucket and fingerprint.  Kernels call it only for keys that need i2.
template <class G>
__device__ __forceinline__ uint32_t alt_index(const DevFilter& d, uint32_t i1,
                                              uint32_t fp) {
  if constexpr (G::POLICY == 0) {
    return i1 ^ (fp_hash(fp) & uint32_t(d.mask));
  } else {
    const uint64_t j = uint64_t(i1) + offset_of<G>(d, fp);
    return uint32_t(j >= d.m ? j - d.m : j);
  }
}

// Fingerprint and primary bucket (Sec. 4.3 step 1): the upper 32 bits of
// the hash give the fingerprint (0 is EMPTY, so 0 becomes 1), the lower 32
// bits the primary bucket.
template <class G>
__device__ __forceinline__ KeyHash hash_from_h(const DevFilter& d, uint64_t h) {
  KeyHash k;
  k.h = h;
  const uint32_t raw = uint32_t(k.h >> 32) & G::kFpMask;
  k.fp = raw ? raw : 1u;
  if constexpr (G::POLICY == 0)
    k.i1 = uint32_t(k.h) & uint32_t(d.mask);
  else
    k.i1 = uint32_t(fastmod32(uint32_t(k.h), d.fm_m, d.m));
  k.i2 = 0;
  return k;
}

template <class G>
__device__ __forceinline__ KeyHash hash_primary(const DevFilter& d,
                                                uint64_t key) {
  return hash_from_h<G>(d, xxh64_u64(key));
}

template <class G>
__device__ __forceinline__ KeyHash hash_key(const DevFilter& d, uint64_t key) {
  KeyHash k = hash_primary<G>(d, key);
  k.i2 = alt_index<G>(d, k.i1, k.fp);
  return k;
}

// The full hash record of a key from its 64-bit hash alone.
template <class G>
__device__ __forceinline__ KeyHash hash_full_from_h(const DevFilter& d, uint64_t h) {
  KeyHash k = hash_from_h<G>(d, h);
  k.i2 = alt_index<G>(d, k.i1, k.fp);
  return k;
}

// Alternate bucket of a tag stored in bucket j; *moved is the tag as it is
// stored there (the Offset policy flips the choice bit).
template <class G>
__device__ __forceinline__ uint64_t alt_of(const DevFilter& d, uint64_t j,
                                           uint32_t tag, uint32_t& moved) {
  if constexpr (G::POLICY == 0) {
    moved = tag;
    return j ^ (uint64_t(fp_hash(tag)) & d.mask);
  } else {
    const uint32_t fp = tag & G::kFpMask;
    const uint64_t off = offset_of<G>(d, fp);
    if (tag & G::kChoice) {
      moved = fp;
      return j >= off ? j - off : j + d.m - off;
    }
    moved = fp | G::kChoice;
    uint64_t a = j + off;
    return a >= d.m ? a - d.m : a;
  }
}

// Per-key random stream for the eviction loop: splitmix64 seeded with the
// key's 64-bit hash (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t rng_next(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// A failed CAS at retry depth r (0: the loop's first attempt) goes into the
// filter's CAS-retry histogram.  Failures are frequent wherever many keys
// meet in few buckets (the slice-grouped passes, small tables), so every bin
// is counted in the thread: the first-attempt bin in a word, the deeper bins
// (1, 2-3, 4-7, 8-15, 16-63, >= 64) as 5-bit fields of another word, each
// field added to the histogram when it would pass 30 and at the kernel's end.
// Only the failure path pays.
struct CasCount {
  uint32_t first = 0;  // bin 0
  uint32_t deep = 0;   // bins 1..6, 5 bits each
};
// n failed CAS attempts at retry depth r.  The multi-key loops tally a
// round's failures and call this once per round, so the bin arithmetic is
// not repeated for every key of the unrolled loop.  n <= 30.
__device__ __forceinline__ void note_cas_fails(const DevFilter& d, uint32_t r, uint32_t n,
                                               CasCount& cc) {
  if (!CF_CAS_HIST) return;
  if (r == 0) {
    cc.first += n;
    return;
  }
  const int bin = r == 1 ? 1 : r < 4 ? 2 : r < 8 ? 3 : r < 16 ? 4 : r < 64 ? 5 : 6;
  const int sh = 5 * (bin - 1);
  const uint32_t v = ((cc.deep >> sh) & 31u) + n;
  if (v > 30u) {
    atomicAdd(&d.ctrl->cas_retry[bin], (unsigned long long)v);
    cc.deep &= ~(31u << sh);
  } else {
    cc.deep += n << sh;
  }
}
__device__ __forceinline__ void note_cas_fail(const DevFilter& d, uint32_t r,
                                              CasCount& cc) {
  note_cas_fails(d, r, 1u, cc);
}
// The thread's counts, added by one thread (single-thread kernels and the
// per-round flush of the multi-filter eviction kernel).
__device__ __forceinline__ void cas_count_add(const DevFilter& d, CasCount& cc) {
  if (cc.first) atomicAdd(&d.ctrl->cas_retry[0], (unsigned long long)cc.first);
  for (int bin = 1; cc.deep && bin <= 6; ++bin) {
    const uint32_t v = (cc.deep >> (5 * (bin - 1))) & 31u;
    if (v) atomicAdd(&d.ctrl->cas_retry[bin], (unsigned long long)v);
  }
  cc = CasCount{};
}

// ---------------------------------------------------------------------------
// Single-key bucket operations (used by the eviction loops, the serial
// kernel and the rollback path).
// ---------------------------------------------------------------------------
enum : int { TI_FULL = 0, TI_OK = 1, TI_CONTENTION = -1 };

// Bounds-checked builds (-DCF_DEBUG_BOUNDS=1, the library's debug variant):
// every bucket index is checked against m before its address is formed; a
// bad one sets error-word bit 3, the first one is kept (index + 1) in the
// control block, and bucket 0 is used instead, so the access stays inside
// the table (the results are then wrong, and the error word says so).
#ifndef CF_DEBUG_BOUNDS
#define CF_DEBUG_BOUNDS 0
#endif
constexpr uint32_t kErrBounds = 8u;

__device__ __forceinline__ uint64_t checked_bucket(const DevFilter& d, uint64_t j) {
  if (CF_DEBUG_BOUNDS && j >= d.m) {
    atomicOr(&d.ctrl->error_word, kErrBounds);
    atomicCAS(&d.ctrl->debug_bad_index, 0ull, (unsigned long long)j + 1ull);
    return 0;
  }
  return j;
}

template <class G>
__device__ __forceinline__ typename G::Word* bucket_ptr(const DevFilter& d,
                                                        uint64_t j) {
  return reinterpret_cast<typename G::Word*>(d.table) + checked_bucket(d, j) * G::kWpb;
}

// TryInsert (Alg. 1): start word (tag mod b) / tpw, wrap-around scan, CAS
// the tag into the lowest empty lane; on a lost CAS continue from the
// returned word.  `bk` is the bucket as the caller last saw it (stale values
// are safe: the CAS validates); on TI_FULL it holds the words as last
// observed, so the caller can keep using it without another load.
template <class G>
__device__ int try_insert_loaded(const DevFilter& d, uint64_t j, uint32_t tag,
                                 Bucket<G>& bk, CasCount& first) {
  using W = typename G::Word;
  W* base = bucket_ptr<G>(d, j);
  const int start = int((tag % G::B) / G::kTpw);
#pragma unroll
  for (int i = 0; i < G::kWpb; ++i) {
    const int w = (start + i) & (G::kWpb - 1);
    W cur = select_word<G>(bk, w);
    for (int tries = 0;; ++tries) {
      const W z = zero_lanes<G>(cur);
      if (!z) break;
      if (uint32_t(tries) >= cas_bound(d)) return TI_CONTENTION;
      const int lane = first_lane<G>(z);
      const W desired = cur | (W(tag) << (lane * G::F));
      const W old = atomicCAS(base + w, cur, desired);
      if (old == cur) {
        set_word<G>(bk, w, desired);
        return TI_OK;
      }
      note_cas_fail(d, uint32_t(tries), first);
      cur = old;
    }
    set_word<G>(bk, w, cur);
  }
  return TI_FULL;
}

template <class G>
__device__ int try_insert(const DevFilter& d, uint64_t j, uint32_t tag,
                          CasCount& first) {
  Bucket<G> bk = load_bucket<G, false>(bucket_ptr<G>(d, j));
  return try_insert_loaded<G>(d, j, tag, bk, first);
}

// TryRemove (Alg. 3): same scan order; CAS the lowest matching lane to 0.
template <class G>
__device__ int try_remove(const DevFilter& d, uint64_t j, uint32_t tag,
                          CasCount& first) {
  using W = typename G::Word;
  W* base = bucket_ptr<G>(d, j);
  const Bucket<G> bk = load_bucket<G, false>(base);
  const W pat = broadcast<G>(tag);
  const int start = int((tag % G::B) / G::kTpw);
#pragma unroll
  for (int i = 0; i < G::kWpb; ++i) {
    const int w = (start + i) & (G::kWpb - 1);
    W cur = select_word<G>(bk, w);
    for (int tries = 0;; ++tries) {
      const W z = zero_lanes<G>(cur ^ pat);
      if (!z) break;
      if (uint32_t(tries) >= cas_bound(d)) return TI_CONTENTION;
      const int lane = first_lane<G>(z);
      const W desired = cur & ~(G::kLaneMask << (lane * G::F));
      const W old = atomicCAS(base + w, cur, desired);
      if (old == cur) return TI_OK;
      note_cas_fail(d, uint32_t(tries), first);
      cur = old;
    }
  }
  return TI_FULL;
}

struct EvictCounters {
  uint32_t rollbacks = 0, rollback_lost = 0, contention = 0;
  CasCount cas;  // failed CAS attempts by retry depth (note_cas_fail)
};

// Result codes of the eviction loops (the key's flag).
enum : int { EV_FAIL = 0, EV_OK = 1, EV_CONTENTION = 2 };

// State of one key's eviction chain between rounds: the tag in hand, the
// bucket it is destined for (and that bucket's words as last seen), the
// key's random stream and the overwrites so far.
template <class G>
struct Chain {
  uint64_t rng;
  uint64_t cur;
  uint32_t tag;
  uint32_t ev;
  Bucket<G> bk;
};

// A round that neither placed the tag nor gave up.
constexpr int ROUND_CONTINUE = -1;

// One round of the BFS eviction heuristic (Sec. 4.6.1), for a tag destined
// for the full bucket c.cur.  The round inspects b/2 consecutive slots from
// a random start and probes their alternate buckets.  If some candidate's
// alternate has an empty slot, the first such candidate (in order) moves
// there and the new tag takes its slot; otherwise the last candidate is
// evicted and the chain continues from its alternate bucket.
//
// Order of the two writes of a move: the paper inserts the candidate into
// its alternate first and then CASes the new tag over it, undoing the
// insert if that CAS finds the slot changed.  Under contention the undo can
// miss (another thread may have carried the copy on already) and leave a
// duplicate.  Here the new tag is CASed into the candidate's slot first
// (taking whatever that slot holds at that moment), then the evicted tag is
// inserted into its alternate bucket, using the words the probe loaded.  If
// that bucket lost its room meanwhile, the evicted tag stays in hand and
// the chain goes on from there.  A tag is never duplicated or lost; run by
// one thread, both orders leave the same table.  The evicted tag's bucket
// is the chosen candidate's alternate bucket, which the probe has just
// loaded: its words serve the next step (a stale word only costs the CAS
// that detects it), so no round reloads it.
//
// FW alternate buckets (the frontier) are probed together per group,
// groups in candidate order; the choice does not depend on FW.
// Returns EV_OK, EV_CONTENTION (vt/vb = the tag dropped and its bucket) or
// ROUND_CONTINUE.  Precondition: c.ev < max_evictions.
template <class G, int FW>
__device__ int bfs_round(const DevFilter& d, Chain<G>& c, uint32_t& vt,
                         uint64_t& vb, EvictCounters& ec) {
  using W = typename G::Word;
  constexpr int H = G::B / 2;
  static_assert(FW >= 1 && H % FW == 0, "frontier width divides b/2");
  const uint32_t start = uint32_t(rng_next(c.rng) & (G::B - 1));
  W* cbase = bucket_ptr<G>(d, c.cur);
  if (has_empty<G>(c.bk)) {
    // Only reachable under concurrency (a slot freed by a delete).
    if (try_insert_loaded<G>(d, c.cur, c.tag, c.bk, ec.cas) == TI_OK) return EV_OK;
  }
  uint32_t t[H], mv[H];
  uint64_t a[H];
  bool cand[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    t[k] = get_slot<G>(c.bk, (start + k) & (G::B - 1));
    a[k] = alt_of<G>(d, c.cur, t[k], mv[k]);
    cand[k] = t[k] != 0 && a[k] != c.cur;
  }
  int chosen = H - 1;
  bool open = false;
  Bucket<G> tb{};
#pragma unroll
  for (int g = 0; g < H; g += FW) {
    if (open) break;
    Bucket<G> ab[FW];
#pragma unroll
    for (int q = 0; q < FW; ++q)
      if (cand[g + q]) ab[q] = load_bucket_ev<G>(bucket_ptr<G>(d, a[g + q]));
#pragma unroll
    for (int q = 0; q < FW; ++q) {
      if (!open && cand[g + q] && has_empty<G>(ab[q])) {
        open = true;
        chosen = g + q;
        tb = ab[q];
      }
    }
    // No bucket open after the last group: the swap goes to the last
    // candidate, whose alternate bucket's words are ab[FW - 1].
    if (!open && g + FW == H) tb = ab[FW - 1];
  }
  // Swap the new tag into the chosen slot.
  const uint32_t sl = (start + uint32_t(chosen)) & (G::B - 1);
  const int wi = int(sl / G::kTpw), lane = int(sl % G::kTpw);
  W w = select_word<G>(c.bk, wi);
  bool swapped = false;
  uint32_t evicted = 0;
  for (uint32_t tries = 0; tries < cas_bound(d); ++tries) {
    const W old = atomicCAS(cbase + wi, w, replace_lane<G>(w, lane, c.tag));
    if (old == w) {
      evicted = get_lane<G>(w, lane);
      swapped = true;
      break;
    }
    note_cas_fail(d, tries, ec.cas);
    w = old;
  }
  if (!swapped) {
    ec.contention++;
    vt = c.tag;
    vb = c.cur;
    return EV_CONTENTION;
  }
  c.ev++;
  if (evicted == 0) return EV_OK;
  // Carry the evicted tag to its alternate bucket and insert it there.  The
  // evicted tag is the chosen candidate's unless another thread changed the
  // slot meanwhile; only then is its alternate bucket hashed again.
  uint64_t an = 0;
  uint32_t tk = 0, moved = 0;
  bool pre = false;
#pragma unroll
  for (int k = 0; k < H; ++k)
    if (k == chosen) {
      an = a[k];
      tk = t[k];
      moved = mv[k];
      pre = cand[k];
    }
  if (evicted == tk) {
    c.cur = an;
  } else {
    c.cur = alt_of<G>(d, c.cur, evicted, moved);
  }
  c.tag = moved;
  if (pre && evicted == tk)
    c.bk = tb;  // the probe's words of that very bucket
  else
    c.bk = load_bucket_ev<G>(bucket_ptr<G>(d, c.cur));
  const int r = try_insert_loaded<G>(d, c.cur, c.tag, c.bk, ec.cas);
  if (r == TI_OK) return EV_OK;
  if (r == TI_CONTENTION) {
    ec.contention++;
    vt = c.tag;
    vb = c.cur;
    return EV_CONTENTION;
  }
  return ROUND_CONTINUE;
}

// One round of the greedy DFS chain (Alg. 1 phase 2): swap the tag into a
// random slot of c.cur, carry the evicted tag to its alternate bucket, try a
// direct insert there; the words loaded by that attempt serve the next
// round.  Same returns and precondition as bfs_round.
template <class G>
__device__ int dfs_round(const DevFilter& d, Chain<G>& c, uint32_t& vt,
                         uint64_t& vb, EvictCounters& ec) {
  using W = typename G::Word;
  const uint32_t s = uint32_t(rng_next(c.rng) & (G::B - 1));
  const int wi = int(s / G::kTpw), lane = int(s % G::kTpw);
  W* wp = bucket_ptr<G>(d, c.cur) + wi;
  W w = select_word<G>(c.bk, wi);
  bool swapped = false;
  uint32_t evicted = 0;
  for (uint32_t tries = 0; tries < cas_bound(d); ++tries) {
    const W old = atomicCAS(wp, w, replace_lane<G>(w, lane, c.tag));
    if (old == w) {
      evicted = get_lane<G>(w, lane);
      swapped = true;
      break;
    }
    note_cas_fail(d, tries, ec.cas);
    w = old;
  }
  if (!swapped) {
    ec.contention++;
    vt = c.tag;
    vb = c.cur;
    return EV_CONTENTION;
  }
  c.ev++;
  if (evicted == 0) return EV_OK;
  uint32_t moved;
  c.cur = alt_of<G>(d, c.cur, evicted, moved);
  c.tag = moved;
  c.bk = load_bucket_ev<G>(bucket_ptr<G>(d, c.cur));
  const int r = try_insert_loaded<G>(d, c.cur, c.tag, c.bk, ec.cas);
  if (r == TI_OK) return EV_OK;
  if (r == TI_CONTENTION) {
    ec.contention++;
    vt = c.tag;
    vb = c.cur;
    return EV_CONTENTION;
  }
  return ROUND_CONTINUE;
}

// ---------------------------------------------------------------------------
// Full-bucket map of the eviction loop: bit j of the map is set only if
// bucket j has no empty slot.  During an insert batch buckets only gain
// tags, so a bucket once full stays full: a set bit is always right, and a
// clear bit is either right or stale (the bucket has filled since).  The
// map is built by one pass over the table before the eviction kernel and
// kept up by the eviction rounds (a round that fills a bucket, or finds a
// bucket full that the map called open, sets its bit).
// ---------------------------------------------------------------------------
// The map's accesses carry an L2 evict_last policy (CF_MAP_EVICT_LAST): the
// map is read by every round while the rounds' random bucket lines stream
// through L2, and a map word evicted by them costs a round a second DRAM
// access.
#ifndef CF_MAP_EVICT_LAST
#define CF_MAP_EVICT_LAST 1
#endif
__device__ __forceinline__ uint64_t map_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint32_t map_word(const DevFilter& d, const uint32_t* map,
                                             uint64_t j) {
  const uint32_t* p = map + (checked_bucket(d, j) >> 5);
  if (CF_MAP_EVICT_LAST) {
    uint32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(map_policy()));
    return v;
  }
  return ld_cg_u32(p);  // L2: coherent with map_set
}
__device__ __forceinline__ void map_set(const DevFilter& d, uint32_t* map, uint64_t j) {
  j = checked_bucket(d, j);
  uint32_t* p = map + (j >> 5);
  const uint32_t bit = 1u << (j & 31);
  if (CF_MAP_EVICT_LAST) {
    uint32_t old;
    asm volatile("atom.global.L2::cache_hint.or.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(p), "r"(bit), "l"(map_policy()) : "memory");
  } else {
    atomicOr(p, bit);
  }
}
__device__ __forceinline__ void map_store(uint32_t* p, uint32_t v) {
  if (CF_MAP_EVICT_LAST)
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;"
                 :: "l"(p), "r"(v), "l"(map_policy()) : "memory");
  else
    *p = v;
}

// The tag as stored in the alternate bucket of a bucket that holds t (the
// `moved` of alt_of: the Offset policy flips the choice bit).
template <class G>
__device__ __forceinline__ uint32_t moved_tag(uint32_t t) {
  return G::POLICY == 0 ? t : (t ^ G::kChoice);
}

// The CAS loop of a swap: c.tag into lane `lane` of word wi of bucket c.cur,
// from the word as last seen (w), attempts tries0 .. the bound.  True with
// the lane's previous tag in evicted; false if the bound ran out.
template <class G>
__device__ __forceinline__ bool swap_cas(const DevFilter& d, const Chain<G>& c, int wi, int lane,
                                         typename G::Word w, uint32_t tries0, CasCount& cc,
                                         uint32_t& evicted) {
  using W = typename G::Word;
  W* p = bucket_ptr<G>(d, c.cur) + wi;
  for (uint32_t tries = tries0; tries < cas_bound(d); ++tries) {
    const W old = atomicCAS(p, w, replace_lane<G>(w, lane, c.tag));
    if (old == w) {
      evicted = get_lane<G>(w, lane);
      return true;
    }
    note_cas_fail(d, tries, cc);
    w = old;
  }
  return false;
}

// After a swap took `evicted` from the chosen slot (whose tag was tk when
// the candidates were read; its alternate bucket an, a candidate when pre,
// open if the map called an open): EV_OK if the slot was empty, else
// ROUND_CONTINUE with c at the evicted tag's alternate bucket and tag as
// stored there, and mark = whether that bucket's map bit may be clear (the
// map called it open, or the move went elsewhere than the chosen
// candidate's bucket).  The evicted tag is tk unless another thread changed
// the slot meanwhile; only then is its alternate bucket hashed again.
template <class G>
__device__ __forceinline__ int swap_tail(const DevFilter& d, Chain<G>& c, uint32_t evicted,
                                         uint32_t tk, uint64_t an, bool pre, bool open,
                                         bool& mark) {
  c.ev++;
  if (evicted == 0) return EV_OK;
  uint32_t moved = moved_tag<G>(tk);
  uint64_t dest = an;
  if (evicted != tk) dest = alt_of<G>(d, c.cur, evicted, moved);
  mark = open || !pre || evicted != tk;
  c.cur = dest;
  c.tag = moved;
  return ROUND_CONTINUE;
}

// The choice and the swap of a BFS round with the full-bucket map, for the
// tag c.tag destined for the full bucket c.cur (words c.bk), with the
// round's random start.  Returns EV_OK (the swap took an empty slot),
// EV_CONTENTION (vt/vb = the tag dropped and its bucket) or ROUND_CONTINUE
// (see swap_tail).  With PREFETCH the chosen candidate's alternate bucket is
// loaded while the swap's CAS runs: nb holds its words when have_nb.
template <class G, bool PREFETCH>
__device__ __forceinline__ int bfs_swap_map(const DevFilter& d, Chain<G>& c, uint32_t start,
                                            uint32_t* map, uint32_t& vt, uint64_t& vb,
                                            EvictCounters& ec, bool& mark, Bucket<G>& nb,
                                            bool& have_nb) {
  constexpr int H = G::B / 2;
  uint32_t t[H], mw[H];
  uint64_t a[H];
  bool cand[H];
#pragma unroll
  for (int k = 0; k < H; ++k) {
    t[k] = get_slot<G>(c.bk, (start + k) & (G::B - 1));
    uint32_t mv;
    a[k] = alt_of<G>(d, c.cur, t[k], mv);
    cand[k] = t[k] != 0 && a[k] != c.cur;
  }
#pragma unroll
  for (int k = 0; k < H; ++k) mw[k] = cand[k] ? map_word(d, map, a[k]) : ~0u;
  int chosen = H - 1;
  bool open = false;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    if (!open && cand[k] && !((mw[k] >> (a[k] & 31)) & 1u)) {
      open = true;
      chosen = k;
    }
  }
  // The chosen candidate's tag and alternate bucket (computed above).
  uint64_t an = 0;
  uint32_t tk = 0;
  bool pre = false;
#pragma unroll
  for (int k = 0; k < H; ++k)
    if (k == chosen) {
      an = a[k];
      tk = t[k];
      pre = cand[k];
    }
  if (PREFETCH && pre) nb = load_bucket_ev<G>(bucket_ptr<G>(d, an));
  const uint32_t sl = (start + uint32_t(chosen)) & (G::B - 1);
  const int wi = int(sl / G::kTpw), lane = int(sl % G::kTpw);
  uint32_t evicted = 0;
  if (!swap_cas<G>(d, c, wi, lane, select_word<G>(c.bk, wi), 0, ec.cas, evicted)) {
    ec.contention++;
    vt = c.tag;
    vb = c.cur;
    return EV_CONTENTION;
  }
  have_nb = PREFETCH && pre && evicted == tk;
  return swap_tail<G>(d, c, evicted, tk, an, pre, open, mark);
}

// One round of the BFS eviction heuristic (Sec. 4.6.1) that asks the
// full-bucket map, not the buckets themselves, whether each candidate's
// alternate bucket has an empty slot.  Same candidates, same choice (the
// first candidate, in order, whose alternate is open; else the last), same
// swap-first move as bfs_round.  Only the bucket that receives the evicted
// tag is loaded: it is the chosen candidate's alternate, which the next
// step needs anyway (to insert into it, or as the next round's bucket), so
// a round costs one bucket load from DRAM instead of one per inspected
// candidate.  A stale clear bit costs what a stale loaded word costs under
// concurrency: the insert finds the bucket full, the tag stays in hand and
// the chain goes on from there (and the bit is set).  Run by one thread on
// an exact map, the round takes the same steps as bfs_round.
template <class G>
__device__ int bfs_round_map(const DevFilter& d, Chain<G>& c, uint32_t* map,
                             uint32_t& vt, uint64_t& vb, EvictCounters& ec) {
  const uint32_t start = uint32_t(rng_next(c.rng) & (G::B - 1));
  if (has_empty<G>(c.bk)) {
    // Only reachable under concurrency (a slot freed by a delete).
    if (try_insert_loaded<G>(d, c.cur, c.tag, c.bk, ec.cas) == TI_OK) {
      if (!has_empty<G>(c.bk)) map_set(d, map, c.cur);
      return EV_OK;
    }
  }
  bool mark = false, have_nb = false;
  Bucket<G> nb{};
  const int sw = bfs_swap_map<G, true>(d, c, start, map, vt, vb, ec, mark, nb, have_nb);
  if (sw != ROUND_CONTINUE) return sw;
  c.bk = have_nb ? nb : load_bucket_ev<G>(bucket_ptr<G>(d, c.cur));
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
  // c.cur is full.  Its bit is set already unless the swap marked it.
  if (mark) map_set(d, map, c.cur);
  return ROUND_CONTINUE;
}

// Start of phase 2 of Alg. 1 for a key whose two buckets were full: the
// key's first random draw picks i1 or i2, whose words are loaded.
template <class G>
__device__ __forceinline__ Chain<G> chain_start(const DevFilter& d,
                                                const KeyHash& kh) {
  Chain<G> c;
  c.rng = kh.h;
  const bool first = (rng_next(c.rng) & 1) == 0;
  c.cur = first ? kh.i1 : kh.i2;
  c.tag = first ? kh.fp : (kh.fp | G::kChoice);
  c.ev = 0;
  c.bk = load_bucket_ev<G>(bucket_ptr<G>(d, c.cur));
  return c;
}

// The start of a chain without its bucket's words: the random stream after
// the first draw, the bucket it picked (i1 or i2) and the tag as stored
// there, from the key's 64-bit hash.  The alternate bucket is hashed only
// when the draw picks it.
template <class G>
struct ChainHead {
  uint64_t rng;
  uint64_t cur;
  uint32_t tag;
};
template <class G>
__device__ __forceinline__ ChainHead<G> chain_head(const DevFilter& d, uint64_t h) {
  const KeyHash kh = hash_from_h<G>(d, h);
  ChainHead<G> p;
  p.rng = h;
  const bool first = (rng_next(p.rng) & 1) == 0;
  p.cur = first ? kh.i1 : alt_index<G>(d, kh.i1, kh.fp);
  p.tag = first ? kh.fp : (kh.fp | G::kChoice);
  return p;
}

// chain_start from a head whose bucket's words were loaded beforehand.
template <class G>
__device__ __forceinline__ Chain<G> chain_start_loaded(const ChainHead<G>& p,
                                                       const Bucket<G>& bk) {
  Chain<G> c;
  c.rng = p.rng;
  c.cur = p.cur;
  c.tag = p.tag;
  c.ev = 0;
  c.bk = bk;
  return c;
}

// One round of the filter's eviction policy, or EV_FAIL when the chain has
// used max_evictions overwrites (the tag in hand is the victim).
template <class G, int FW = G::B / 2>
__device__ __forceinline__ int evict_round(const DevFilter& d, Chain<G>& c,
                                           uint32_t& vt, uint64_t& vb,
                                           EvictCounters& ec) {
  if (c.ev >= d.max_ev) {
    vt = c.tag;
    vb = c.cur;
    return EV_FAIL;
  }
  return d.eviction == 1 ? dfs_round<G>(d, c, vt, vb, ec)
                         : bfs_round<G, FW>(d, c, vt, vb, ec);
}

// Phase 2 of Alg. 1 for one key, run to the end by one thread.
template <class G, int FW = G::B / 2>
__device__ int evict_key(const DevFilter& d, const KeyHash& kh, uint32_t& ev,
                         uint32_t& vt, uint64_t& vb, EvictCounters& ec) {
  ev = 0;
  if (d.max_ev == 0) {
    vt = kh.fp;
    vb = kh.i1;
    return EV_FAIL;
  }
  Chain<G> c = chain_start<G>(d, kh);
  int r;
  do {
    r = evict_round<G, FW>(d, c, vt, vb, ec);
  } while (r == ROUND_CONTINUE);
  ev = c.ev;
  return r;
}

// evict_round with the full-bucket map for BFS (DFS never probes, so it
// has no use for the map).
template <class G>
__device__ __forceinline__ int evict_round_map(const DevFilter& d, Chain<G>& c,
                                               uint32_t* map, uint32_t& vt,
                                               uint64_t& vb, EvictCounters& ec) {
  if (c.ev >= d.max_ev) {
    vt = c.tag;
    vb = c.cur;
    return EV_FAIL;
  }
  return d.eviction == 1 ? dfs_round<G>(d, c, vt, vb, ec)
                         : bfs_round_map<G>(d, c, map, vt, vb, ec);
}

// evict_key with the full-bucket map (one thread; the serial kernel).
template <class G>
__device__ int evict_key_map(const DevFilter& d, const KeyHash& kh, uint32_t* map,
                             uint32_t& ev, uint32_t& vt, uint64_t& vb,
                             EvictCounters& ec) {
  ev = 0;
  if (d.max_ev == 0) {
    vt = kh.fp;
    vb = kh.i1;
    return EV_FAIL;
  }
  Chain<G> c = chain_start<G>(d, kh);
  int r;
  do {
    r = evict_round_map<G>(d, c, map, vt, vb, ec);
  } while (r == ROUND_CONTINUE);
  ev = c.ev;
  return r;
}

__device__ __forceinline__ void log_victim(const DevFilter& d, uint32_t tag,
                                           uint64_t bucket) {
  const unsigned long long i = atomicAdd(&d.ctrl->victims, 1ull);
  if (i < d.victim_cap) {
    d.victims[i].tag = tag;
    d.victims[i].bucket = bucket;
  } else {
    atomicOr(&d.ctrl->error_word, 2u);
  }
}

// Block-wide sum of a per-thread count, added to *dst by one atomic per
// block (the hierarchical reduction of Sec. 4.3: warp shuffle, shared
// memory, one global atomic).  Every thread of the block must call it.
__device__ __forceinline__ void block_add(unsigned long long* dst, uint32_t v,
                                          bool negate = false) {
  __shared__ unsigned long long s_part[32];
  unsigned long long x = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) s_part[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long y = lane < nw ? s_part[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xFFFFFFFFu, y, o);
    if (lane == 0 && y) atomicAdd(dst, negate ? (0ull - y) : y);
  }
  __syncthreads();
}

// The block's CAS counts added to the histogram (every thread of the block
// must call it; the deep bins cost barriers only when some thread has them).
__device__ __forceinline__ void cas_count_block_add(const DevFilter& d, const CasCount& cc) {
  if (!CF_CAS_HIST) return;
  block_add(&d.ctrl->cas_retry[0], cc.first);
  if (__syncthreads_or(cc.deep != 0)) {
#pragma unroll
    for (int bin = 1; bin <= 6; ++bin)
      block_add(&d.ctrl->cas_retry[bin], (cc.deep >> (5 * (bin - 1))) & 31u);
  }
}

}  // namespace cfk
