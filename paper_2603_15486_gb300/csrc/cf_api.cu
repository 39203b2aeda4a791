// Host side of libcf: the C ABI declared in include/cf.h.
//
// One filter = one device allocation laid out as
//   [control block 256 B][victim log, 16 B per entry][table]
// (each piece 256-byte aligned), plus library-owned scratch: the eviction
// work queue of the insert (4 bytes per key of the largest chunk seen), the
// scratch of the slice-partitioned path (about 48 bytes per key of its chunk),
// the full-bucket map of the eviction loop (m/8 bytes) and, for the *_host
// calls, four staging slots of keys and two device buffers of flags.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "cf.h"
#include "cf_internal.h"
#include "cf_kernels.cuh"

using cfk::Ctrl;
using cfk::DevFilter;
using cfk::Victim;
using cfk::Stage;

namespace {

constexpr uint64_t kInsertChunk = 1ull << 28;  // keys per insert launch pair
// Slice-partitioned path: defaults and the automatic rule.  A slice of 32 MiB
// stays resident in L2 (129 MB) next to the streams (measured on the 2 GiB
// table: 2 / 4 / 8 / 16 / 32 MiB slices gave 187 / 174 / 162 / 157 / 154
// ms per benchmark step; smaller slices shorten the runs the result gathers
// walk); the path pays off when the table is several times L2 and a batch
// touches each slice many times.
constexpr uint64_t kSliceBytes = 32ull << 20;
constexpr uint64_t kSliceChunk = 1ull << 28;   // keys per sliced pass
constexpr uint64_t kSliceChunkMax = 1ull << 30;
constexpr uint64_t kSliceAutoTable = 256ull << 20;
constexpr uint32_t kDefaultVictims = 4096;
constexpr uint32_t kMaxVictims = 1u << 26;

thread_local char g_err[256] = "";

void set_err(const char* what, cudaError_t e) {
  snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
}

#define CF_CUDA(call)                   \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) {            \
      set_err(#call, e_);               \
      return CF_ECUDA;                  \
    }                                   \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

bool valid_config(const cf_config* c) {
  if (!c) return false;
  if (!(c->fp_bits == 8 || c->fp_bits == 16 || c->fp_bits == 32)) return false;
  if (!(c->slots_per_bucket == 4 || c->slots_per_bucket == 8 ||
        c->slots_per_bucket == 16))
    return false;
  if (c->policy == CF_POLICY_XOR) {
    if (!is_pow2(c->num_buckets) || c->num_buckets > (1ull << 32)) return false;
  } else if (c->policy == CF_POLICY_OFFSET) {
    if (c->num_buckets < 2 || c->num_buckets >= (1ull << 32)) return false;
  } else {
    return false;
  }
  if (c->eviction != CF_EVICT_BFS && c->eviction != CF_EVICT_DFS) return false;
  if (c->victim_capacity > kMaxVictims) return false;
  return true;
}

uint32_t victim_cap(const cf_config* c) {
  return c->victim_capacity ? c->victim_capacity : kDefaultVictims;
}

uint64_t bucket_bytes(const cf_config* c) {
  return uint64_t(c->slots_per_bucket) * c->fp_bits / 8;
}

size_t table_bytes(const cf_config* c) {
  return size_t(c->num_buckets) * c->slots_per_bucket * c->fp_bits / 8;
}

uint64_t fastmod_magic(uint64_t d) {
  // floor((2^64 - 1) / d) + 1; d == 1 gives 0, which yields x mod 1 == 0.
  return d ? (~0ull / d + 1) : 0;
}

DevFilter make_dev(const cf_config* c, char* mem) {
  DevFilter d{};
  d.ctrl = reinterpret_cast<Ctrl*>(mem);
  d.victims = reinterpret_cast<Victim*>(mem + 256);
  d.victim_cap = victim_cap(c);
  d.table = mem + 256 + align256(size_t(d.victim_cap) * sizeof(Victim));
  d.m = c->num_buckets;
  d.mask = c->num_buckets - 1;
  d.fm_m = fastmod_magic(c->num_buckets);
  d.fm_m1 = fastmod_magic(c->num_buckets - 1);
  d.max_ev = c->max_evictions;
  d.eviction = c->eviction;
  d.max_cas = cfk::kMaxCas;
  return d;
}

std::mutex g_mu;
std::unordered_map<int, int> g_sms;
std::unordered_map<const void*, int> g_occ[64];

}  // namespace

namespace cfk {

int device_sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  g_sms[dev] = sms;
  return sms;
}

int cached_occupancy(const void* fn, int block) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto& m = g_occ[dev & 63];
  auto it = m.find(fn);
  if (it != m.end()) return it->second;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, 0) !=
          cudaSuccess ||
      occ < 1)
    occ = 1;
  m[fn] = occ;
  return occ;
}

cf_status order_on(cf_filter* f, cudaStream_t s) {
  if (f->has_last && f->last_stream != s) {
    cudaEvent_t ev = f->ext_ev ? f->ext_ev : f->last_ev;
    cudaError_t e = cudaStreamWaitEvent(s, ev, 0);
    if (e != cudaSuccess) {
      set_error("cudaStreamWaitEvent", e);
      return CF_ECUDA;
    }
  }
  return CF_OK;
}

cf_status mark(cf_filter* f, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(f->last_ev, s);
  if (e != cudaSuccess) {
    set_error("cudaEventRecord", e);
    return CF_ECUDA;
  }
  f->ext_ev = nullptr;
  f->last_stream = s;
  f->has_last = true;
  return CF_OK;
}

void mark_external(cf_filter* f, cudaStream_t s, cudaEvent_t ev) {
  f->ext_ev = ev;
  f->last_stream = s;
  f->has_last = true;
}

cudaEvent_t pooled_event() {
  // Events handed to filters by batched launches live until process exit.
  cudaEvent_t ev = nullptr;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  return ev;
}

void set_error(const char* what, cudaError_t e) { set_err(what, e); }
void set_error_text(const char* text) { snprintf(g_err, sizeof g_err, "%s", text); }

}  // namespace cfk

namespace {

using cfk::mark;
using cfk::order_on;

cf_status ensure_queue(cf_filter* f, uint64_t keys, uint64_t cap = kInsertChunk) {
  const uint64_t want = keys < cap ? keys : cap;
  if (want <= f->queue_cap) return CF_OK;
  if (f->queue) CF_CUDA(cudaFree(f->queue));
  f->queue = nullptr;
  f->queue_cap = 0;
  if (cudaMalloc(&f->queue, want * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_err, sizeof g_err, "eviction queue of %llu keys",
             (unsigned long long)want);
    return CF_ENOMEM;
  }
  f->queue_cap = want;
  return CF_OK;
}

cf_status init_filter(cf_filter* f, const cf_config* cfg, char* mem,
                      size_t bytes, bool owns) {
  f->cfg = *cfg;
  if (!f->cfg.victim_capacity) f->cfg.victim_capacity = kDefaultVictims;
  CF_CUDA(cudaGetDevice(&f->device));
  f->mem = mem;
  f->mem_bytes = bytes;
  f->owns = owns;
  f->d = make_dev(&f->cfg, mem);
  f->ops = cfk::get_ops(int(cfg->fp_bits), int(cfg->slots_per_bucket),
                        int(cfg->policy));
  if (!f->ops) return CF_ENOTSUP;
  CF_CUDA(cudaEventCreateWithFlags(&f->last_ev, cudaEventDisableTiming));
  CF_CUDA(cudaMemset(mem, 0, bytes));
  CF_CUDA(cudaDeviceSynchronize());
  return CF_OK;
}

void free_staging(cf_filter* f) {
  for (auto& st : f->stage) {
    if (st.keys) cudaFree(st.keys);
    if (st.in_done) cudaEventDestroy(st.in_done);
    if (st.comp_done) cudaEventDestroy(st.comp_done);
    st = Stage{};
  }
  for (auto& g : f->fgroup) {
    if (g.flags) cudaFree(g.flags);
    if (g.comp_done) cudaEventDestroy(g.comp_done);
    if (g.out_done) cudaEventDestroy(g.out_done);
    g = cfk::FlagGroup{};
  }
  if (f->s_in) cudaStreamDestroy(f->s_in);
  if (f->s_out) cudaStreamDestroy(f->s_out);
  f->s_in = f->s_out = nullptr;
  f->next_slot = f->next_group = 0;
  f->stage_ready = false;
}

cf_status ensure_staging(cf_filter* f) {
  if (f->stage_ready) return CF_OK;
  const uint64_t c = f->stage_chunk;
  f->group_chunks = cfk::kFlagGroupBytes / c ? cfk::kFlagGroupBytes / c : 1;
  for (auto& st : f->stage) {
    if (cudaMalloc(&st.keys, c * sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();
      free_staging(f);
      return CF_ENOMEM;
    }
    CF_CUDA(cudaEventCreateWithFlags(&st.in_done, cudaEventDisableTiming));
    CF_CUDA(cudaEventCreateWithFlags(&st.comp_done, cudaEventDisableTiming));
  }
  for (auto& g : f->fgroup) {
    CF_CUDA(cudaEventCreateWithFlags(&g.comp_done, cudaEventDisableTiming));
    CF_CUDA(cudaEventCreateWithFlags(&g.out_done, cudaEventDisableTiming));
  }
  CF_CUDA(cudaStreamCreateWithFlags(&f->s_in, cudaStreamNonBlocking));
  CF_CUDA(cudaStreamCreateWithFlags(&f->s_out, cudaStreamNonBlocking));
  f->stage_ready = true;
  return CF_OK;
}

// Both flag buffers hold at least `bytes`.  Growing one waits for the work
// that still uses it.
cf_status ensure_flag_groups(cf_filter* f, uint64_t bytes) {
  for (auto& g : f->fgroup) {
    if (g.cap >= bytes) continue;
    if (g.used) CF_CUDA(cudaEventSynchronize(g.out_done));
    if (g.flags) CF_CUDA(cudaFree(g.flags));
    g.flags = nullptr;
    g.cap = 0;
    if (cudaMalloc(&g.flags, bytes) != cudaSuccess) {
      cudaGetLastError();
      snprintf(g_err, sizeof g_err, "flag staging of %llu bytes", (unsigned long long)bytes);
      return CF_ENOMEM;
    }
    g.cap = bytes;
  }
  return CF_OK;
}

enum Op { OP_INSERT, OP_CONTAINS, OP_REMOVE };  // = cfk::SOP_* values

// Slice geometry of a filter: 2^shift buckets per slice, S slices, S at most
// kSliceMax (larger tables get larger slices).
void slice_geometry(const cf_filter* f, uint32_t* shift, uint32_t* S) {
  const uint64_t bb = uint64_t(f->cfg.slots_per_bucket) * f->cfg.fp_bits / 8;
  const uint64_t want = (f->slice_bytes ? f->slice_bytes : kSliceBytes) / bb;
  uint32_t sh = 0;
  while ((2ull << sh) <= want) ++sh;
  const uint64_t m = f->cfg.num_buckets;
  while (((m + (1ull << sh) - 1) >> sh) > cfk::kSliceMax) ++sh;
  *shift = sh;
  *S = uint32_t((m + (1ull << sh) - 1) >> sh);
}

uint64_t slice_chunk(const cf_filter* f) {
  return f->slice_chunk ? f->slice_chunk : kSliceChunk;
}

bool use_sliced(const cf_filter* f, uint64_t n, const uint32_t* evout) {
  if (evout || f->slice_mode == 0) return false;
  if (f->slice_mode == 2) return true;
  return table_bytes(&f->cfg) >= kSliceAutoTable && n >= f->cfg.num_buckets / 8;
}

// Full-bucket map of the eviction loop (bfs_round_map).  Automatic rule:
// BFS filters whose table L2 does not hold (more than 64 MiB), for eviction
// queues of at least m/16 keys.  Building the map reads the whole table
// once (about 0.33 ms for 2 GiB); each BFS round then loads one bucket
// instead of one per inspected candidate, which pays once the queue holds a
// few million chains.  Below the threshold the map kernel returns at once
// and the eviction loop probes buckets as before.
uint32_t map_min_queue(const cf_filter* f) {
  if (f->map_min_queue) return uint32_t(f->map_min_queue < 0xFFFFFFFFull ? f->map_min_queue : 0xFFFFFFFFull);
  if (f->map_mode == 2) return 0;
  const uint64_t q = f->cfg.num_buckets / 16;
  return uint32_t(q < 0xFFFFFFFFull ? (q ? q : 1) : 0xFFFFFFFFull);
}

bool use_map(const cf_filter* f) {
  if (f->map_mode == 0 || f->cfg.eviction != CF_EVICT_BFS) return false;
  if (f->map_mode == 2) return true;
  return table_bytes(&f->cfg) > cfk::kL2TableBytes;
}

cf_status ensure_map(cf_filter* f) {
  if (f->fullmap) return CF_OK;
  const size_t words = size_t((f->cfg.num_buckets + 31) / 32);
  if (cudaMalloc(&f->fullmap, words * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    f->fullmap = nullptr;
    snprintf(g_err, sizeof g_err, "full-bucket map of %zu bytes", words * 4);
    return CF_ENOMEM;
  }
  return CF_OK;
}

// Slice-grouped eviction levels (cf_levels.cuh), for sliced BFS inserts
// with the full-bucket map.  Defaults: 12 levels; the levels run for
// eviction queues of at least 2^20 keys, and stop once a level would have
// fewer than 2^18 chains (the rest run to their end in the loop's manner).
// The record buffers hold half a pass (two buffers of 24 bytes per record,
// about 26 bytes per key of the pass); a larger queue takes the eviction
// loop.
constexpr uint32_t kLevelsDefault = 12;
constexpr uint32_t kLevelsMax = 256;
constexpr uint64_t kLevelMinQueue = 1ull << 20;
constexpr uint64_t kLevelStopQueue = 1ull << 18;

uint32_t clamp_u32(uint64_t v) { return uint32_t(v < 0xFFFFFFFFull ? v : 0xFFFFFFFFull); }

void free_levels(cf_filter* f) {
  if (f->lv_mem) cudaFree(f->lv_mem);
  f->lv_mem = nullptr;
  f->lv = cfk::LevelBufs{};
  f->lv_cap_n = 0;
}

// Buffers for passes of up to n keys over the slice geometry of f->sb.
cf_status ensure_levels(cf_filter* f, uint64_t n) {
  const uint32_t S = f->sb.n_slices;
  const uint32_t L = f->lv_levels ? f->lv_levels : kLevelsDefault;
  if (f->lv_mem && f->lv_cap_n >= n && f->lv.n_levels == L &&
      f->lv.fill && f->lv.cap && f->lv_slices == S)
    return CF_OK;
  free_levels(f);
  const uint64_t R = (n + 1) / 2;
  const double per = double(R) / S;
  const uint64_t cap = uint64_t(per + 6.0 * sqrt(per)) + 64;
  const uint64_t spill = R / 16 + 1024;
  const uint64_t recs = uint64_t(S) * cap + spill;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  // Counters and ctl adjacent: one memset clears both.
  const size_t fill_bytes = size_t(L + 1) * (S + 2) * 128;
  const size_t o_fill = take(fill_bytes + size_t(L + 2) * 4);
  const size_t o_r0 = take(recs * 24), o_r1 = take(recs * 24);
  char* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_err, sizeof g_err, "eviction level buffers of %llu bytes",
             (unsigned long long)off);
    return CF_ENOMEM;
  }
  cfk::LevelBufs& lb = f->lv;
  lb.fill = reinterpret_cast<uint32_t*>(mem + o_fill);
  lb.ctl = reinterpret_cast<uint32_t*>(mem + o_fill + fill_bytes);
  lb.rec[0] = reinterpret_cast<uint64_t*>(mem + o_r0);
  lb.rec[1] = reinterpret_cast<uint64_t*>(mem + o_r1);
  lb.cap = cap;
  lb.spill = spill;
  lb.n_levels = L;
  f->lv_mem = mem;
  f->lv_cap_n = n;
  f->lv_slices = S;
  return CF_OK;
}

// The map argument of one insert call (allocating the map on first use);
// with level_n > 0 (a sliced pass of up to level_n keys) also the eviction
// levels.
cf_status evict_map_for(cf_filter* f, cfk::EvictMap* em, uint64_t level_n = 0) {
  *em = cfk::EvictMap{};
  if (!use_map(f)) return CF_OK;
  cf_status st = ensure_map(f);
  if (st != CF_OK) return st;
  em->bits = f->fullmap;
  em->min_q = map_min_queue(f);
  if (level_n) {
    // Without room for the level buffers the insert keeps the loop (and
    // the failed allocation is not the call's error).
    if (ensure_levels(f, level_n) != CF_OK) {
      g_err[0] = 0;
      return CF_OK;
    }
    em->lv = f->lv;
    em->lv.min_q = clamp_u32(f->lv_min_queue ? f->lv_min_queue : kLevelMinQueue);
    em->lv.stop_q = clamp_u32(f->lv_stop_queue ? f->lv_stop_queue : kLevelStopQueue);
  }
  return CF_OK;
}

void free_slice(cf_filter* f) {
  if (f->sb_mem) cudaFree(f->sb_mem);
  f->sb_mem = nullptr;
  f->sb = cfk::SliceBufs{};
  f->sb_cap = 0;
}

// Scratch for chunks of up to n keys (one allocation, 256-byte aligned
// pieces).  rec1 and rec2 hold S regions plus a spill region of n:
// n/S + 6 sqrt(n/S) + 64 records per region keep uniform hashes inside their
// slice (rec1's rounded up to 256 records, so that its regions and tiles
// start on 2 KB boundaries).  Positions in rec1 and rec2 fit 32 bits: both
// hold at most about 2n + S * (6 sqrt(n/S) + 320) records, n <= 2^30.
cf_status ensure_slice(cf_filter* f, uint64_t n) {
  uint32_t shift = 0, S = 0;
  slice_geometry(f, &shift, &S);
  if (f->sb_mem && f->sb_cap >= n && f->sb.n_slices == S && f->sb.shift == shift)
    return CF_OK;
  free_slice(f);
  const double per = double(n) / S;
  const uint64_t cap2 = uint64_t(per + 6.0 * sqrt(per)) + 64;
  const uint64_t cap1 = (cap2 + 255) / 256 * 256;
  const uint64_t n1 = uint64_t(S) * cap1 + n;
  const uint64_t n2 = uint64_t(S) * cap2 + n;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  // Counters one per 128-byte line (32 words apart); fill1 and fill2 are
  // adjacent so that one memset clears both.
  const size_t o_fill1 = take(size_t(S + 1) * 128);
  const size_t o_fill2 = take(size_t(S + cfk::kFill2Extra) * 128);
  const size_t o_dst = take(n * 4), o_rec1 = take(n1 * 8), o_f1 = take(n1);
  const size_t o_link = take(n1 * 4), o_rec2 = take(n2 * 8), o_f2 = take(n2);
  char* mem = nullptr;
  if (cudaMalloc(&mem, off) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_err, sizeof g_err, "slice scratch of %llu bytes", (unsigned long long)off);
    return CF_ENOMEM;
  }
  cfk::SliceBufs& b = f->sb;
  b.n_slices = S;
  b.shift = shift;
  b.cap1 = cap1;
  b.cap2 = cap2;
  b.rec2_len = n2;
  b.fill1 = reinterpret_cast<uint32_t*>(mem + o_fill1);
  b.fill2 = reinterpret_cast<uint32_t*>(mem + o_fill2);
  b.dst = reinterpret_cast<uint32_t*>(mem + o_dst);
  b.rec1 = reinterpret_cast<uint64_t*>(mem + o_rec1);
  b.f1 = reinterpret_cast<uint8_t*>(mem + o_f1);
  b.link = reinterpret_cast<uint32_t*>(mem + o_link);
  b.rec2 = reinterpret_cast<uint64_t*>(mem + o_rec2);
  b.f2 = reinterpret_cast<uint8_t*>(mem + o_f2);
  f->sb_mem = mem;
  f->sb_cap = n;
  return CF_OK;
}

cf_status run_sliced(cf_filter* f, Op op, const uint64_t* keys, uint64_t n,
                     uint8_t* flags, cudaStream_t s) {
  // Equal passes of at most the chunk: a short last pass would sweep the
  // table's slices for few records.
  const uint64_t cap = slice_chunk(f);
  const uint64_t passes = (n + cap - 1) / cap;
  const uint64_t chunk = (n + passes - 1) / passes;
  cf_status st = ensure_slice(f, chunk);
  if (st != CF_OK) return st;
  cfk::EvictMap em;
  if (op == OP_INSERT) {
    st = ensure_queue(f, chunk, kSliceChunkMax);
    if (st != CF_OK) return st;
    // Automatic mode: buckets of up to 8 bytes (with wider buckets the
    // levels measured slower than the loop: f16 b16 fill to LF 0.95 on
    // 2^28 slots 21.7 against 23.9 G inserts/s).
    const bool lv = f->lv_mode == 2 || (f->lv_mode == 1 && bucket_bytes(&f->cfg) <= 8);
    st = evict_map_for(f, &em, lv ? chunk : 0);
    if (st != CF_OK) return st;
  }
  for (uint64_t off = 0; off < n; off += chunk) {
    const uint64_t len = (n - off) < chunk ? (n - off) : chunk;
    const cudaError_t e = f->ops->sliced(f->d, int(op), keys + off, len,
                                         flags ? flags + off : nullptr, f->sb,
                                         f->queue, em, s, f->timer);
    if (e != cudaSuccess) {
      set_err("sliced kernel launch", e);
      return CF_ECUDA;
    }
  }
  return CF_OK;
}

cf_status run_op(cf_filter* f, Op op, const uint64_t* keys, uint64_t n,
                 uint8_t* flags, uint32_t* evout, cudaStream_t s) {
  if (use_sliced(f, n, evout)) return run_sliced(f, op, keys, n, flags, s);
  cudaError_t e = cudaSuccess;
  if (op == OP_CONTAINS) {
    e = f->ops->contains(f->d, keys, n, flags, s, f->timer);
  } else if (op == OP_REMOVE) {
    e = f->ops->remove(f->d, keys, n, flags, s, f->timer);
  } else {
    cf_status st = ensure_queue(f, n);
    if (st != CF_OK) return st;
    cfk::EvictMap em;
    st = evict_map_for(f, &em);
    if (st != CF_OK) return st;
    for (uint64_t off = 0; off < n && e == cudaSuccess; off += kInsertChunk) {
      const uint64_t len = (n - off) < kInsertChunk ? (n - off) : kInsertChunk;
      e = f->ops->insert_chunk(f->d, keys + off, uint32_t(len),
                               flags ? flags + off : nullptr,
                               evout ? evout + off : nullptr, f->queue, em, s,
                               f->timer);
    }
  }
  if (e != cudaSuccess) {
    set_err("kernel launch", e);
    return CF_ECUDA;
  }
  return CF_OK;
}

cf_status device_op(cf_filter* f, Op op, const uint64_t* keys, uint64_t n,
                    uint8_t* flags, uint32_t* evout, void* stream) {
  if (!f) return CF_EINVAL;
  if (n == 0) return CF_OK;
  if (!keys) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  st = run_op(f, op, keys, n, flags, evout, s);
  if (st != CF_OK) return st;
  return mark(f, s);
}

// Host-buffer forms.  Keys go through the kStageSlots staging slots in turn
// (stream s_in); a slot is reused once the kernels that read its previous
// chunk are done.  Flags are written to one of two device flag buffers
// (used in turn) and copied back in one piece per buffer fill (stream
// s_out); a buffer is reused once its previous copy is done.  Slots and
// buffers rotate across calls, so consecutive asynchronous calls overlap:
// the next call's key copies run while this call's kernels run.  At the
// end the caller's stream waits for the last flag copy, so the caller's
// stream completing means the flags are in host memory.

// One staging chunk of keys onto the device; returns its slot (the caller's
// stream waits for the copy).
cf_status stage_keys(cf_filter* f, const uint64_t* keys_h, uint64_t len, cudaStream_t s,
                     Stage** out) {
  Stage& sg = f->stage[f->next_slot];
  f->next_slot = (f->next_slot + 1) % cfk::kStageSlots;
  if (sg.used) CF_CUDA(cudaStreamWaitEvent(f->s_in, sg.comp_done, 0));
  if (f->timer) f->timer->begin(cfk::KK_H2D, f->s_in);
  CF_CUDA(cudaMemcpyAsync(sg.keys, keys_h, len * sizeof(uint64_t), cudaMemcpyHostToDevice,
                          f->s_in));
  if (f->timer) f->timer->end(cfk::KK_H2D, f->s_in);
  CF_CUDA(cudaEventRecord(sg.in_done, f->s_in));
  CF_CUDA(cudaStreamWaitEvent(s, sg.in_done, 0));
  *out = &sg;
  return CF_OK;
}

// The next flag buffer, once its previous copy to the host is done.
cfk::FlagGroup* take_group(cf_filter* f, cudaStream_t s) {
  cfk::FlagGroup* g = &f->fgroup[f->next_group];
  f->next_group ^= 1u;
  if (g->used) cudaStreamWaitEvent(s, g->out_done, 0);
  return g;
}

// Copy `bytes` of flags from a buffer to the host after the kernels so far.
cf_status flush_group(cf_filter* f, cfk::FlagGroup* g, uint8_t* dst_h, uint64_t bytes,
                      cudaStream_t s, cudaEvent_t* last_out) {
  CF_CUDA(cudaEventRecord(g->comp_done, s));
  CF_CUDA(cudaStreamWaitEvent(f->s_out, g->comp_done, 0));
  if (f->timer) f->timer->begin(cfk::KK_D2H, f->s_out);
  CF_CUDA(cudaMemcpyAsync(dst_h, g->flags, bytes, cudaMemcpyDeviceToHost, f->s_out));
  if (f->timer) f->timer->end(cfk::KK_D2H, f->s_out);
  CF_CUDA(cudaEventRecord(g->out_done, f->s_out));
  g->used = true;
  *last_out = g->out_done;
  return CF_OK;
}

// The device address at which kernels can read host keys in place: pinned
// host memory mapped into the device's address space; null for any other
// buffer (which takes the staged copies).
const uint64_t* host_keys_in_place(const uint64_t* keys_h) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, keys_h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer)
    return static_cast<const uint64_t*>(a.devicePointer);
  return nullptr;
}

// Sliced path: passes of up to the filter's pass size; each pass's keys
// arrive in staging chunks, each scattered as it lands, then the pass's
// bucket passes, eviction loop and result passes run once, and the pass's
// flags go back in one copy.
cf_status host_sliced(cf_filter* f, Op op, const uint64_t* keys_h, uint64_t n,
                      uint8_t* flags_h, cudaStream_t s, cudaEvent_t* last_out) {
  const uint64_t cap = slice_chunk(f);
  const uint64_t passes = (n + cap - 1) / cap;
  const uint64_t plen = (n + passes - 1) / passes;
  cf_status st = ensure_slice(f, plen);
  if (st != CF_OK) return st;
  cfk::EvictMap em;
  if (op == OP_INSERT) {
    st = ensure_queue(f, plen, kSliceChunkMax);
    if (st != CF_OK) return st;
    // The levels slow the host-to-device copies that run beside them
    // (measured on this path: 15-45% more copy time per step), which bound
    // these calls; automatic mode leaves them to device-buffer calls.
    st = evict_map_for(f, &em, f->lv_mode == 2 ? plen : 0);
    if (st != CF_OK) return st;
  }
  if (flags_h) {
    st = ensure_flag_groups(f, plen);
    if (st != CF_OK) return st;
  }
  const uint64_t chunk = f->stage_chunk;
  // In-place reads (cf_set_host_reads): the scatter reads the pass's keys
  // over the host link itself, with no copy engine and no staging.
  const uint64_t* kd = f->host_reads ? host_keys_in_place(keys_h) : nullptr;
  for (uint64_t p0 = 0; p0 < n; p0 += plen) {
    const uint64_t pl = (n - p0) < plen ? (n - p0) : plen;
    cudaError_t e = f->ops->sliced_begin(f->sb, s);
    if (kd && e == cudaSuccess)
      e = f->ops->sliced_scatter(f->d, kd + p0, pl, 0, flags_h != nullptr, f->sb, s, f->timer);
    for (uint64_t c0 = 0; !kd && c0 < pl && e == cudaSuccess; c0 += chunk) {
      const uint64_t len = (pl - c0) < chunk ? (pl - c0) : chunk;
      Stage* sg = nullptr;
      st = stage_keys(f, keys_h + p0 + c0, len, s, &sg);
      if (st != CF_OK) return st;
      e = f->ops->sliced_scatter(f->d, sg->keys, len, c0, flags_h != nullptr, f->sb, s,
                                 f->timer);
      if (e == cudaSuccess) e = cudaEventRecord(sg->comp_done, s);
      sg->used = true;
    }
    cfk::FlagGroup* g = flags_h ? take_group(f, s) : nullptr;
    if (e == cudaSuccess)
      e = f->ops->sliced_finish(f->d, int(op), pl, g ? g->flags : nullptr, f->sb, f->queue,
                                em, s, f->timer);
    if (e != cudaSuccess) {
      set_err("sliced kernel launch", e);
      return CF_ECUDA;
    }
    if (g) {
      st = flush_group(f, g, flags_h + p0, pl, s, last_out);
      if (st != CF_OK) return st;
    }
  }
  return CF_OK;
}

// Plain path: every staging chunk runs the single-filter kernels; the flags
// of group_chunks consecutive chunks share one buffer and one copy back.
cf_status host_chunked(cf_filter* f, Op op, const uint64_t* keys_h, uint64_t n,
                       uint8_t* flags_h, cudaStream_t s, cudaEvent_t* last_out) {
  const uint64_t chunk = f->stage_chunk;
  const uint64_t G = f->group_chunks;
  if (op == OP_INSERT) {
    cf_status st = ensure_queue(f, chunk);
    if (st != CF_OK) return st;
  }
  if (flags_h) {
    cf_status st = ensure_flag_groups(f, G * chunk);
    if (st != CF_OK) return st;
  }
  const uint64_t nchunks = (n + chunk - 1) / chunk;
  cfk::FlagGroup* g = nullptr;
  uint64_t g0 = 0;
  for (uint64_t c = 0; c < nchunks; ++c) {
    const uint64_t off = c * chunk;
    const uint64_t len = (n - off) < chunk ? (n - off) : chunk;
    Stage* sg = nullptr;
    cf_status st = stage_keys(f, keys_h + off, len, s, &sg);
    if (st != CF_OK) return st;
    if (flags_h && c % G == 0) {
      g = take_group(f, s);
      g0 = off;
    }
    st = run_op(f, op, sg->keys, len, g ? g->flags + (off - g0) : nullptr, nullptr, s);
    if (st != CF_OK) return st;
    CF_CUDA(cudaEventRecord(sg->comp_done, s));
    sg->used = true;
    if (g && (c % G == G - 1 || c == nchunks - 1)) {
      st = flush_group(f, g, flags_h + g0, off + len - g0, s, last_out);
      if (st != CF_OK) return st;
      g = nullptr;
    }
  }
  return CF_OK;
}

cf_status host_op(cf_filter* f, Op op, const uint64_t* keys_h, uint64_t n,
                  uint8_t* flags_h, void* stream, bool wait) {
  if (!f) return CF_EINVAL;
  if (n == 0) return CF_OK;
  if (!keys_h) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = ensure_staging(f);
  if (st != CF_OK) return st;
  st = order_on(f, s);
  if (st != CF_OK) return st;
  cudaEvent_t last_out = nullptr;
  st = use_sliced(f, n, nullptr) ? host_sliced(f, op, keys_h, n, flags_h, s, &last_out)
                                 : host_chunked(f, op, keys_h, n, flags_h, s, &last_out);
  if (st != CF_OK) return st;
  if (last_out) CF_CUDA(cudaStreamWaitEvent(s, last_out, 0));
  st = mark(f, s);
  if (st != CF_OK) return st;
  if (wait) CF_CUDA(cudaStreamSynchronize(s));
  return CF_OK;
}

void put32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
void put64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
uint32_t get32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
uint64_t get64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

constexpr uint32_t kSnapMagic = 0x31474643u;  // "CFG1"
constexpr size_t kSnapHdr = 64;

}  // namespace

extern "C" {

const char* cf_last_error(void) { return g_err; }

cf_status cf_set_kernel_timing(cf_filter* f, int enable) {
  if (!f) return CF_EINVAL;
  if (enable && !f->timer) f->timer = new cfk::FilterTimer();
  if (!enable && f->timer) {
    if (f->has_last) cudaEventSynchronize(f->ext_ev ? f->ext_ev : f->last_ev);
    delete f->timer;
    f->timer = nullptr;
  }
  return CF_OK;
}

cf_status cf_read_kernel_times(cf_filter* f, cf_kernel_times* out, int reset) {
  if (!f || !out) return CF_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (!f->timer) return CF_OK;
  for (auto& r : f->timer->recs) {
    CF_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    if (r.kind >= 0 && r.kind < cfk::KK_NUM) {
      out->launches[r.kind] += 1;
      out->ms[r.kind] += ms;
    }
  }
  if (reset) {
    for (auto& r : f->timer->recs) {
      f->timer->pool.push_back(r.a);
      f->timer->pool.push_back(r.b);
    }
    f->timer->recs.clear();
  }
  return CF_OK;
}

cf_status cf_set_slicing(cf_filter* f, int mode, uint64_t slice_bytes,
                         uint64_t max_chunk) {
  if (!f || mode < 0 || mode > 2) return CF_EINVAL;
  const uint64_t bb = uint64_t(f->cfg.slots_per_bucket) * f->cfg.fp_bits / 8;
  if (slice_bytes && slice_bytes < bb) return CF_EINVAL;
  if (max_chunk > kSliceChunkMax) return CF_EINVAL;
  // Scratch in use by queued work is freed only after that work.
  if (f->has_last) CF_CUDA(cudaEventSynchronize(f->ext_ev ? f->ext_ev : f->last_ev));
  f->slice_mode = mode;
  if (slice_bytes != f->slice_bytes || max_chunk != f->slice_chunk) free_slice(f);
  f->slice_bytes = slice_bytes;
  f->slice_chunk = max_chunk;
  return CF_OK;
}

cf_status cf_set_eviction_map(cf_filter* f, int mode, uint64_t min_queue) {
  if (!f || mode < 0 || mode > 2) return CF_EINVAL;
  f->map_mode = mode;
  f->map_min_queue = min_queue;
  return CF_OK;
}

cf_status cf_set_host_reads(cf_filter* f, int mode) {
  if (!f || mode < 0 || mode > 1) return CF_EINVAL;
  f->host_reads = mode;
  return CF_OK;
}

cf_status cf_set_eviction_levels(cf_filter* f, int mode, uint32_t n_levels,
                                 uint64_t min_queue, uint64_t stop_queue) {
  if (!f || mode < 0 || mode > 2 || n_levels > kLevelsMax) return CF_EINVAL;
  // Buffers in use by queued work are freed only after that work.
  if (f->has_last) CF_CUDA(cudaEventSynchronize(f->ext_ev ? f->ext_ev : f->last_ev));
  if (n_levels != f->lv_levels) free_levels(f);
  f->lv_mode = mode;
  f->lv_levels = n_levels;
  f->lv_min_queue = min_queue;
  f->lv_stop_queue = stop_queue;
  return CF_OK;
}

cf_status cf_debug_set_cas_limit(cf_filter* f, uint32_t limit) {
  if (!f || limit > cfk::kMaxCas) return CF_EINVAL;
  f->d.max_cas = limit ? limit : cfk::kMaxCas;
  return CF_OK;
}

int cf_version(void) { return 10200; }

const char* cf_status_str(cf_status s) {
  switch (s) {
    case CF_OK: return "ok";
    case CF_EINVAL: return "invalid argument";
    case CF_ENOMEM: return "out of memory";
    case CF_ECUDA: return "CUDA error";
    case CF_ETIMEOUT: return "timeout";
    case CF_ECONTENTION: return "contention";
    case CF_EBUSY: return "busy";
    case CF_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

size_t cf_table_bytes(uint64_t num_buckets, uint32_t fp_bits, uint32_t slots_per_bucket) {
  if (!(fp_bits == 8 || fp_bits == 16 || fp_bits == 32)) return 0;
  if (!(slots_per_bucket == 4 || slots_per_bucket == 8 || slots_per_bucket == 16)) return 0;
  if (num_buckets == 0 || num_buckets > (1ull << 32)) return 0;
  return size_t(num_buckets) * slots_per_bucket * fp_bits / 8;
}

size_t cf_required_bytes(const cf_config* cfg) {
  if (!valid_config(cfg)) return 0;
  return 256 + align256(size_t(victim_cap(cfg)) * sizeof(Victim)) +
         align256(table_bytes(cfg));
}

size_t cf_snapshot_bytes(const cf_filter* f) {
  return f ? kSnapHdr + table_bytes(&f->cfg) : 0;
}

cf_status cf_create_ex(const cf_config* cfg, cf_filter** out) {
  if (!out || !valid_config(cfg)) return CF_EINVAL;
  *out = nullptr;
  const size_t bytes = cf_required_bytes(cfg);
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    snprintf(g_err, sizeof g_err, "cudaMalloc of %zu bytes failed", bytes);
    return CF_ENOMEM;
  }
  cf_filter* f = new cf_filter();
  cf_status st = init_filter(f, cfg, mem, bytes, true);
  if (st != CF_OK) {
    cf_destroy(f);
    return st;
  }
  *out = f;
  return CF_OK;
}

cf_status cf_create(uint64_t num_buckets, uint32_t fp_bits,
                    uint32_t slots_per_bucket, uint32_t max_evictions,
                    cf_filter** out) {
  cf_config c{};
  c.num_buckets = num_buckets;
  c.fp_bits = fp_bits;
  c.slots_per_bucket = slots_per_bucket;
  c.max_evictions = max_evictions;
  c.policy = CF_POLICY_XOR;
  c.eviction = CF_EVICT_BFS;
  return cf_create_ex(&c, out);
}

cf_status cf_create_at(void* dev_mem, size_t bytes, const cf_config* cfg,
                       cf_filter** out) {
  if (!out || !dev_mem || !valid_config(cfg)) return CF_EINVAL;
  *out = nullptr;
  if (bytes < cf_required_bytes(cfg)) return CF_EINVAL;
  if (reinterpret_cast<uintptr_t>(dev_mem) & 255) return CF_EINVAL;
  cf_filter* f = new cf_filter();
  cf_status st = init_filter(f, cfg, static_cast<char*>(dev_mem),
                             cf_required_bytes(cfg), false);
  if (st != CF_OK) {
    cf_destroy(f);
    return st;
  }
  *out = f;
  return CF_OK;
}

cf_status cf_destroy(cf_filter* f) {
  if (!f) return CF_OK;
  if (f->has_last) cudaEventSynchronize(f->ext_ev ? f->ext_ev : f->last_ev);
  free_staging(f);
  if (f->queue) cudaFree(f->queue);
  if (f->fullmap) cudaFree(f->fullmap);
  free_levels(f);
  free_slice(f);
  if (f->last_ev) cudaEventDestroy(f->last_ev);
  delete f->timer;
  if (f->owns && f->mem) cudaFree(f->mem);
  delete f;
  return CF_OK;
}

cf_status cf_get_config(const cf_filter* f, cf_config* out) {
  if (!f || !out) return CF_EINVAL;
  *out = f->cfg;
  return CF_OK;
}

void* cf_table_ptr(const cf_filter* f) { return f ? f->d.table : nullptr; }

cf_status cf_insert(cf_filter* f, const uint64_t* keys, uint64_t n,
                    uint8_t* out_flags, void* stream) {
  return device_op(f, OP_INSERT, keys, n, out_flags, nullptr, stream);
}

cf_status cf_insert_ex(cf_filter* f, const uint64_t* keys, uint64_t n,
                       uint8_t* out_flags, uint32_t* evictions_out,
                       void* stream) {
  return device_op(f, OP_INSERT, keys, n, out_flags, evictions_out, stream);
}

cf_status cf_contains(cf_filter* f, const uint64_t* keys, uint64_t n,
                      uint8_t* out_flags, void* stream) {
  if (f && n && !out_flags) return CF_EINVAL;  // a query without output
  return device_op(f, OP_CONTAINS, keys, n, out_flags, nullptr, stream);
}

cf_status cf_remove(cf_filter* f, const uint64_t* keys, uint64_t n,
                    uint8_t* out_flags, void* stream) {
  return device_op(f, OP_REMOVE, keys, n, out_flags, nullptr, stream);
}

cf_status cf_insert_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream) {
  return host_op(f, OP_INSERT, keys_host, n, out_flags_host, stream, true);
}

cf_status cf_contains_host(cf_filter* f, const uint64_t* keys_host,
                           uint64_t n, uint8_t* out_flags_host, void* stream) {
  if (f && n && !out_flags_host) return CF_EINVAL;
  return host_op(f, OP_CONTAINS, keys_host, n, out_flags_host, stream, true);
}

cf_status cf_remove_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream) {
  return host_op(f, OP_REMOVE, keys_host, n, out_flags_host, stream, true);
}

cf_status cf_insert_host_async(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                               uint8_t* out_flags_host, void* stream) {
  return host_op(f, OP_INSERT, keys_host, n, out_flags_host, stream, false);
}

cf_status cf_contains_host_async(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                                 uint8_t* out_flags_host, void* stream) {
  if (f && n && !out_flags_host) return CF_EINVAL;
  return host_op(f, OP_CONTAINS, keys_host, n, out_flags_host, stream, false);
}

cf_status cf_remove_host_async(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                               uint8_t* out_flags_host, void* stream) {
  return host_op(f, OP_REMOVE, keys_host, n, out_flags_host, stream, false);
}

cf_status cf_set_staging_chunk(cf_filter* f, uint64_t keys_per_chunk) {
  if (!f || keys_per_chunk == 0 || keys_per_chunk > kInsertChunk)
    return CF_EINVAL;
  if (f->has_last) cudaEventSynchronize(f->ext_ev ? f->ext_ev : f->last_ev);
  free_staging(f);
  f->stage_chunk = keys_per_chunk;
  return CF_OK;
}

cf_status cf_clear(cf_filter* f, void* stream) {
  if (!f) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  CF_CUDA(cudaMemsetAsync(f->d.table, 0, table_bytes(&f->cfg), s));
  CF_CUDA(cudaMemsetAsync(f->d.ctrl, 0, sizeof(Ctrl), s));
  return mark(f, s);
}

cf_status cf_stats(cf_filter* f, cf_stats_t* out, void* stream) {
  if (!f || !out) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  Ctrl c;
  CF_CUDA(cudaMemcpyAsync(&c, f->d.ctrl, sizeof c, cudaMemcpyDeviceToHost, s));
  CF_CUDA(cudaStreamSynchronize(s));
  out->occupancy = c.occupancy;
  out->insert_ok = c.insert_ok;
  out->insert_fail = c.insert_fail;
  out->remove_ok = c.remove_ok;
  out->remove_fail = c.remove_fail;
  out->evictions = c.evictions;
  out->victims = c.victims;
  out->rollbacks = c.rollbacks;
  out->rollback_lost = c.rollback_lost;
  out->contention = c.contention;
  out->error_word = c.error_word;
  out->victim_capacity = f->d.victim_cap;
  out->map_builds = c.map_builds;
  for (int i = 0; i < 7; ++i) out->cas_retry[i] = c.cas_retry[i];
  out->debug_bad_index = c.debug_bad_index;
  out->level_passes = c.level_passes;
  out->level_steps = c.level_steps;
  out->level_runout = c.level_runout;
  return mark(f, s);
}

cf_status cf_victims(cf_filter* f, uint32_t* tags_host, uint64_t* buckets_host,
                     uint64_t max, uint64_t* count, void* stream) {
  if (!f) return CF_EINVAL;
  cf_stats_t stt;
  cf_status st = cf_stats(f, &stt, stream);
  if (st != CF_OK) return st;
  uint64_t logged = stt.victims < f->d.victim_cap ? stt.victims : f->d.victim_cap;
  if (count) *count = logged;
  uint64_t n = logged < max ? logged : max;
  if (n == 0) return CF_OK;
  Victim* tmp = static_cast<Victim*>(malloc(n * sizeof(Victim)));
  if (!tmp) return CF_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(tmp, f->d.victims, n * sizeof(Victim),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free(tmp);
    set_err("victims copy", e);
    return CF_ECUDA;
  }
  for (uint64_t i = 0; i < n; ++i) {
    if (tags_host) tags_host[i] = tmp[i].tag;
    if (buckets_host) buckets_host[i] = tmp[i].bucket;
  }
  free(tmp);
  return CF_OK;
}

cf_status cf_snapshot(cf_filter* f, void* dst, size_t bytes, int dst_is_device,
                      void* stream) {
  if (!f || !dst || bytes < cf_snapshot_bytes(f)) return CF_EINVAL;
  cf_stats_t stt;
  cf_status st = cf_stats(f, &stt, stream);
  if (st != CF_OK) return st;
  uint8_t hdr[kSnapHdr] = {0};
  put32(hdr + 0, kSnapMagic);
  put32(hdr + 4, 1);
  put64(hdr + 8, f->cfg.num_buckets);
  put32(hdr + 16, f->cfg.fp_bits);
  put32(hdr + 20, f->cfg.slots_per_bucket);
  put32(hdr + 24, f->cfg.max_evictions);
  put32(hdr + 28, f->cfg.policy);
  put64(hdr + 32, stt.occupancy);
  put64(hdr + 40, table_bytes(&f->cfg));
  put32(hdr + 48, 1);
  put32(hdr + 52, f->cfg.eviction);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* d8 = static_cast<uint8_t*>(dst);
  const cudaMemcpyKind k1 = dst_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  const cudaMemcpyKind k2 = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CF_CUDA(cudaMemcpyAsync(d8, hdr, kSnapHdr, k1, s));
  CF_CUDA(cudaMemcpyAsync(d8 + kSnapHdr, f->d.table, table_bytes(&f->cfg), k2, s));
  CF_CUDA(cudaStreamSynchronize(s));
  return mark(f, s);
}

cf_status cf_load(cf_filter* f, const void* src, size_t bytes,
                  int src_is_device, void* stream) {
  if (!f || !src || bytes < cf_snapshot_bytes(f)) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  uint8_t hdr[kSnapHdr];
  CF_CUDA(cudaMemcpyAsync(hdr, src, kSnapHdr,
                          src_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  CF_CUDA(cudaStreamSynchronize(s));
  if (get32(hdr) != kSnapMagic || get32(hdr + 4) != 1 ||
      get64(hdr + 8) != f->cfg.num_buckets || get32(hdr + 16) != f->cfg.fp_bits ||
      get32(hdr + 20) != f->cfg.slots_per_bucket || get32(hdr + 28) != f->cfg.policy ||
      get64(hdr + 40) != table_bytes(&f->cfg)) {
    snprintf(g_err, sizeof g_err, "snapshot header does not match the filter");
    return CF_EINVAL;
  }
  const uint8_t* s8 = static_cast<const uint8_t*>(src);
  CF_CUDA(cudaMemcpyAsync(f->d.table, s8 + kSnapHdr, table_bytes(&f->cfg),
                          src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CF_CUDA(cudaMemsetAsync(f->d.ctrl, 0, sizeof(Ctrl), s));
  cudaError_t e = f->ops->count(f->d, &f->d.ctrl->occupancy, s);
  if (e != cudaSuccess) {
    set_err("count kernel", e);
    return CF_ECUDA;
  }
  CF_CUDA(cudaStreamSynchronize(s));
  return mark(f, s);
}

cf_status cf_count_occupied(cf_filter* f, uint64_t* out, void* stream) {
  if (!f || !out) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  CF_CUDA(cudaMemsetAsync(&f->d.ctrl->scratch_count, 0, 8, s));
  cudaError_t e = f->ops->count(f->d, &f->d.ctrl->scratch_count, s);
  if (e != cudaSuccess) {
    set_err("count kernel", e);
    return CF_ECUDA;
  }
  unsigned long long v = 0;
  CF_CUDA(cudaMemcpyAsync(&v, &f->d.ctrl->scratch_count, 8, cudaMemcpyDeviceToHost, s));
  CF_CUDA(cudaStreamSynchronize(s));
  *out = v;
  return mark(f, s);
}

cf_status cf_hash_debug(const uint64_t* keys, uint64_t n, uint32_t fp_bits,
                        uint64_t num_buckets, uint32_t policy, uint32_t* fp,
                        uint64_t* i1, uint64_t* i2, void* stream) {
  cf_config c{};
  c.num_buckets = num_buckets;
  c.fp_bits = fp_bits;
  c.slots_per_bucket = 4;
  c.policy = policy;
  if (!valid_config(&c)) return CF_EINVAL;
  if (n == 0) return CF_OK;
  if (!keys) return CF_EINVAL;
  DevFilter d = make_dev(&c, nullptr);
  const cfk::Ops* ops = cfk::get_ops(int(fp_bits), 4, int(policy));
  if (!ops) return CF_ENOTSUP;
  cudaError_t e = ops->hash(d, keys, n, fp, i1, i2, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_err("hash kernel", e);
    return CF_ECUDA;
  }
  return CF_OK;
}

cf_status cf_debug_touch_bucket(cf_filter* f, uint64_t bucket, uint64_t* occupied,
                                void* stream) {
  if (!f) return CF_EINVAL;
#if !CF_DEBUG_BOUNDS
  // Without the kernels' own range check, an index beyond the table is
  // refused here: the kernel would read outside the allocation.
  if (bucket >= f->cfg.num_buckets) return CF_EINVAL;
#endif
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  CF_CUDA(cudaMemsetAsync(&f->d.ctrl->scratch_count, 0, 8, s));
  cudaError_t e = f->ops->touch(f->d, bucket, &f->d.ctrl->scratch_count, s);
  if (e != cudaSuccess) {
    set_err("touch kernel", e);
    return CF_ECUDA;
  }
  unsigned long long v = 0;
  CF_CUDA(cudaMemcpyAsync(&v, &f->d.ctrl->scratch_count, 8, cudaMemcpyDeviceToHost, s));
  CF_CUDA(cudaStreamSynchronize(s));
  if (occupied) *occupied = v;
  return mark(f, s);
}

int cf_debug_bounds_checked(void) { return CF_DEBUG_BOUNDS; }

cf_status cf_debug_insert_serial(cf_filter* f, const uint64_t* keys,
                                 uint64_t n, uint8_t* out_flags,
                                 uint32_t* evictions_out, void* stream) {
  if (!f) return CF_EINVAL;
  if (n == 0) return CF_OK;
  if (!keys) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_on(f, s);
  if (st != CF_OK) return st;
  // The serial kernel uses the full-bucket map when the filter's map mode
  // is "always" (and keeps it exact), so that the map-based BFS round can
  // be compared with the sequential oracle bit for bit.
  uint32_t* map = nullptr;
  if (f->map_mode == 2 && f->cfg.eviction == CF_EVICT_BFS) {
    st = ensure_map(f);
    if (st != CF_OK) return st;
    map = f->fullmap;
  }
  cudaError_t e = f->ops->insert_serial(f->d, keys, n, out_flags, evictions_out, map, s);
  if (e != cudaSuccess) {
    set_err("serial insert", e);
    return CF_ECUDA;
  }
  return mark(f, s);
}

}  // extern "C"
