/*
 * cf.h -- C ABI of the GB300 cuckoo filter library (libcf.so).
 *
 * A partial-key cuckoo filter ("Cuckoo-GPU: Accelerating Cuckoo Filters on
 * Modern GPUs", Dortmann, Vieth, Schmidt, 2026) for 64-bit keys, with the hot
 * path as hand-written sm_103a CUDA kernels:
 *   insert   -- Alg. 1 direct insertion + the BFS eviction of Sec. 4.6.1
 *               (or the greedy DFS chain of Alg. 1), lock-free CAS slots;
 *   contains -- Alg. 2, vector loads + SWAR compare, read-only;
 *   remove   -- Alg. 3, SWAR match + CAS to EMPTY.
 * Hashing follows Sec. 2.1 Eq. 1-3 and Sec. 4.3: h = XXH64(key, seed 0) over
 * the key's 8 little-endian bytes; fp = upper 32 bits masked to the
 * fingerprint width (0 mapped to 1, since 0 is EMPTY); i1 = lower 32 bits
 * mod m; XOR policy: i2 = i1 ^ (low 32 bits of XXH64(fp) mod m).
 *
 * Table layout (Sec. 4.2, Fig. 2): m buckets of b slots of f bits, stored as
 * m * (b*f/64) little-endian 64-bit words (one 32-bit word per bucket when
 * b*f == 32); slot s of bucket j is lane s mod (64/f) of word s div (64/f),
 * lane L at bits [L*f, L*f+f).  On a little-endian machine this is simply an
 * array of m*b f-bit integers.
 *
 * Conventions for every call:
 *  - Pointers named *_dev (and `keys`, `out_flags`, `dev_mem`, ...) are CUDA
 *    DEVICE pointers owned by the caller unless stated; *_host pointers are
 *    host memory (pinned memory gives copy/compute overlap).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Kernel work is enqueued asynchronously on it; results are
 *    valid once the stream has synchronised.  Calls documented as
 *    "synchronous" return after their work has completed.
 *  - Calls on one filter execute on the device in call order, even across
 *    streams: a call made on a different stream than the previous call on
 *    that filter first waits (cudaStreamWaitEvent) for the previous call.
 *    This enforces the rule that a query never overlaps an insert or a
 *    delete (Sec. 4.4: the non-coherent vector loads could see torn words).
 *  - Per-key flags (uint8): CF_FLAG_OK = inserted / found / removed;
 *    CF_FLAG_FAIL = insert gave up after max_evictions / absent / not
 *    removed; CF_FLAG_CONTENTION = a bounded CAS retry loop ran out (never
 *    expected; counted in cf_stats_t.contention).  out_flags may be NULL.
 *  - n == 0 is a no-op returning CF_OK.  Errors never leave a kernel
 *    running: validation happens on the host before any launch.
 *  - Not thread-safe per filter: one host thread at a time per cf_filter.
 */
#ifndef CF_H
#define CF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cf_filter cf_filter;

typedef enum {
  CF_OK = 0,
  CF_EINVAL = 1,       /* bad parameter, size or buffer                     */
  CF_ENOMEM = 2,       /* device/host allocation failed, or budget exceeded */
  CF_ECUDA = 3,        /* a CUDA runtime call failed                        */
  CF_ETIMEOUT = 4,     /* a watchdog deadline passed (serving loop)         */
  CF_ECONTENTION = 5,  /* reserved: per-key contention is reported in flags */
  CF_EBUSY = 6,        /* the object is in use (e.g. a pool slot)           */
  CF_ENOTSUP = 7       /* parameter combination not compiled in             */
} cf_status;

enum { CF_POLICY_XOR = 0, CF_POLICY_OFFSET = 1 };
enum { CF_EVICT_BFS = 0, CF_EVICT_DFS = 1 };
enum { CF_FLAG_FAIL = 0, CF_FLAG_OK = 1, CF_FLAG_CONTENTION = 2 };

/* Filter parameters.
 *  num_buckets      m.  XOR policy: a power of two, 1 <= m <= 2^32 (the XOR
 *                   of Eq. 3 needs a power of two, Sec. 4.6.2; i1 has 32
 *                   bits, Sec. 4.3).  Offset policy: 2 <= m < 2^32.
 *  fp_bits          f in {8, 16, 32} (Sec. 6: hardware-friendly widths).
 *  slots_per_bucket b in {4, 8, 16}.
 *  max_evictions    bound of the eviction loop (Alg. 1 "maxEvictions");
 *                   0 disables eviction.
 *  policy           CF_POLICY_XOR (Eq. 3) or CF_POLICY_OFFSET (Sec. 4.6.2:
 *                   the top tag bit is a choice bit, offset(fp) in [1,m-1]).
 *  eviction         CF_EVICT_BFS (Sec. 4.6.1) or CF_EVICT_DFS (Alg. 1).
 *  victim_capacity  entries of the device victim log (0 -> 4096).  A failed
 *                   insert drops one tag ("table too full", Alg. 1); the log
 *                   keeps the first victim_capacity of them. */
typedef struct {
  uint64_t num_buckets;
  uint32_t fp_bits;
  uint32_t slots_per_bucket;
  uint32_t max_evictions;
  uint32_t policy;
  uint32_t eviction;
  uint32_t victim_capacity;
} cf_config;

/* Device counters, read by cf_stats (all cumulative since create/clear). */
typedef struct {
  uint64_t occupancy;      /* stored tags                                   */
  uint64_t insert_ok;
  uint64_t insert_fail;    /* includes contention failures                  */
  uint64_t remove_ok;
  uint64_t remove_fail;
  uint64_t evictions;      /* slot overwrites inside eviction loops         */
  uint64_t victims;        /* tags dropped (may exceed the log capacity)    */
  uint64_t rollbacks;      /* BFS relocations undone after a lost CAS       */
  uint64_t rollback_lost;  /* rollbacks whose copy was already gone         */
  uint64_t contention;     /* bounded CAS loops that ran out                */
  uint32_t error_word;     /* bit 0: contention; bit 1: victim log full     */
  uint32_t victim_capacity;
} cf_stats_t;

/* ---- sizes ------------------------------------------------------------- */
/* Bytes of the raw table: m * b * f / 8.  0 if the config is invalid. */
size_t cf_table_bytes(const cf_config* cfg);
/* Bytes of device memory a filter needs (control block + victim log +
 * table, 256-byte aligned pieces).  0 if the config is invalid. */
size_t cf_required_bytes(const cf_config* cfg);
/* Bytes of a snapshot: 64-byte header + table. */
size_t cf_snapshot_bytes(const cf_filter* f);

/* ---- lifetime ----------------------------------------------------------- */
/* cf_create: the library cudaMalloc's cf_required_bytes and zeroes it
 * (synchronous).  Uses XOR + BFS with the default victim log.
 * Errors: CF_EINVAL (parameters), CF_ENOMEM, CF_ECUDA. */
cf_status cf_create(uint64_t num_buckets, uint32_t fp_bits,
                    uint32_t slots_per_bucket, uint32_t max_evictions,
                    cf_filter** out);
cf_status cf_create_ex(const cf_config* cfg, cf_filter** out);
/* cf_create_at: build a filter inside caller-owned device memory of at
 * least cf_required_bytes(cfg) bytes, 256-byte aligned (e.g. a torch
 * tensor).  The memory is zeroed (synchronous) and must outlive the filter;
 * cf_destroy does not free it. */
cf_status cf_create_at(void* dev_mem, size_t bytes, const cf_config* cfg,
                       cf_filter** out);
/* Waits for the filter's outstanding work, then frees what the library
 * allocated.  NULL is accepted. */
cf_status cf_destroy(cf_filter* f);
cf_status cf_get_config(const cf_filter* f, cf_config* out);
/* Device address of the raw table (for tests and zero-copy inspection). */
void* cf_table_ptr(const cf_filter* f);

/* ---- the hot path (asynchronous on `stream`) ---------------------------- */
/* Insert keys[0..n) (Alg. 1 + Sec. 4.6.1).  Placement under concurrency is
 * nondeterministic; each key ends with flag OK, or FAIL with one victim
 * logged.  evictions_out (may be NULL): per-key eviction-loop overwrites. */
cf_status cf_insert(cf_filter* f, const uint64_t* keys, uint64_t n,
                    uint8_t* out_flags, void* stream);
cf_status cf_insert_ex(cf_filter* f, const uint64_t* keys, uint64_t n,
                       uint8_t* out_flags, uint32_t* evictions_out,
                       void* stream);
/* Membership of keys[0..n) (Alg. 2).  Read-only; bit-exact. */
cf_status cf_contains(cf_filter* f, const uint64_t* keys, uint64_t n,
                      uint8_t* out_flags, void* stream);
/* Delete keys[0..n) (Alg. 3): clears one matching tag from i1, else i2. */
cf_status cf_remove(cf_filter* f, const uint64_t* keys, uint64_t n,
                    uint8_t* out_flags, void* stream);
/* Zero the table and all counters (asynchronous). */
cf_status cf_clear(cf_filter* f, void* stream);

/* Same three operations on HOST buffers: keys are streamed to the device in
 * chunks through library-owned staging buffers, flags are streamed back.
 * Synchronous (returns when out_flags_host is filled).  Host buffers should
 * be pinned (cudaHostRegister / torch pin_memory) for overlap. */
cf_status cf_insert_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream);
cf_status cf_contains_host(cf_filter* f, const uint64_t* keys_host,
                           uint64_t n, uint8_t* out_flags_host, void* stream);
cf_status cf_remove_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream);
/* Keys per staging chunk for the *_host calls (default 2^24). */
cf_status cf_set_staging_chunk(cf_filter* f, uint64_t keys_per_chunk);

/* ---- state, stats, snapshots (synchronous) ------------------------------ */
cf_status cf_stats(cf_filter* f, cf_stats_t* out, void* stream);
/* Copy the first min(max, logged) victims (tag, bucket) to host arrays;
 * *count receives the number logged (capped at the capacity). */
cf_status cf_victims(cf_filter* f, uint32_t* tags_host, uint64_t* buckets_host,
                     uint64_t max, uint64_t* count, void* stream);
/* Snapshot = 64-byte little-endian header (magic "CFG1", version 1, m, f,
 * b, max_evictions, policy, occupancy, table bytes, hash id 1, eviction)
 * followed by the raw table.  dst/src may be host (is_device = 0) or
 * device (is_device = 1) memory of at least cf_snapshot_bytes bytes.
 * cf_load checks that the header matches the filter's parameters
 * (CF_EINVAL otherwise), copies the table, recounts occupancy on the device
 * and resets the other counters and the victim log. */
cf_status cf_snapshot(cf_filter* f, void* dst, size_t bytes, int dst_is_device,
                      void* stream);
cf_status cf_load(cf_filter* f, const void* src, size_t bytes,
                  int src_is_device, void* stream);
/* Count nonzero slots of the table on the device (synchronous). */
cf_status cf_count_occupied(cf_filter* f, uint64_t* out, void* stream);

/* ---- test exports ------------------------------------------------------- */
/* fp / i1 / i2 of keys[0..n) (device arrays) for the given parameters
 * (Eq. 1-3, Sec. 4.3).  Asynchronous. */
cf_status cf_hash_debug(const uint64_t* keys, uint64_t n, uint32_t fp_bits,
                        uint64_t num_buckets, uint32_t policy, uint32_t* fp,
                        uint64_t* i1, uint64_t* i2, void* stream);
/* The same insert algorithm run by ONE GPU thread over the keys in order,
 * so that placement is deterministic (matches a sequential
 * implementation bit for bit).  For tests only; slow. */
cf_status cf_debug_insert_serial(cf_filter* f, const uint64_t* keys,
                                 uint64_t n, uint8_t* out_flags,
                                 uint32_t* evictions_out, void* stream);

/* ---- insert without device allocation ------------------------------------
 * The paper has no counterpart to this entry point.
 *
 * cf_insert keeps a work queue of 4 bytes per key in device memory that the
 * library cudaMalloc's on a filter's first large insert (and reuses after).
 * Some callers cannot allow a device allocation there: code whose device
 * memory is all handed out by another allocator or a fixed-size arena,
 * code on a path that must not stall on cudaMalloc's implicit device
 * synchronisation, and code that must not fail with out-of-memory halfway
 * through a batch.  cf_insert_noalloc does exactly the insert of cf_insert
 * (same kernels, same results and flags) with its queue in a fixed array
 * compiled into the library: a file-scope __device__ array of
 * CF_NOALLOC_MAX_KEYS entries (4 MiB), which every GPU that loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or other device-allocating routine.  Keys and flags are still the
 * caller's; build the filter with cf_create_at to keep the whole path free
 * of library allocations.
 *  - n > CF_NOALLOC_MAX_KEYS returns CF_EINVAL (split larger batches).
 *  - The filter's device must be the current device (CF_EINVAL otherwise).
 *    The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress; make that first call before any stream capture.
 *  - Every call shares the one array: calls whose GPU work overlaps (on
 *    streams not ordered with each other, on any filters) race and corrupt
 *    each other's results.  Issue them on one stream or order the streams.
 *  - The array keeps the previous call's entries.  None of it has to start
 *    at zero: each entry is written before it is read, and the entry count
 *    lives in the filter's control block. */
#define CF_NOALLOC_MAX_KEYS (1u << 20)
cf_status cf_insert_noalloc(cf_filter* f, const uint64_t* keys, uint64_t n,
                            uint8_t* out_flags, void* stream);

/* ---- measurement helpers ------------------------------------------------ */
/* Random-gather ceiling: n_access independent loads of access_bytes (8, 16
 * or 32) at pseudo-random aligned offsets within the first power-of-two
 * part of the device buffer `buf` (32-byte aligned), with the load
 * instructions of the query kernel, loads_per_thread (4, 8 or 16) in
 * flight per thread.  Asynchronous; `sink` is a device uint64 the kernel
 * may write.  Time it with events on `stream` to get random loads/s. */
cf_status cf_probe_gather(const void* buf, uint64_t bytes, uint64_t n_access,
                          uint32_t access_bytes, uint32_t loads_per_thread,
                          uint64_t seed, unsigned long long* sink,
                          void* stream);
/* The CUDA context limit cudaLimitMaxL2FetchGranularity of the current
 * device (0..128 bytes): how much L2 fetches from DRAM around a missed
 * sector.  Random bucket probes use one 32-byte sector; a larger fetch
 * moves bytes nobody reads.  Process-wide for the current context; it
 * does not outlive the process. */
cf_status cf_set_l2_fetch_granularity(uint32_t bytes);
cf_status cf_get_l2_fetch_granularity(uint32_t* bytes);

const char* cf_status_str(cf_status s);
/* Text of the last error seen by a cf_* call on this host thread. */
const char* cf_last_error(void);
/* Library version (major * 10000 + minor * 100 + patch). */
int cf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CF_H */
