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
  uint64_t rollbacks;      /* undone BFS moves: always 0 (a move swaps the
                              new tag in first, so nothing is ever undone) */
  uint64_t rollback_lost;  /* always 0, as rollbacks                        */
  uint64_t contention;     /* bounded CAS loops that ran out                */
  uint32_t error_word;     /* bit 0: contention; bit 1: victim log full;
                              bit 2: an asynchronous copy of the sliced
                              path timed out (its records were skipped);
                              bit 3: (bounds-checked build only) a bucket
                              index was out of range, see debug_bad_index */
  uint32_t victim_capacity;
  uint64_t map_builds;     /* eviction launches that built and used the
                              full-bucket map (cf_set_eviction_map)        */
  uint64_t cas_retry[7];   /* CAS-retry histogram: failed CAS attempts by
                              retry depth within one retry loop, bins 0, 1,
                              2-3, 4-7, 8-15, 16-63, >= 64 (bin 0: a loop's
                              first attempt failed; bin k counts loops that
                              needed more retries than bins below k allow) */
  uint64_t debug_bad_index;/* bounds-checked build: first out-of-range
                              bucket index + 1; 0 if none (always 0 in the
                              normal build, which does not check)          */
  uint64_t level_passes;   /* slice-grouped eviction levels that ran
                              (cf_set_eviction_levels)                     */
  uint64_t level_steps;    /* chain steps those levels took                */
  uint64_t level_runout;   /* chains run to their end at once for want of
                              room in a level's record buffer             */
} cf_stats_t;

/* ---- sizes ------------------------------------------------------------- */
/* Bytes of the raw table (Sec. 4.2: m buckets of b tags of f bits, packed):
 * m * b * f / 8.  0 unless f is 8, 16 or 32, b is 4, 8 or 16 and
 * 1 <= m <= 2^32 (the bucket policy's own rule on m is checked at create). */
size_t cf_table_bytes(uint64_t num_buckets, uint32_t fp_bits, uint32_t slots_per_bucket);
/* Bytes of device memory a filter needs (control block + victim log +
 * table, 256-byte aligned pieces).  0 if the config is invalid. */
size_t cf_required_bytes(const cf_config* cfg);
/* Bytes of a snapshot: 64-byte header + table. */
size_t cf_snapshot_bytes(const cf_filter* f);

/* ---- lifetime ----------------------------------------------------------- */
/* Sec. 4.7 describes a C-style interface over raw device pointers and batch
 * lengths, with the parameters fixed per filter (there as compile-time
 * template constants; here runtime arguments dispatched to the compiled
 * instances, f x b x policy).  The calls below are that interface.
 * cf_create: the library cudaMalloc's cf_required_bytes and zeroes it
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
/* Zero the table and all counters (asynchronous; Sec. 4.7 interface: the
 * paper's filter is rebuilt by the caller after an insert failure, Alg. 1). */
cf_status cf_clear(cf_filter* f, void* stream);

/* Same three operations on HOST buffers: keys are streamed to the device in
 * chunks through library-owned staging buffers (four slots of keys, so
 * that copies of later chunks overlap the kernels of earlier ones); flags
 * are gathered on the device and copied back in pieces of about 256 MiB
 * (two alternating device buffers).
 * Synchronous (returns when out_flags_host is filled).  Host buffers should
 * be pinned (cudaHostRegister / torch pin_memory) for overlap. */
cf_status cf_insert_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream);
cf_status cf_contains_host(cf_filter* f, const uint64_t* keys_host,
                           uint64_t n, uint8_t* out_flags_host, void* stream);
cf_status cf_remove_host(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                         uint8_t* out_flags_host, void* stream);
/* The same three calls, asynchronous: they enqueue the copies and kernels
 * and return.  The flags are in out_flags_host once `stream` has
 * synchronised (the stream waits for the last flag copy); keys_host must
 * stay valid, and out_flags_host untouched, until then.  Consecutive calls
 * on a filter overlap on the device (the next call's key copies run while
 * the previous call's kernels run); they still execute in call order.
 * When a call takes the slice-partitioned path (cf_set_slicing), each pass
 * of up to the pass size gathers its keys staging chunk by staging chunk,
 * so the pass size, not the staging chunk, sets how often the table is
 * swept. */
cf_status cf_insert_host_async(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                               uint8_t* out_flags_host, void* stream);
cf_status cf_contains_host_async(cf_filter* f, const uint64_t* keys_host,
                                 uint64_t n, uint8_t* out_flags_host, void* stream);
cf_status cf_remove_host_async(cf_filter* f, const uint64_t* keys_host, uint64_t n,
                               uint8_t* out_flags_host, void* stream);
/* Keys per staging chunk for the *_host calls (default 2^24; the library
 * keeps eight chunks of keys and two flag buffers of at least 256 MiB or a
 * sliced pass).  Waits for the filter's queued work. */
cf_status cf_set_staging_chunk(cf_filter* f, uint64_t keys_per_chunk);
/* How the sliced passes of the *_host calls get their keys: mode 0 (the
 * default) copies them to the device in staging chunks on a copy stream;
 * mode 1 lets the pass's scatter kernel read them in place over the host
 * link when the key buffer is pinned host memory mapped into the device's
 * address space (other buffers keep the copies).  The copies overlap the
 * previous work, but run slower beside the inserts' and deletes' CAS
 * kernels (measured: 211 GB/s alone or beside queries, 124 GB/s beside
 * inserts and deletes); in-place reads overlap nothing and always run at
 * the link's rate.  Flags still come back by copies.  CF_EINVAL for a bad
 * mode. */
cf_status cf_set_host_reads(cf_filter* f, int mode);

/* Slice-partitioned execution of cf_insert / cf_contains / cf_remove (and of
 * each staging chunk of the *_host calls).  The paper's kernels have no
 * counterpart: they give every key one thread and let it touch its buckets in
 * batch order.  Here a batch is grouped by the table slice of each key's
 * primary bucket and processed slice by slice, so that bucket accesses hit
 * L2; keys left pending (not found / not removed / bucket full) are grouped
 * by the slice of their alternate bucket and processed again; the insert's
 * eviction loop (Sec. 4.6.1) then runs on the keys whose two buckets were
 * full.  Each key follows Alg. 1 / 2 / 3 exactly as on the plain path; only
 * the interleaving of keys differs, so query flags are identical and insert
 * / delete results satisfy the same invariants (which keys win a contended
 * bucket may differ, as between any two concurrent runs).
 *  - mode: 0 never, 1 automatic (the default: tables of at least 256 MiB and
 *    batches of at least num_buckets / 8 keys), 2 always.
 *  - slice_bytes: table bytes per slice, rounded down to a power-of-two
 *    number of buckets (0: 32 MiB).  At most 1024 slices: larger tables get
 *    larger slices.  CF_EINVAL if smaller than one bucket.
 *  - max_chunk: keys per sliced pass (0: 2^28, at most 2^30, CF_EINVAL
 *    above).  Larger batches run as consecutive passes.
 *  - Scratch: about 48 bytes per key of a pass (its largest pass so far),
 *    allocated by the library on the first sliced call and freed by
 *    cf_destroy or by a change of slice_bytes / max_chunk.  CF_ENOMEM if it
 *    cannot be allocated.
 *  - Calls that ask for per-key eviction counts (cf_insert_ex with
 *    out_evictions) take the plain path.
 * Waits for the filter's queued work before changing the settings. */
cf_status cf_set_slicing(cf_filter* f, int mode, uint64_t slice_bytes,
                         uint64_t max_chunk);

/* Full-bucket map of the insert's eviction loop.  The BFS heuristic of
 * Sec. 4.6.1 asks, for each of b/2 candidates, whether the candidate's
 * alternate bucket has an empty slot.  On a table L2 cannot hold, asking the
 * bucket is a random DRAM access per candidate.  With the map, one bit per
 * bucket (m/8 bytes, allocated by the library on first use, freed by
 * cf_destroy) answers instead: it is built from the table by one pass
 * before the eviction kernel, and the eviction rounds set the bit of every
 * bucket they fill or find full.  During an insert a full bucket stays full,
 * so a set bit is always right; a clear bit that has gone stale costs one
 * failed insert attempt, after which the chain goes on from that bucket as
 * it would had a concurrent insert taken the room.  Every key still follows
 * Alg. 1 and Sec. 4.6.1, and a single thread (cf_debug_insert_serial) takes
 * exactly the same steps with or without the map.
 *  - mode: 0 never; 1 automatic (the default): BFS filters whose table is
 *    larger than 64 MiB; 2 always (BFS filters).
 *  - min_queue: the map is built and used only for eviction queues of at
 *    least this many keys (0: m/16 in automatic mode, every queue in mode
 *    2); smaller queues probe the buckets.
 *  - cf_debug_insert_serial uses (and keeps exact) the map in mode 2.
 * CF_EINVAL for a bad mode.  Takes effect with the next insert call. */
cf_status cf_set_eviction_map(cf_filter* f, int mode, uint64_t min_queue);

/* Slice-grouped eviction levels of the sliced insert (Alg. 1 phase 2 with
 * the BFS heuristic of Sec. 4.6.1, run level by level).  Instead of walking
 * each key's eviction chain to its end (a random DRAM access per round on a
 * table L2 cannot hold), every chain advances one step per level and a
 * level's steps are grouped by the table slice of the bucket they touch, as
 * the bucket passes group keys, so they hit L2.  A step: place the tag in
 * hand into its bucket if it has an empty slot; else give up after
 * max_evictions overwrites; else choose a candidate as the BFS heuristic
 * does (asking the full-bucket map) and swap the tag in.  Each chain takes
 * the same steps and random draws as in the eviction loop; only the
 * interleaving of chains changes.
 * Used for sliced inserts (cf_set_slicing) of BFS filters when the
 * full-bucket map is (cf_set_eviction_map), for passes whose eviction queue
 * holds at least min_queue keys (0: 2^20) and at most half the pass; after
 * n_levels levels (0: 12), or once a level would have fewer than stop_queue
 * chains (0: 2^18), the remaining chains run to their end as in the loop.
 * The library allocates two record buffers of about 12 bytes per key of a
 * pass each on first use (freed by cf_destroy, or here when n_levels
 * changes); if that allocation fails, the insert runs the loop instead.
 * mode: 0 off; 1 (the default) for inserts of device buffers into filters
 * with buckets of at most 8 bytes: beside the host-buffer calls' copies
 * the levels slow those copies more than they save (measured: 15-45% more
 * copy time per step of the large workload), and with wider buckets they
 * measured slower than the loop (f16 b16 fill to LF 0.95 on 2^28 slots:
 * 21.7 against 23.9 G inserts/s); 2 for every sliced insert.
 * CF_EINVAL for a bad mode or n_levels > 256.  Waits for the filter's
 * queued work; takes effect with the next insert call. */
cf_status cf_set_eviction_levels(cf_filter* f, int mode, uint32_t n_levels,
                                 uint64_t min_queue, uint64_t stop_queue);

/* ---- state, stats, snapshots (synchronous) ------------------------------ */
/* Counters of the filter (Sec. 4.3: the occupancy count kept by the
 * insert's hierarchical reduction; Sec. 4.7 interface).  Syncs `stream`. */
cf_status cf_stats(cf_filter* f, cf_stats_t* out, void* stream);
/* Copy the first min(max, logged) victims (tag, bucket) to host arrays;
 * *count receives the number logged (capped at the capacity). */
cf_status cf_victims(cf_filter* f, uint32_t* tags_host, uint64_t* buckets_host,
                     uint64_t max, uint64_t* count, void* stream);
/* Snapshot and restore of the table of Sec. 4.2 (Sec. 4.7 interface; the
 * paper has no file format, this one is the library's own).
 * Snapshot = 64-byte little-endian header (magic "CFG1", version 1, m, f,
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
/* Bound of every CAS retry loop of the filter's kernels (attempts on one
 * word before the key is given up with CF_FLAG_CONTENTION): 1 .. 4096, 0
 * restores the default 4096; CF_EINVAL above 4096.  Lowering it makes the
 * bounded loops run out under ordinary contention, so that tests can reach
 * the contention path (flags, counter, victim, error-word bit 0) without
 * any kernel waiting unboundedly.  Applies to calls made after it. */
cf_status cf_debug_set_cas_limit(cf_filter* f, uint32_t limit);
/* 1 if this build of the library range-checks every bucket index on the
 * device (libcf_debug.so, built with -DCF_DEBUG_BOUNDS=1), else 0.  In a
 * checked build an out-of-range index never reaches memory: bucket 0 is
 * used instead, error-word bit 3 is set and the first such index is kept
 * (cf_stats_t.debug_bad_index). */
int cf_debug_bounds_checked(void);
/* Test export: load bucket `bucket` on the device (through the same bucket
 * addressing as the kernels) and return its number of occupied slots in
 * *occupied (may be NULL).  Synchronous.  The normal build returns
 * CF_EINVAL for bucket >= num_buckets; the checked build lets the kernel's
 * own check catch it (the way to test that check). */
cf_status cf_debug_touch_bucket(cf_filter* f, uint64_t bucket, uint64_t* occupied,
                                void* stream);

/* ---- multi-filter launch --------------------------------------------------
 * Many filters' insert / query / delete batches in ONE persistent kernel
 * (plus one eviction kernel over the inserts' combined eviction queue):
 * warps take 32*K-key tiles of all items from a device counter, so items of
 * very different sizes keep every SM busy and no host loop launches per
 * filter.  The algorithms per key are those of cf_insert / cf_contains /
 * cf_remove (Alg. 1-3, Sec. 4.6.1), with the same results and flags.
 *
 * Rules for one batch (CF_EINVAL otherwise):
 *  - all filters share fp_bits, slots_per_bucket and policy;
 *  - a filter may appear in several items, but either only in queries or
 *    only in inserts/removes (a query must not overlap a mutation, Sec. 4.4);
 *  - n < 2^32 per item, sum of n <= max_keys, n_items <= max_items;
 *  - out_flags is required for CF_OP_CONTAINS (device, n bytes).
 * Ordering: the launch waits for each filter's previous work on other
 * streams, and later calls on those filters wait for the batch. */
typedef struct cf_batch cf_batch;
enum { CF_OP_INSERT = 0, CF_OP_CONTAINS = 1, CF_OP_REMOVE = 2 };
typedef struct {
  cf_filter* filter;
  const uint64_t* keys;  /* device */
  uint64_t n;
  uint8_t* out_flags;    /* device, may be NULL except for CF_OP_CONTAINS */
  uint32_t op;
  uint32_t reserved;
} cf_batch_item;
/* One configuration of the batched kernels (see cf_batch_autotune). */
typedef struct {
  uint32_t variant;          /* index in the geometry's variant list       */
  uint32_t keys_per_thread;  /* K: keys a thread handles per tile          */
  uint32_t block;            /* threads per block of the tile kernel       */
  uint32_t frontier;         /* BFS candidates whose alternate buckets are
                                probed together (1 .. b/2)                 */
  float ms;                  /* launch time measured by the autotuner      */
} cf_tuning;

/* A reusable plan: device descriptor buffer, pinned host staging and an
 * eviction queue of max_keys entries (8 bytes each).  Allocates. */
cf_status cf_batch_create(uint32_t max_items, uint64_t max_keys,
                          cf_batch** out);
/* Waits for the plan's outstanding work and frees it.  NULL accepted. */
cf_status cf_batch_destroy(cf_batch* b);
/* Stage items (host work only; waits if the previous launch's upload has
 * not run yet).  Picks the variant cached for this batch's class if the
 * autotuner has seen one, else the pinned variant, else the default. */
cf_status cf_batch_set(cf_batch* b, const cf_batch_item* items,
                       uint32_t n_items);
/* Enqueue the staged batch on `stream`: descriptor upload (H2D from the
 * pinned staging), the tile kernel, the eviction kernel if any item
 * inserts.  Asynchronous. */
cf_status cf_batch_launch(cf_batch* b, void* stream);
/* The same work as one CUDA-graph launch: captured on first use for the
 * current variant, replayed afterwards (new items via cf_batch_set). */
cf_status cf_batch_graph_launch(cf_batch* b, void* stream);
/* Time every variant of the staged batch's geometry on the staged batch
 * itself (the filters' device state is saved before and restored after
 * each trial, so the batch's effect is not applied), keep the fastest for
 * this plan and for later batches of the same class (geometry, ops, size
 * class).  Synchronous; needs scratch memory of the filters' size. */
cf_status cf_batch_autotune(cf_batch* b, void* stream, cf_tuning* chosen);
cf_status cf_batch_set_variant(cf_batch* b, uint32_t variant);
cf_status cf_batch_get_tuning(const cf_batch* b, cf_tuning* out);
/* Number of variants for the staged batch's geometry (0 if none staged). */
uint32_t cf_batch_variant_count(const cf_batch* b);

/* ---- serving loop with continuous batching -------------------------------
 * A server owns many live filters (all device-resident) and a scheduler
 * thread.  Clients submit requests (filter, op, device keys, device flags)
 * at any time.  The scheduler keeps up to max_inflight waves on the GPU,
 * each wave one multi-filter launch (cf_batch) on its own stream: as soon
 * as a wave slot frees up it takes the waiting requests of every filter
 * that has no work in flight, so requests that arrive while others run are
 * admitted as slots free up and their work overlaps on the device.
 * Per filter, requests run in submission order (a filter is in at most one
 * wave at a time; consecutive requests of the same kind may share a wave),
 * so a query never overlaps a mutation of its filter (Sec. 4.4).
 * New filters are admitted against an HBM budget: a filter that does not
 * fit waits (its requests queue) until removed filters free enough.
 * Thread safety: submit / add / remove / poll / drain may be called from
 * any host thread. */
typedef struct cf_server cf_server;
typedef struct {
  uint64_t hbm_budget_bytes;  /* sum of cf_required_bytes of live filters   */
  uint32_t max_inflight;      /* waves on the GPU at once (streams), >= 1   */
  uint32_t max_wave_items;    /* requests per wave                          */
  uint64_t max_wave_keys;     /* keys per wave; also the largest request    */
  uint32_t use_graphs;        /* replay each wave slot's launch as a graph  */
  uint32_t watchdog_us;       /* a wave running longer (launch to observed
                                 completion, microseconds) is "late": its
                                 requests complete with CF_ETIMEOUT (their
                                 results are still written); 0 = off        */
} cf_server_config;
typedef struct {
  uint32_t filter_id;
  uint32_t op;              /* CF_OP_INSERT / CF_OP_CONTAINS / CF_OP_REMOVE */
  const uint64_t* keys;     /* device, valid until the request completes   */
  uint64_t n;
  uint8_t* out_flags;       /* device; required for CF_OP_CONTAINS          */
  uint64_t tag;             /* returned in the completion                   */
} cf_request;
typedef struct {
  uint64_t request_id;
  uint64_t tag;
  int32_t status;           /* CF_OK, or CF_ETIMEOUT for a late wave        */
  uint32_t wave_size;       /* requests in the wave that ran this one       */
  double submit_s;          /* host steady-clock seconds                    */
  double launch_s;
  double done_s;            /* when the scheduler saw the wave complete     */
} cf_completion;
typedef struct {
  uint64_t submitted, completed, waves, late_waves;
  uint64_t keys_completed;
  uint64_t used_bytes;      /* HBM held by live filters                     */
  uint32_t live_filters, pending_filters;
} cf_server_stats_t;
enum { CF_FILTER_PENDING = 0, CF_FILTER_LIVE = 1, CF_FILTER_CLOSING = 2,
       CF_FILTER_CLOSED = 3 };

cf_status cf_server_create(const cf_server_config* cfg, cf_server** out);
/* Drains outstanding requests, stops the scheduler, frees every filter. */
cf_status cf_server_destroy(cf_server* s);
/* Register a filter; it becomes live when the budget allows (CF_ENOMEM if
 * it can never fit).  Requests may be submitted to it at once. */
cf_status cf_server_add_filter(cf_server* s, const cf_config* cfg,
                               uint32_t* filter_id);
/* Close a filter after its queued requests; frees its budget. */
cf_status cf_server_remove_filter(cf_server* s, uint32_t filter_id);
cf_status cf_server_filter_state(cf_server* s, uint32_t filter_id,
                                 int32_t* state);
/* The live filter object (for cf_stats / cf_snapshot once its requests
 * have drained); NULL unless live. */
cf_filter* cf_server_get_filter(cf_server* s, uint32_t filter_id);
/* Queue one request (non-blocking).  CF_EINVAL for an unknown filter, a bad
 * op, n > max_wave_keys, or a query without out_flags. */
cf_status cf_server_submit(cf_server* s, const cf_request* r,
                           uint64_t* request_id);
/* Move up to max completions (in completion order) to `out`; returns how
 * many were written. */
uint32_t cf_server_poll(cf_server* s, cf_completion* out, uint32_t max);
/* Wait until every submitted request has completed; CF_ETIMEOUT after
 * timeout_ms (the work keeps running; the context is untouched). */
cf_status cf_server_drain(cf_server* s, uint32_t timeout_ms);
cf_status cf_server_stats(cf_server* s, cf_server_stats_t* out);
/* Replay a trace through the server: request i is submitted at
 * arrival_s[i] seconds after the call starts (busy-waiting the host
 * clock), then everything is drained; completions are written by request
 * index (out[i]).  The latency of request i is out[i].done_s -
 * out[i].submit_s. */
cf_status cf_server_run_trace(cf_server* s, const cf_request* reqs,
                              const double* arrival_s, uint32_t n,
                              cf_completion* out);
/* The baseline the server is compared with: the same trace run by one
 * host thread with one plain cf_insert / cf_contains / cf_remove call per
 * request on one stream, each synchronised before the next starts (a
 * request waits for every earlier one).  filters[r.filter_id] is used. */
cf_status cf_plain_run_trace(cf_filter* const* filters, uint32_t n_filters,
                             const cf_request* reqs, const double* arrival_s,
                             uint32_t n, cf_completion* out, void* stream);

/* ---- insert without device allocation ------------------------------------
 * The paper has no counterpart to this entry point.
 *
 * cf_insert keeps a work queue of 4 bytes per key in device memory that the
 * library cudaMalloc's on a filter's first large insert (and reuses after).
 * Some callers cannot allow a device allocation there: code whose device
 * memory is all handed out by another allocator or a fixed-size arena,
 * code on a path that must not stall on cudaMalloc's implicit device
 * synchronisation, and code that must not fail with out-of-memory halfway
 * through a batch.  cf_insert_noalloc runs the plain two-kernel insert
 * (direct insertion into i1 / i2, then the eviction loop of Sec. 4.6.1 over
 * the queued keys) with its queue in a fixed array compiled into the
 * library: a file-scope __device__ array of CF_NOALLOC_MAX_KEYS entries
 * (4 MiB), which every GPU that loads the library holds until the process
 * exits.  It ignores the filter's slicing mode (cf_set_slicing): it never
 * takes the slice-partitioned path, which needs scratch memory.  Its
 * results obey the same rules as cf_insert's (flags, counters, victims,
 * the multiset of stored tags); where several placements are valid, the
 * two entry points may pick different ones.  It calls no cudaMalloc,
 * cudaFree or other device-allocating routine.  Keys and flags are still
 * the caller's; build the filter with cf_create_at to keep the whole path
 * free of library allocations.
 *  - n > CF_NOALLOC_MAX_KEYS returns CF_EINVAL (split larger batches).
 *  - The filter's device must be the current device (CF_EINVAL otherwise).
 *    Every call looks up the array's device address in the current context
 *    with cudaGetSymbolAddress (CF_ECUDA if that fails).  The first call on
 *    a device also loads the library's device code there; make that first
 *    call before any stream capture.
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
/* Per-kernel device time of one filter's single-filter calls: while enabled,
 * an event pair is recorded on the launching stream around every kernel
 * launch (around each group of launches for the sliced passes).  Index 0:
 * insert phase 1 (direct insertion into i1 / i2), 1: insert phase 2
 * (eviction loop, both paths), 2: contains, 3: remove; slice-partitioned
 * path (cf_set_slicing): 4: grouping by slice (counter reset, scatter),
 * 5: bucket-i1 pass, 6: bucket-i2 pass, 7: results back to key order;
 * 8: the full-bucket map of the eviction loop (cf_set_eviction_map);
 * the host-buffer calls' copies, timed on their own streams: 9: keys to the
 * device (one record per staging chunk), 10: flags back to the host;
 * 11: the slice-grouped eviction levels of a sliced insert (the seed and
 * the levels; cf_set_eviction_levels), whose remaining chains run to their
 * end under kind 1 (which then also holds the loop's launch for a queue the
 * levels left alone).
 * cf_read_kernel_times waits for the recorded events, sums their elapsed
 * times and (reset != 0) recycles them. */
#define CF_KERNEL_KINDS 12
typedef struct {
  uint64_t launches[CF_KERNEL_KINDS];
  double ms[CF_KERNEL_KINDS];
} cf_kernel_times;
cf_status cf_set_kernel_timing(cf_filter* f, int enable);
cf_status cf_read_kernel_times(cf_filter* f, cf_kernel_times* out, int reset);

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
