/*
 * Sequential CPU cuckoo filter: the ORACLE for the GPU path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may call this library.  The product path never
 * links, loads or calls it, and it shares no code with the GPU path.
 *
 * It follows "Cuckoo-GPU: Accelerating Cuckoo Filters on Modern GPUs"
 * (Dortmann, Vieth, Schmidt, 2026) step by step, one slot at a time:
 *   - partial-key cuckoo hashing, Sec. 2.1 Eq. 1-3;
 *   - the hash split (upper 32 bits -> fingerprint, lower 32 -> i1), Sec. 4.3;
 *   - the bucket/word/tag layout, Sec. 4.2 and Fig. 2;
 *   - TryInsert and the insertion of Algorithm 1, the BFS eviction heuristic
 *     of Sec. 4.6.1 and (for comparison) the greedy DFS chain of Algorithm 1;
 *   - Find/Contains of Algorithm 2 and TryRemove/Remove of Algorithm 3;
 *   - the Offset ("choice bit") bucket policy of Sec. 4.6.2.
 * Readings of points the paper leaves open are stated beside the code that
 * takes them.
 *
 * Parameters: m = number of buckets, f = fingerprint bits in {8,16,32},
 * b = slots per bucket in {4,8,16}.  The XOR policy needs m a power of two;
 * the Offset policy takes any m >= 2.
 */
#ifndef CF_ORACLE_H
#define CF_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { CFO_POLICY_XOR = 0, CFO_POLICY_OFFSET = 1 };
enum { CFO_EVICT_BFS = 0, CFO_EVICT_DFS = 1 };

typedef struct cfo_filter cfo_filter;

typedef struct {
  uint64_t occupancy;        /* stored tags = sum(insert ok) - sum(remove ok) */
  uint64_t insert_ok;        /* keys whose Insert returned Success           */
  uint64_t insert_fail;      /* keys whose Insert returned Failure           */
  uint64_t remove_ok;
  uint64_t remove_fail;
  uint64_t evictions;        /* slot overwrites inside the eviction loop     */
  uint64_t victims;          /* tags dropped by failed inserts               */
  /* Bucket-touch counters (see cfo_insert / cfo_contains / cfo_remove):   */
  uint64_t ins_bucket_reads;   /* distinct buckets read, summed over keys    */
  uint64_t ins_bucket_writes;  /* distinct buckets written, summed over keys */
  uint64_t qry_bucket_reads;   /* buckets probed by Alg. 2 with short-circuit*/
  uint64_t rem_bucket_reads;   /* buckets probed by Alg. 3 with short-circuit*/
  uint64_t rem_bucket_writes;  /* buckets written by successful removes      */
  /* The insert counters split by phase of Alg. 1: direct insertion into i1
   * / i2, and the eviction loop (distinct buckets first touched there). */
  uint64_t ins_direct_reads, ins_direct_writes;
  uint64_t ins_evict_keys;     /* keys that entered the eviction loop        */
} cfo_stats;

/* Returns NULL on invalid parameters or allocation failure. */
cfo_filter* cfo_create(uint64_t m, uint32_t f, uint32_t b,
                       uint32_t max_evictions, uint32_t policy,
                       uint32_t eviction);
void cfo_destroy(cfo_filter* F);
void cfo_clear(cfo_filter* F);

/* XXH64 of the key's 8 little-endian bytes (public XXH64 specification). */
uint64_t cfo_xxh64_u64(uint64_t key, uint64_t seed);

/* Per-key fingerprint and candidate buckets (Sec. 2.1 Eq. 1-3, Sec. 4.3). */
void cfo_hash(const cfo_filter* F, uint64_t key, uint32_t* fp, uint64_t* i1,
              uint64_t* i2);
/* The alternate bucket of a tag stored in bucket j (XOR policy: the
 * involution j ^ H(fp); Offset policy: move by offset(fp) in the direction
 * given by the choice bit). */
uint64_t cfo_alt(const cfo_filter* F, uint64_t j, uint32_t tag);

/* One operation on one key.  insert returns 1 on success, 0 on failure and
 * writes the number of eviction-loop overwrites to *evictions (may be NULL).
 * contains/remove return 1 when found / removed. */
int cfo_insert(cfo_filter* F, uint64_t key, uint32_t* evictions);
int cfo_contains(cfo_filter* F, uint64_t key);
int cfo_remove(cfo_filter* F, uint64_t key);

/* Batches: keys processed strictly in order, flags[i] in {0,1}. */
void cfo_insert_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                      uint8_t* flags, uint32_t* evictions);
void cfo_contains_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                        uint8_t* flags);
void cfo_remove_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                      uint8_t* flags);
void cfo_hash_batch(const cfo_filter* F, const uint64_t* keys, uint64_t n,
                    uint32_t* fp, uint64_t* i1, uint64_t* i2);
/* The same hash for given (m, f, policy) without a table; -1 if invalid. */
int cfo_hash_params_batch(uint64_t m, uint32_t f, uint32_t policy,
                          const uint64_t* keys, uint64_t n, uint32_t* fp,
                          uint64_t* i1, uint64_t* i2);

/* Raw slot access for tests: slot s of bucket j. */
uint32_t cfo_get_slot(const cfo_filter* F, uint64_t j, uint32_t s);
void cfo_set_slot(cfo_filter* F, uint64_t j, uint32_t s, uint32_t tag);

/* Snapshot = 64-byte header + raw table in the GPU byte layout. */
uint64_t cfo_table_bytes(const cfo_filter* F);
uint64_t cfo_snapshot_bytes(const cfo_filter* F);
int cfo_snapshot(const cfo_filter* F, void* dst, uint64_t bytes);
int cfo_load(cfo_filter* F, const void* src, uint64_t bytes);

void cfo_get_stats(const cfo_filter* F, cfo_stats* out);
/* Victim log: (tag, bucket) of every tag dropped by a failed insert. */
uint64_t cfo_victims(const cfo_filter* F, uint32_t* tags, uint64_t* buckets,
                     uint64_t max);

#ifdef __cplusplus
}
#endif
#endif
