/*
 * Sequential CPU cuckoo filter: the ORACLE for the GPU path.
 *
 * TEST INFRASTRUCTURE ONLY (see cf_oracle.h).  Plain C, one slot at a time,
 * no SWAR, no vector loads, no concurrency.  Each function names the part of
 * "Cuckoo-GPU: Accelerating Cuckoo Filters on Modern GPUs" it follows.
 */
#include "cf_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* XXH64 (public xxHash specification, 64-bit variant), specialised to one   */
/* 8-byte little-endian input.  Sec. 4.3 step 1 names xxHash64 as the hash.  */
/* ------------------------------------------------------------------------ */
#define XXP1 0x9E3779B185EBCA87ULL
#define XXP2 0xC2B2AE3D27D4EB4FULL
#define XXP3 0x165667B19E3779F9ULL
#define XXP4 0x85EBCA77C2B2AE63ULL
#define XXP5 0x27D4EB2F165667C5ULL

static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

uint64_t cfo_xxh64_u64(uint64_t key, uint64_t seed) {
  /* Inputs shorter than 32 bytes: the accumulator starts at seed + PRIME5
   * plus the input length. */
  uint64_t acc = seed + XXP5 + 8u;
  /* One 8-byte lane: round(0, lane) = rotl(lane * PRIME2, 31) * PRIME1. */
  uint64_t lane = key * XXP2;
  lane = rotl64(lane, 31);
  lane *= XXP1;
  acc ^= lane;
  acc = rotl64(acc, 27) * XXP1 + XXP4;
  /* Final avalanche. */
  acc ^= acc >> 33;
  acc *= XXP2;
  acc ^= acc >> 29;
  acc *= XXP3;
  acc ^= acc >> 32;
  return acc;
}

/* splitmix64 (Steele, Lea, Flood 2014): the per-key random stream used for
 * the "random bucket" and "random slot" choices of the eviction loop
 * (Alg. 1, Sec. 4.6.1).  Reading: the stream is seeded with the key's 64-bit
 * hash, so the draws are a pure function of the key. */
static uint64_t rng_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Filter state.                                                             */
/* ------------------------------------------------------------------------ */
struct cfo_filter {
  uint64_t m;
  uint32_t f, b, max_ev, policy, eviction;
  uint32_t word_bits; /* 32 when a bucket is exactly 32 bits, else 64      */
  uint32_t tpw;       /* tags per word                                     */
  uint32_t wpb;       /* words per bucket                                  */
  uint32_t lane_mask; /* mask of one stored tag (f bits)                   */
  uint32_t fp_mask;   /* mask of the fingerprint proper                    */
  uint32_t choice;    /* Offset policy: the choice bit; XOR policy: 0      */
  uint64_t* w64;
  uint32_t* w32;
  cfo_stats st;
  uint32_t* vic_tag;
  uint64_t* vic_bucket;
  uint64_t vic_n, vic_cap;
  uint64_t* seen_r; /* distinct buckets read by the current insert        */
  uint64_t* seen_w; /* distinct buckets written by the current insert     */
  uint64_t n_r, n_w, seen_cap;
};

static int is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

cfo_filter* cfo_create(uint64_t m, uint32_t f, uint32_t b,
                       uint32_t max_evictions, uint32_t policy,
                       uint32_t eviction) {
  if (!(f == 8 || f == 16 || f == 32)) return NULL;
  if (!(b == 4 || b == 8 || b == 16)) return NULL;
  if (policy == CFO_POLICY_XOR) {
    if (!is_pow2(m) || m > (1ULL << 32)) return NULL;
  } else if (policy == CFO_POLICY_OFFSET) {
    if (m < 2 || m > (1ULL << 32)) return NULL;
  } else {
    return NULL;
  }
  if (eviction != CFO_EVICT_BFS && eviction != CFO_EVICT_DFS) return NULL;
  cfo_filter* F = (cfo_filter*)calloc(1, sizeof(cfo_filter));
  if (!F) return NULL;
  F->m = m;
  F->f = f;
  F->b = b;
  F->max_ev = max_evictions;
  F->policy = policy;
  F->eviction = eviction;
  /* Sec. 4.2: buckets are arrays of 64-bit words with tags packed in; a
   * bucket of exactly 32 bits (f = 8, b = 4) is one 32-bit word. */
  F->word_bits = (f * b == 32) ? 32u : 64u;
  F->tpw = F->word_bits / f;
  F->wpb = (f * b) / F->word_bits;
  F->lane_mask = (f == 32) ? 0xFFFFFFFFu : ((1u << f) - 1u);
  if (policy == CFO_POLICY_OFFSET) {
    F->choice = 1u << (f - 1);
    F->fp_mask = F->choice - 1u;
  } else {
    F->choice = 0;
    F->fp_mask = F->lane_mask;
  }
  uint64_t words = m * F->wpb;
  if (F->word_bits == 64)
    F->w64 = (uint64_t*)calloc(words, sizeof(uint64_t));
  else
    F->w32 = (uint32_t*)calloc(words, sizeof(uint32_t));
  F->seen_cap = 64;
  F->seen_r = (uint64_t*)malloc(F->seen_cap * sizeof(uint64_t));
  F->seen_w = (uint64_t*)malloc(F->seen_cap * sizeof(uint64_t));
  if ((!F->w64 && !F->w32) || !F->seen_r || !F->seen_w) {
    cfo_destroy(F);
    return NULL;
  }
  return F;
}

void cfo_destroy(cfo_filter* F) {
  if (!F) return;
  free(F->w64);
  free(F->w32);
  free(F->vic_tag);
  free(F->vic_bucket);
  free(F->seen_r);
  free(F->seen_w);
  free(F);
}

void cfo_clear(cfo_filter* F) {
  uint64_t words = F->m * F->wpb;
  if (F->w64) memset(F->w64, 0, words * sizeof(uint64_t));
  if (F->w32) memset(F->w32, 0, words * sizeof(uint32_t));
  memset(&F->st, 0, sizeof(F->st));
  F->vic_n = 0;
}

/* ------------------------------------------------------------------------ */
/* Layout (Sec. 4.2, Fig. 2): slot s of bucket j is lane (s mod tpw) of word */
/* (s div tpw) of that bucket; lane L occupies bits [L*f, L*f + f).          */
/* Zero is EMPTY (Alg. 3).                                                   */
/* ------------------------------------------------------------------------ */
uint32_t cfo_get_slot(const cfo_filter* F, uint64_t j, uint32_t s) {
  uint64_t wi = j * F->wpb + s / F->tpw;
  uint32_t shift = (s % F->tpw) * F->f;
  uint64_t word = F->word_bits == 64 ? F->w64[wi] : (uint64_t)F->w32[wi];
  return (uint32_t)((word >> shift) & F->lane_mask);
}

void cfo_set_slot(cfo_filter* F, uint64_t j, uint32_t s, uint32_t tag) {
  uint64_t wi = j * F->wpb + s / F->tpw;
  uint32_t shift = (s % F->tpw) * F->f;
  uint64_t lm = (uint64_t)F->lane_mask << shift;
  uint64_t val = ((uint64_t)(tag & F->lane_mask)) << shift;
  if (F->word_bits == 64)
    F->w64[wi] = (F->w64[wi] & ~lm) | val;
  else
    F->w32[wi] = (uint32_t)(((uint64_t)F->w32[wi] & ~lm) | val);
}

/* ------------------------------------------------------------------------ */
/* Hashing: Eq. 1-3 with the split of Sec. 4.3 step 1.                       */
/* ------------------------------------------------------------------------ */
static uint32_t fp_hash(uint32_t fp) {
  /* H(fp) of Eq. 3: the same xxHash64, applied to the fingerprint value
   * zero-extended to 8 bytes; its lower 32 bits are used. */
  return (uint32_t)cfo_xxh64_u64((uint64_t)fp, 0);
}

static uint64_t offset_of(const cfo_filter* F, uint32_t fp) {
  /* Offset policy (Sec. 4.6.2): offset(fp) in [1, m-1], so that the two
   * candidate buckets always differ. */
  return 1u + (uint64_t)fp_hash(fp) % (F->m - 1);
}

static void hash_key(const cfo_filter* F, uint64_t key, uint64_t* h,
                     uint32_t* fp, uint64_t* i1, uint64_t* i2) {
  *h = cfo_xxh64_u64(key, 0);
  /* Upper 32 bits -> fingerprint; zero is EMPTY, so a zero fingerprint is
   * mapped to 1. */
  uint32_t raw = (uint32_t)(*h >> 32) & F->fp_mask;
  if (raw == 0) raw = 1;
  *fp = raw;
  if (F->policy == CFO_POLICY_XOR) {
    /* Lower 32 bits -> primary bucket; Eq. 3 for the alternate. */
    *i1 = (uint64_t)(uint32_t)*h & (F->m - 1);
    *i2 = *i1 ^ ((uint64_t)fp_hash(raw) & (F->m - 1));
  } else {
    *i1 = (uint64_t)(uint32_t)*h % F->m;
    *i2 = (*i1 + offset_of(F, raw)) % F->m;
  }
}

void cfo_hash(const cfo_filter* F, uint64_t key, uint32_t* fp, uint64_t* i1,
              uint64_t* i2) {
  uint64_t h;
  hash_key(F, key, &h, fp, i1, i2);
}

void cfo_hash_batch(const cfo_filter* F, const uint64_t* keys, uint64_t n,
                    uint32_t* fp, uint64_t* i1, uint64_t* i2) {
  for (uint64_t i = 0; i < n; ++i) cfo_hash(F, keys[i], &fp[i], &i1[i], &i2[i]);
}

int cfo_hash_params_batch(uint64_t m, uint32_t f, uint32_t policy,
                          const uint64_t* keys, uint64_t n, uint32_t* fp,
                          uint64_t* i1, uint64_t* i2) {
  /* Same hash as a filter with these parameters, without allocating one. */
  cfo_filter F;
  memset(&F, 0, sizeof F);
  if (!(f == 8 || f == 16 || f == 32)) return -1;
  if (policy == CFO_POLICY_XOR ? (!is_pow2(m) || m > (1ULL << 32))
                               : (m < 2 || m > (1ULL << 32)))
    return -1;
  F.m = m;
  F.f = f;
  F.policy = policy;
  F.lane_mask = (f == 32) ? 0xFFFFFFFFu : ((1u << f) - 1u);
  F.choice = policy == CFO_POLICY_OFFSET ? 1u << (f - 1) : 0u;
  F.fp_mask = policy == CFO_POLICY_OFFSET ? F.choice - 1u : F.lane_mask;
  cfo_hash_batch(&F, keys, n, fp, i1, i2);
  return 0;
}

/* Alternate location of a tag stored in bucket j.  XOR policy: Eq. 3 is an
 * involution, the tag is unchanged.  Offset policy: the choice bit says
 * whether j is the primary (bit 0: go forward by offset) or the alternate
 * (bit 1: go back); the bit flips with the move. */
static uint64_t alt_of(const cfo_filter* F, uint64_t j, uint32_t tag,
                       uint32_t* moved_tag) {
  if (F->policy == CFO_POLICY_XOR) {
    *moved_tag = tag;
    return j ^ ((uint64_t)fp_hash(tag) & (F->m - 1));
  }
  uint32_t fp = tag & F->fp_mask;
  uint64_t off = offset_of(F, fp);
  if (tag & F->choice) {
    *moved_tag = fp;
    return (j + F->m - off) % F->m;
  }
  *moved_tag = fp | F->choice;
  return (j + off) % F->m;
}

uint64_t cfo_alt(const cfo_filter* F, uint64_t j, uint32_t tag) {
  uint32_t t;
  return alt_of(F, j, tag, &t);
}

/* ------------------------------------------------------------------------ */
/* Bucket primitives.                                                        */
/* ------------------------------------------------------------------------ */

/* TryInsert of Alg. 1: start at word (tag mod b) / tpw, scan the words with
 * wrap-around, take the lowest empty lane of the first word that has one. */
static int try_insert(cfo_filter* F, uint64_t j, uint32_t tag) {
  uint32_t start = (tag % F->b) / F->tpw;
  for (uint32_t i = 0; i < F->wpb; ++i) {
    uint32_t w = (start + i) % F->wpb;
    for (uint32_t lane = 0; lane < F->tpw; ++lane) {
      uint32_t s = w * F->tpw + lane;
      if (cfo_get_slot(F, j, s) == 0) {
        cfo_set_slot(F, j, s, tag);
        return 1;
      }
    }
  }
  return 0;
}

static int has_empty(const cfo_filter* F, uint64_t j) {
  for (uint32_t s = 0; s < F->b; ++s)
    if (cfo_get_slot(F, j, s) == 0) return 1;
  return 0;
}

/* Find of Alg. 2: does any slot of bucket j hold `tag`? */
static int find(const cfo_filter* F, uint64_t j, uint32_t tag) {
  for (uint32_t s = 0; s < F->b; ++s)
    if (cfo_get_slot(F, j, s) == tag) return 1;
  return 0;
}

/* TryRemove of Alg. 3: same start word and scan order as TryInsert; clear
 * the lowest matching lane of the first word that has one. */
static int try_remove(cfo_filter* F, uint64_t j, uint32_t tag) {
  uint32_t start = (tag % F->b) / F->tpw;
  for (uint32_t i = 0; i < F->wpb; ++i) {
    uint32_t w = (start + i) % F->wpb;
    for (uint32_t lane = 0; lane < F->tpw; ++lane) {
      uint32_t s = w * F->tpw + lane;
      if (cfo_get_slot(F, j, s) == tag) {
        cfo_set_slot(F, j, s, 0);
        return 1;
      }
    }
  }
  return 0;
}

/* Distinct-bucket bookkeeping for the insert byte counters (which = 0: the
 * buckets read by the current insert, which = 1: the buckets written). */
static void note(cfo_filter* F, int which, uint64_t j) {
  uint64_t* set = which ? F->seen_w : F->seen_r;
  uint64_t* n = which ? &F->n_w : &F->n_r;
  for (uint64_t i = 0; i < *n; ++i)
    if (set[i] == j) return;
  if (*n == F->seen_cap) {
    uint64_t cap = F->seen_cap * 2;
    uint64_t* r = (uint64_t*)realloc(F->seen_r, cap * sizeof(uint64_t));
    if (!r) return; /* counters become a lower bound; never fatal */
    F->seen_r = r;
    uint64_t* w = (uint64_t*)realloc(F->seen_w, cap * sizeof(uint64_t));
    if (!w) return;
    F->seen_w = w;
    F->seen_cap = cap;
    set = which ? F->seen_w : F->seen_r;
  }
  set[(*n)++] = j;
}
#define NOTE_READ(F, j) note((F), 0, (j))
#define NOTE_WRITE(F, j) note((F), 1, (j))

static void log_victim(cfo_filter* F, uint32_t tag, uint64_t bucket) {
  if (F->vic_n == F->vic_cap) {
    uint64_t cap = F->vic_cap ? F->vic_cap * 2 : 64;
    uint32_t* t = (uint32_t*)realloc(F->vic_tag, cap * sizeof(uint32_t));
    if (t) F->vic_tag = t;
    uint64_t* bk = (uint64_t*)realloc(F->vic_bucket, cap * sizeof(uint64_t));
    if (bk) F->vic_bucket = bk;
    if (!t || !bk) return;
    F->vic_cap = cap;
  }
  F->vic_tag[F->vic_n] = tag;
  F->vic_bucket[F->vic_n] = bucket;
  F->vic_n++;
}

/* ------------------------------------------------------------------------ */
/* Eviction loops.  Both start from `cur` holding `tag` as it is stored in  */
/* cur; both return 1 on success.  *ev counts slot overwrites.              */
/* ------------------------------------------------------------------------ */

/* BFS heuristic of Sec. 4.6.1.  Readings: the inspected candidates are b/2
 * consecutive slots from a random start; a candidate whose alternate bucket
 * equals cur cannot be relocated and is skipped; "the last candidate" is the
 * last of the b/2 inspected. */
static int evict_bfs(cfo_filter* F, uint64_t* rng, uint64_t cur, uint32_t tag,
                     uint32_t* ev, uint32_t* vt, uint64_t* vb) {
  const uint32_t half = F->b / 2;
  while (*ev < F->max_ev) {
    uint32_t start = (uint32_t)(rng_next(rng) % F->b);
    NOTE_READ(F, cur);
    for (uint32_t k = 0; k < half; ++k) {
      uint32_t c = (start + k) % F->b;
      uint32_t t = cfo_get_slot(F, cur, c);
      uint32_t moved;
      uint64_t a = alt_of(F, cur, t, &moved);
      if (a == cur) continue;
      NOTE_READ(F, a);
      if (has_empty(F, a)) {
        /* Two-step relocation: the candidate goes to its alternate bucket,
         * then the new tag takes the candidate's slot. */
        try_insert(F, a, moved);
        NOTE_WRITE(F, a);
        cfo_set_slot(F, cur, c, tag);
        NOTE_WRITE(F, cur);
        (*ev)++;
        return 1;
      }
    }
    /* No shallow path: evict the last candidate and restart from its
     * alternate bucket. */
    uint32_t c = (start + half - 1) % F->b;
    uint32_t t = cfo_get_slot(F, cur, c);
    uint32_t moved;
    uint64_t a = alt_of(F, cur, t, &moved);
    cfo_set_slot(F, cur, c, tag);
    NOTE_WRITE(F, cur);
    (*ev)++;
    tag = moved;
    cur = a;
    NOTE_READ(F, cur);
    if (try_insert(F, cur, tag)) {
      NOTE_WRITE(F, cur);
      return 1;
    }
  }
  *vt = tag;
  *vb = cur;
  return 0;
}

/* Greedy chain of Alg. 1 phase 2: swap the tag into a random slot, carry the
 * evicted tag to its alternate bucket, try a direct insert there, repeat. */
static int evict_dfs(cfo_filter* F, uint64_t* rng, uint64_t cur, uint32_t tag,
                     uint32_t* ev, uint32_t* vt, uint64_t* vb) {
  while (*ev < F->max_ev) {
    uint32_t s = (uint32_t)(rng_next(rng) % F->b);
    NOTE_READ(F, cur);
    uint32_t evicted = cfo_get_slot(F, cur, s);
    cfo_set_slot(F, cur, s, tag);
    NOTE_WRITE(F, cur);
    (*ev)++;
    uint32_t moved;
    cur = alt_of(F, cur, evicted, &moved);
    tag = moved;
    NOTE_READ(F, cur);
    if (try_insert(F, cur, tag)) {
      NOTE_WRITE(F, cur);
      return 1;
    }
  }
  *vt = tag;
  *vb = cur;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Operations.                                                               */
/* ------------------------------------------------------------------------ */

/* Insert of Alg. 1: direct insertion into i1, then i2; otherwise the
 * eviction loop, starting from a randomly picked candidate bucket. */
int cfo_insert(cfo_filter* F, uint64_t key, uint32_t* evictions) {
  uint64_t h, i1, i2;
  uint32_t fp;
  hash_key(F, key, &h, &fp, &i1, &i2);
  const uint32_t t1 = fp;             /* tag as stored in i1 */
  const uint32_t t2 = fp | F->choice; /* tag as stored in i2 */
  uint32_t ev = 0;
  int ok = 0;
  F->n_r = F->n_w = 0;
  NOTE_READ(F, i1);
  if (try_insert(F, i1, t1)) {
    NOTE_WRITE(F, i1);
    ok = 1;
  } else {
    NOTE_READ(F, i2);
    if (try_insert(F, i2, t2)) {
      NOTE_WRITE(F, i2);
      ok = 1;
    }
  }
  F->st.ins_direct_reads += F->n_r;
  F->st.ins_direct_writes += F->n_w;
  if (!ok) {
    uint32_t vt = t1;
    uint64_t vb = i1;
    F->st.ins_evict_keys++;
    if (F->max_ev > 0) {
      uint64_t rng = h;
      int first = (rng_next(&rng) & 1) == 0;
      uint64_t cur = first ? i1 : i2;
      uint32_t tag = first ? t1 : t2;
      ok = (F->eviction == CFO_EVICT_BFS)
               ? evict_bfs(F, &rng, cur, tag, &ev, &vt, &vb)
               : evict_dfs(F, &rng, cur, tag, &ev, &vt, &vb);
    }
    if (!ok) {
      /* "Table too full, caller will have to rebuild": the tag in hand is
       * dropped and logged. */
      log_victim(F, vt, vb);
      F->st.victims++;
    }
  }
  F->st.evictions += ev;
  F->st.ins_bucket_reads += F->n_r;
  F->st.ins_bucket_writes += F->n_w;
  if (ok) {
    F->st.insert_ok++;
    F->st.occupancy++;
  } else {
    F->st.insert_fail++;
  }
  if (evictions) *evictions = ev;
  return ok;
}

/* Contains of Alg. 2: Find(i1) or Find(i2), short-circuit. */
int cfo_contains(cfo_filter* F, uint64_t key) {
  uint64_t h, i1, i2;
  uint32_t fp;
  hash_key(F, key, &h, &fp, &i1, &i2);
  F->st.qry_bucket_reads++;
  if (find(F, i1, fp)) return 1;
  F->st.qry_bucket_reads++;
  return find(F, i2, fp | F->choice);
}

/* Remove of Alg. 3: TryRemove(i1) or TryRemove(i2), short-circuit. */
int cfo_remove(cfo_filter* F, uint64_t key) {
  uint64_t h, i1, i2;
  uint32_t fp;
  hash_key(F, key, &h, &fp, &i1, &i2);
  int ok;
  F->st.rem_bucket_reads++;
  ok = try_remove(F, i1, fp);
  if (!ok) {
    F->st.rem_bucket_reads++;
    ok = try_remove(F, i2, fp | F->choice);
  }
  if (ok) {
    F->st.rem_bucket_writes++;
    F->st.remove_ok++;
    F->st.occupancy--;
  } else {
    F->st.remove_fail++;
  }
  return ok;
}

void cfo_insert_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                      uint8_t* flags, uint32_t* evictions) {
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t ev = 0;
    int ok = cfo_insert(F, keys[i], &ev);
    if (flags) flags[i] = (uint8_t)ok;
    if (evictions) evictions[i] = ev;
  }
}

void cfo_contains_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                        uint8_t* flags) {
  for (uint64_t i = 0; i < n; ++i) flags[i] = (uint8_t)cfo_contains(F, keys[i]);
}

void cfo_remove_batch(cfo_filter* F, const uint64_t* keys, uint64_t n,
                      uint8_t* flags) {
  for (uint64_t i = 0; i < n; ++i) {
    int ok = cfo_remove(F, keys[i]);
    if (flags) flags[i] = (uint8_t)ok;
  }
}

/* ------------------------------------------------------------------------ */
/* Snapshot: a 64-byte little-endian header followed by the raw table.       */
/*   0 magic u32 'CFG1'   4 version u32 = 1   8 m u64                         */
/*  16 f u32   20 b u32   24 max_evictions u32   28 policy u32                */
/*  32 occupancy u64   40 table bytes u64   48 hash id u32 = 1                */
/*  52 eviction u32   56 reserved u64 = 0                                     */
/* ------------------------------------------------------------------------ */
#define SNAP_MAGIC 0x31474643u
#define SNAP_HDR 64u

uint64_t cfo_table_bytes(const cfo_filter* F) {
  return F->m * F->wpb * (F->word_bits / 8u);
}

uint64_t cfo_snapshot_bytes(const cfo_filter* F) {
  return SNAP_HDR + cfo_table_bytes(F);
}

static void put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static void put64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t get32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
static uint64_t get64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

int cfo_snapshot(const cfo_filter* F, void* dst, uint64_t bytes) {
  if (bytes < cfo_snapshot_bytes(F)) return -1;
  uint8_t* p = (uint8_t*)dst;
  memset(p, 0, SNAP_HDR);
  put32(p + 0, SNAP_MAGIC);
  put32(p + 4, 1);
  put64(p + 8, F->m);
  put32(p + 16, F->f);
  put32(p + 20, F->b);
  put32(p + 24, F->max_ev);
  put32(p + 28, F->policy);
  put64(p + 32, F->st.occupancy);
  put64(p + 40, cfo_table_bytes(F));
  put32(p + 48, 1);
  put32(p + 52, F->eviction);
  /* Table bytes, word by word in little-endian order. */
  uint8_t* t = p + SNAP_HDR;
  uint64_t words = F->m * F->wpb;
  for (uint64_t w = 0; w < words; ++w) {
    if (F->word_bits == 64)
      put64(t + 8 * w, F->w64[w]);
    else
      put32(t + 4 * w, F->w32[w]);
  }
  return 0;
}

int cfo_load(cfo_filter* F, const void* src, uint64_t bytes) {
  const uint8_t* p = (const uint8_t*)src;
  if (bytes < SNAP_HDR) return -1;
  if (get32(p) != SNAP_MAGIC || get32(p + 4) != 1) return -2;
  if (get64(p + 8) != F->m || get32(p + 16) != F->f || get32(p + 20) != F->b ||
      get32(p + 28) != F->policy)
    return -3;
  if (get64(p + 40) != cfo_table_bytes(F) ||
      bytes < SNAP_HDR + cfo_table_bytes(F))
    return -4;
  const uint8_t* t = p + SNAP_HDR;
  uint64_t words = F->m * F->wpb;
  for (uint64_t w = 0; w < words; ++w) {
    if (F->word_bits == 64)
      F->w64[w] = get64(t + 8 * w);
    else
      F->w32[w] = get32(t + 4 * w);
  }
  memset(&F->st, 0, sizeof(F->st));
  F->vic_n = 0;
  /* Occupancy is recounted from the table rather than trusted. */
  uint64_t occ = 0;
  for (uint64_t j = 0; j < F->m; ++j)
    for (uint32_t s = 0; s < F->b; ++s) occ += cfo_get_slot(F, j, s) != 0;
  F->st.occupancy = occ;
  return 0;
}

void cfo_get_stats(const cfo_filter* F, cfo_stats* out) { *out = F->st; }

uint64_t cfo_victims(const cfo_filter* F, uint32_t* tags, uint64_t* buckets,
                     uint64_t max) {
  uint64_t n = F->vic_n < max ? F->vic_n : max;
  for (uint64_t i = 0; i < n; ++i) {
    if (tags) tags[i] = F->vic_tag[i];
    if (buckets) buckets[i] = F->vic_bucket[i];
  }
  return F->vic_n;
}
