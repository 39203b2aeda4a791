// Types shared by the kernels and the host side of libcf.
#pragma once

#include <cstdint>

namespace cfk {

// Device control block: counters of one filter (256 bytes, at the start of
// the filter's device memory).
struct Ctrl {
  unsigned long long occupancy;
  unsigned long long insert_ok;
  unsigned long long insert_fail;
  unsigned long long remove_ok;
  unsigned long long remove_fail;
  unsigned long long evictions;
  unsigned long long victims;
  unsigned long long rollbacks;
  unsigned long long rollback_lost;
  unsigned long long contention;
  unsigned int error_word;
  unsigned int queue_count;  // eviction work queue fill (insert scratch)
  unsigned int done_blocks;  // last-block-done counter of the evict kernel
  unsigned int pad0;
  unsigned long long scratch_count;  // for cf_count_occupied
  // Eviction launches that built and used the full-bucket map.
  unsigned long long map_builds;
  // CAS-retry histogram: failed CAS attempts by their retry depth within one
  // loop (the attempt that failed was the r-th retry, r = 0 being the first
  // attempt): bins r = 0, 1, 2-3, 4-7, 8-15, 16-63, 64 and more.  Bin k thus
  // counts the loops that needed more than the retries of bins below it.
  unsigned long long cas_retry[7];
  // Bounds-checked builds: the first out-of-range bucket index + 1 (0: none).
  unsigned long long debug_bad_index;
  // Slice-grouped eviction levels that ran, the chain steps they took, and
  // the chains run to their end for want of room in a level's buffer.
  unsigned long long level_passes;
  unsigned long long level_steps;
  unsigned long long level_runout;
  unsigned long long pad[7];
};
static_assert(sizeof(Ctrl) == 256, "control block is 256 bytes");

struct Victim {
  uint32_t tag;
  uint32_t pad;
  uint64_t bucket;
};

// Everything a kernel needs to address one filter (passed by value).
struct DevFilter {
  void* table;
  uint64_t m;       // buckets
  uint64_t mask;    // m - 1 (XOR policy)
  uint64_t fm_m;    // fastmod multiplier for m   (Offset policy)
  uint64_t fm_m1;   // fastmod multiplier for m-1 (Offset policy)
  Ctrl* ctrl;
  Victim* victims;
  uint32_t victim_cap;
  uint32_t max_ev;
  uint32_t eviction;  // 0 BFS, 1 DFS
  uint32_t max_cas;   // bound of every CAS retry loop (attempts per word)
};

constexpr uint32_t kSliceMax = 1024;  // slices per table (shared-memory bins)
constexpr uint32_t kFill2Extra = 3;   // counters after the S per-slice ones

// Scratch of the slice-grouped eviction levels (see cf_levels.cuh): two
// record buffers used in turn, each S slice regions of cap records and a
// spill region of spill records, 3 words per record; per level (L + 1 sets)
// S + 2 counters one per 128-byte line (the S slice fills, the spill fill,
// the tile counter); ctl[0] = 1 when this launch runs the levels, ctl[1 + k]
// = records at the start of level k (k = 0..L).
struct LevelBufs {
  uint64_t* rec[2];
  uint32_t* fill;
  uint32_t* ctl;
  uint64_t cap;
  uint64_t spill;
  uint32_t n_levels;  // L
  uint32_t min_q;     // the levels run when at least this many keys are queued
  uint32_t stop_q;    // level k >= 1 runs only with at least this many records
  uint32_t pad;
};

// Device scratch of the slice-partitioned path for chunks of up to n keys
// (see cf_slice.cuh).
struct SliceBufs {
  uint32_t n_slices;  // S
  uint32_t shift;     // slice of bucket j = j >> shift
  uint64_t cap1;      // rec1 records per slice, a multiple of 256 (the spill region follows)
  uint64_t cap2;      // rec2 records per slice (the spill region follows)
  uint64_t rec2_len;  // S * cap2 + n: records rec2 and f2 hold
  uint32_t* fill1;    // [(S + 1) * 32] rec1 records claimed per slice, then the
                      // spill count (one counter per 128-byte line)
  uint32_t* fill2;    // [(S + 3) * 32] rec2 records claimed per slice, then
                      // the spill count and two tile counters
  uint32_t* dst;      // [n]     rec1 position of key j
  uint64_t* rec1;     // [S * cap1 + n] key hashes grouped by the slice of i1
  uint8_t* f1;        // [S * cap1 + n] flag of each rec1 record (written by merge)
  uint32_t* link;     // [S * cap1 + n] rec2 position of a pending rec1 record,
                      // else its flag tagged kSettled
  uint64_t* rec2;     // [S * cap2 + n] pending records grouped by i2's slice
  uint8_t* f2;        // [S * cap2 + n] result of probe2 / the eviction loop
};

}  // namespace cfk
