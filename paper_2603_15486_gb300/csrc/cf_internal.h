// Host-side state shared by the translation units of libcf (not part of
// the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "cf.h"
#include "cf_kernels.cuh"

namespace cfk {

// Keys per staging chunk of the host-buffer calls (default).
constexpr uint64_t kDefaultStage = 1ull << 24;

// Staging slots of the host-buffer calls, used in turn (across calls too):
// the copies of the next kStageSlots - 1 chunks can run while a chunk's
// kernels run, so the host-to-device copies follow one another without
// waiting (a copy started on an idle link ran at half its rate).  Eight
// slots of 2^25 keys hold a whole 2^28-key sliced pass, so the next pass's
// keys can cross the link while the current pass finishes.
constexpr int kStageSlots = 8;

struct Stage {
  uint64_t* keys = nullptr;
  cudaEvent_t in_done = nullptr, comp_done = nullptr;
  bool used = false;  // comp_done has been recorded
};

// Flags of the host-buffer calls are gathered on the device for several
// staging chunks and copied back in one piece per group of about
// kFlagGroupBytes: many small device-to-host copies were measured to run at
// a fraction of the link's rate on some boxes (32 MiB pieces at 44 GB/s
// where 1 GiB copies ran at 194 GB/s).  Two groups alternate, so that the
// kernels of one group overlap the copy of the other.
constexpr uint64_t kFlagGroupBytes = 256ull << 20;
struct FlagGroup {
  uint8_t* flags = nullptr;
  uint64_t cap = 0;  // bytes
  cudaEvent_t comp_done = nullptr, out_done = nullptr;
  bool used = false;  // out_done has been recorded
};

// Per-filter call ordering: the event of the filter's last operation and the
// stream it ran on.  A batched launch that touched the filter instead leaves
// a borrowed event (ext_ev) of the batch; such events are never destroyed
// (they come from a process-wide pool), so a filter may outlive the batch.
cf_status order_on(cf_filter* f, cudaStream_t s);
cf_status mark(cf_filter* f, cudaStream_t s);
void mark_external(cf_filter* f, cudaStream_t s, cudaEvent_t ev);
cudaEvent_t pooled_event();
void set_error(const char* what, cudaError_t e);
void set_error_text(const char* text);

// Per-filter kernel timer: an event pair recorded around every launch while
// enabled; read (and recycled) by cf_read_kernel_times.
struct FilterTimer final : KernelTimer {
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int open_kind = -1;
  cudaEvent_t open_a = nullptr;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int kind, cudaStream_t s) override {
    open_kind = kind;
    open_a = take();
    cudaEventRecord(open_a, s);
  }
  void end(int kind, cudaStream_t s) override {
    cudaEvent_t b = take();
    cudaEventRecord(b, s);
    recs.push_back(Rec{kind, open_a, b});
    open_a = nullptr;
  }
  ~FilterTimer() override {
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace cfk

struct cf_filter {
  cf_config cfg{};
  int device = 0;
  char* mem = nullptr;
  size_t mem_bytes = 0;
  bool owns = false;
  cfk::DevFilter d{};
  const cfk::Ops* ops = nullptr;
  cudaEvent_t last_ev = nullptr;
  cudaEvent_t ext_ev = nullptr;  // borrowed from a batch (see order_on)
  cudaStream_t last_stream = nullptr;
  bool has_last = false;
  uint32_t* queue = nullptr;
  uint64_t queue_cap = 0;
  uint64_t stage_chunk = cfk::kDefaultStage;
  cfk::Stage stage[cfk::kStageSlots];
  cfk::FlagGroup fgroup[2];
  uint64_t group_chunks = 1;  // staging chunks per flag group
  uint32_t next_slot = 0;     // staging slot and flag group used next
  uint32_t next_group = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  int host_reads = 0;  // cf_set_host_reads: 0 staged copies, 1 sliced passes read pinned keys in place
  bool stage_ready = false;
  cfk::FilterTimer* timer = nullptr;  // non-null while kernel timing is on
  // Slice-partitioned path (cf_set_slicing): mode, geometry, scratch.
  int slice_mode = 1;                  // 0 off, 1 auto, 2 always
  uint64_t slice_bytes = 0;            // table bytes per slice (0: default)
  uint64_t slice_chunk = 0;            // keys per sliced pass (0: default)
  cfk::SliceBufs sb{};
  uint64_t sb_cap = 0;                 // keys the scratch is sized for
  void* sb_mem = nullptr;
  // Full-bucket map of the eviction loop (cf_set_eviction_map): mode,
  // least queued keys, and the map itself (allocated on first use).
  int map_mode = 1;                    // 0 off, 1 automatic, 2 always
  uint64_t map_min_queue = 0;          // 0: automatic rule
  uint32_t* fullmap = nullptr;
  // Slice-grouped eviction levels (cf_set_eviction_levels): mode, levels,
  // thresholds (0: defaults) and the record buffers (allocated on first use).
  int lv_mode = 1;                     // 0 off, 1 device-buffer calls, 2 all calls
  uint32_t lv_levels = 0;
  uint64_t lv_min_queue = 0;
  uint64_t lv_stop_queue = 0;
  cfk::LevelBufs lv{};
  uint64_t lv_cap_n = 0;               // keys per pass the buffers are sized for
  uint32_t lv_slices = 0;              // slices they are laid out for
  void* lv_mem = nullptr;
};

