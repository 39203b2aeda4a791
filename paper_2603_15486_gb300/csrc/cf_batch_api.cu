// Host side of the multi-filter launch (cf_batch_* in include/cf.h) and its
// autotuner.
//
// A plan owns one device buffer laid out as
//   [BatchCtl 64 B][first-tile index per item, u64 x (max_items+1)]
//   [item descriptors x max_items][eviction queue, uint2 x max_keys]
// and a pinned host copy of the descriptor part.  cf_batch_set writes the
// host copy; a launch uploads it with one cudaMemcpyAsync (which also zeroes
// the device counters) and starts the two kernels, so a launch needs no
// host synchronisation and can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "cf.h"
#include "cf_batch.cuh"
#include "cf_internal.h"

using cfk::BatchCtl;
using cfk::BatchItemDev;
using cfk::BatchVariant;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Autotuner results by batch class: (f, b, policy, op mask, log2 of the
// total keys, log2 of the item count) -> variant index.
using ClassKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<ClassKey, int> g_tuned;

int ilog2(uint64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

}  // namespace

struct cf_batch {
  uint32_t max_items = 0;
  uint64_t max_keys = 0;
  int device = 0;
  char* dev = nullptr;
  size_t dev_bytes = 0;
  char* host = nullptr;
  size_t desc_bytes = 0;
  size_t off_begins = 0, off_items = 0, off_queue = 0;
  // staged batch
  uint32_t n_items = 0;
  uint64_t n_tiles = 0, total_keys = 0;
  bool has_insert = false;
  int f = -1, b = -1, policy = -1, op_mask = 0;
  std::vector<cf_batch_item> items;
  std::vector<cf_filter*> filters;
  const BatchVariant* variants = nullptr;
  int n_variants = 0;
  int variant = 0;
  int pinned_variant = -1;
  float tuned_ms = 0.f;
  // ordering and graph
  cudaEvent_t done_ev = nullptr;
  cudaEvent_t upload_ev = nullptr;
  bool pending = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_variant = -1;
};

namespace {

#define CFB_CUDA(call)                  \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) {            \
      cfk::set_error(#call, e_);        \
      return CF_ECUDA;                  \
    }                                   \
  } while (0)

BatchCtl* ctl_host(cf_batch* b) { return reinterpret_cast<BatchCtl*>(b->host); }
uint64_t* begins_host(cf_batch* b) {
  return reinterpret_cast<uint64_t*>(b->host + b->off_begins);
}
BatchItemDev* items_host(cf_batch* b) {
  return reinterpret_cast<BatchItemDev*>(b->host + b->off_items);
}

// Write the staged items into the pinned descriptor buffer for the current
// variant's tile size.
void restage(cf_batch* b) {
  const uint64_t tile = 32ull * uint64_t(b->variants[b->variant].keys_per_thread);
  BatchCtl* c = ctl_host(b);
  std::memset(c, 0, sizeof(BatchCtl));
  uint64_t* beg = begins_host(b);
  BatchItemDev* it = items_host(b);
  uint64_t t = 0;
  for (uint32_t i = 0; i < b->n_items; ++i) {
    const cf_batch_item& x = b->items[i];
    beg[i] = t;
    t += (x.n + tile - 1) / tile;
    it[i].d = x.filter->d;
    it[i].keys = x.keys;
    it[i].flags = x.out_flags;
    it[i].n = x.n;
    it[i].op = x.op;
    it[i].pad = 0;
  }
  beg[b->n_items] = t;
  c->n_items = b->n_items;
  c->has_insert = b->has_insert ? 1u : 0u;
  c->n_tiles = t;
  b->n_tiles = t;
}

cf_status wait_upload(cf_batch* b) {
  if (b->pending) {
    CFB_CUDA(cudaEventSynchronize(b->upload_ev));
    b->pending = false;
  }
  return CF_OK;
}

unsigned grid_of(const void* fn, int block) {
  return unsigned(cfk::device_sm_count() * cfk::cached_occupancy(fn, block));
}

// Upload + kernels (the part a graph captures).
cf_status enqueue(cf_batch* b, cudaStream_t s, bool always_evict) {
  const BatchVariant& v = b->variants[b->variant];
  CFB_CUDA(cudaMemcpyAsync(b->dev, b->host, b->desc_bytes, cudaMemcpyHostToDevice, s));
  BatchCtl* ctl = reinterpret_cast<BatchCtl*>(b->dev);
  const uint64_t* beg = reinterpret_cast<const uint64_t*>(b->dev + b->off_begins);
  const BatchItemDev* it = reinterpret_cast<const BatchItemDev*>(b->dev + b->off_items);
  uint2* q = reinterpret_cast<uint2*>(b->dev + b->off_queue);
  CFB_CUDA(v.tiles(ctl, it, beg, q, grid_of(v.tiles_fn, v.block), s));
  if (b->has_insert || always_evict)
    CFB_CUDA(v.evict(ctl, it, q, grid_of(v.evict_fn, cfk::kBlock), s));
  return CF_OK;
}

cf_status order_filters(cf_batch* b, cudaStream_t s) {
  for (cf_filter* f : b->filters) {
    cf_status st = cfk::order_on(f, s);
    if (st != CF_OK) return st;
  }
  return CF_OK;
}

void mark_filters(cf_batch* b, cudaStream_t s) {
  for (cf_filter* f : b->filters) cfk::mark_external(f, s, b->done_ev);
}

ClassKey class_of(const cf_batch* b) {
  return ClassKey{b->f, b->b, b->policy, b->op_mask, ilog2(b->total_keys + 1),
                  ilog2(uint64_t(b->n_items) + 1)};
}

}  // namespace

extern "C" {

cf_status cf_batch_create(uint32_t max_items, uint64_t max_keys, cf_batch** out) {
  if (!out || max_items == 0 || max_keys == 0) return CF_EINVAL;
  *out = nullptr;
  cf_batch* b = new cf_batch();
  b->max_items = max_items;
  b->max_keys = max_keys;
  cudaGetDevice(&b->device);
  b->off_begins = sizeof(BatchCtl);
  b->off_items = align256(b->off_begins + (size_t(max_items) + 1) * sizeof(uint64_t));
  b->desc_bytes = align256(b->off_items + size_t(max_items) * sizeof(BatchItemDev));
  b->off_queue = b->desc_bytes;
  b->dev_bytes = b->off_queue + size_t(max_keys) * sizeof(uint2);
  if (cudaMalloc(&b->dev, b->dev_bytes) != cudaSuccess ||
      cudaMallocHost(&b->host, b->desc_bytes) != cudaSuccess) {
    cudaGetLastError();
    cf_batch_destroy(b);
    cfk::set_error_text("cf_batch_create: allocation failed");
    return CF_ENOMEM;
  }
  std::memset(b->host, 0, b->desc_bytes);
  if (cudaEventCreateWithFlags(&b->upload_ev, cudaEventDisableTiming) != cudaSuccess) {
    cf_batch_destroy(b);
    return CF_ECUDA;
  }
  b->done_ev = cfk::pooled_event();
  *out = b;
  return CF_OK;
}

cf_status cf_batch_destroy(cf_batch* b) {
  if (!b) return CF_OK;
  if (b->done_ev) cudaEventSynchronize(b->done_ev);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->upload_ev) cudaEventDestroy(b->upload_ev);
  if (b->dev) cudaFree(b->dev);
  if (b->host) cudaFreeHost(b->host);
  // done_ev stays alive: filters may still refer to it for ordering.
  delete b;
  return CF_OK;
}

cf_status cf_batch_set(cf_batch* b, const cf_batch_item* items, uint32_t n_items) {
  if (!b || (n_items && !items)) return CF_EINVAL;
  if (n_items > b->max_items) {
    cfk::set_error_text("cf_batch_set: more items than the plan's max_items");
    return CF_EINVAL;
  }
  cf_status st = wait_upload(b);
  if (st != CF_OK) return st;
  int f = -1, bb = -1, pol = -1, mask = 0;
  uint64_t total = 0;
  bool ins = false;
  std::unordered_map<cf_filter*, int> cls;
  std::vector<cf_filter*> filters;
  for (uint32_t i = 0; i < n_items; ++i) {
    const cf_batch_item& x = items[i];
    if (!x.filter || x.op > CF_OP_REMOVE) return CF_EINVAL;
    if (x.n && !x.keys) return CF_EINVAL;
    if (x.op == CF_OP_CONTAINS && x.n && !x.out_flags) return CF_EINVAL;
    if (x.n >= (1ull << 32)) return CF_EINVAL;
    const cf_config& c = x.filter->cfg;
    if (f < 0) {
      f = int(c.fp_bits);
      bb = int(c.slots_per_bucket);
      pol = int(c.policy);
    } else if (f != int(c.fp_bits) || bb != int(c.slots_per_bucket) ||
               pol != int(c.policy)) {
      cfk::set_error_text("cf_batch_set: filters of different geometries");
      return CF_EINVAL;
    }
    const int k = (x.op == CF_OP_CONTAINS) ? 1 : 2;
    auto it = cls.find(x.filter);
    if (it == cls.end()) {
      cls.emplace(x.filter, k);
      filters.push_back(x.filter);
    } else if (it->second != k) {
      cfk::set_error_text("cf_batch_set: a filter is both queried and mutated");
      return CF_EINVAL;
    }
    total += x.n;
    mask |= 1 << x.op;
    ins = ins || (x.op == CF_OP_INSERT && x.n);
  }
  if (total > b->max_keys) {
    cfk::set_error_text("cf_batch_set: more keys than the plan's max_keys");
    return CF_EINVAL;
  }
  b->items.assign(items, items + n_items);
  b->filters.swap(filters);
  b->n_items = n_items;
  b->total_keys = total;
  b->has_insert = ins;
  b->op_mask = mask;
  if (n_items == 0) {
    b->n_tiles = 0;
    return CF_OK;
  }
  if (f != b->f || bb != b->b || pol != b->policy) {
    b->variants = cfk::batch_variants(f, bb, pol, &b->n_variants);
    if (!b->variants || b->n_variants == 0) return CF_ENOTSUP;
    b->f = f;
    b->b = bb;
    b->policy = pol;
    if (b->pinned_variant >= b->n_variants) b->pinned_variant = -1;
  }
  int v = 0;
  if (b->pinned_variant >= 0) {
    v = b->pinned_variant;
  } else {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(class_of(b));
    if (it != g_tuned.end() && it->second < b->n_variants) v = it->second;
  }
  b->variant = v;
  restage(b);
  return CF_OK;
}

cf_status cf_batch_launch(cf_batch* b, void* stream) {
  if (!b) return CF_EINVAL;
  if (b->n_items == 0) return CF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cf_status st = order_filters(b, s);
  if (st != CF_OK) return st;
  st = enqueue(b, s, false);
  if (st != CF_OK) return st;
  CFB_CUDA(cudaEventRecord(b->upload_ev, s));
  CFB_CUDA(cudaEventRecord(b->done_ev, s));
  b->pending = true;
  mark_filters(b, s);
  return CF_OK;
}

cf_status cf_batch_graph_launch(cf_batch* b, void* stream) {
  if (!b) return CF_EINVAL;
  if (b->n_items == 0) return CF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->gexec || b->graph_variant != b->variant) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    // Capture on a private stream so the caller's stream state is untouched.
    cudaStream_t cs;
    CFB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cf_status st = CF_OK;
    if (e == cudaSuccess) {
      st = enqueue(b, cs, /*always_evict=*/true);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (st == CF_OK && e2 != cudaSuccess) {
        cfk::set_error("cudaStreamEndCapture", e2);
        st = CF_ECUDA;
      }
      b->graph = g;
    } else {
      cfk::set_error("cudaStreamBeginCapture", e);
      st = CF_ECUDA;
    }
    cudaStreamDestroy(cs);
    if (st != CF_OK) return st;
    CFB_CUDA(cudaGraphInstantiate(&b->gexec, b->graph, 0));
    b->graph_variant = b->variant;
  }
  cf_status st = order_filters(b, s);
  if (st != CF_OK) return st;
  CFB_CUDA(cudaGraphLaunch(b->gexec, s));
  CFB_CUDA(cudaEventRecord(b->upload_ev, s));
  CFB_CUDA(cudaEventRecord(b->done_ev, s));
  b->pending = true;
  mark_filters(b, s);
  return CF_OK;
}

cf_status cf_batch_set_variant(cf_batch* b, uint32_t variant) {
  if (!b) return CF_EINVAL;
  if (b->variants && int(variant) >= b->n_variants) return CF_EINVAL;
  cf_status st = wait_upload(b);
  if (st != CF_OK) return st;
  b->pinned_variant = int(variant);
  if (b->variants && b->n_items) {
    b->variant = int(variant);
    restage(b);
  }
  return CF_OK;
}

uint32_t cf_batch_variant_count(const cf_batch* b) {
  return (b && b->variants) ? uint32_t(b->n_variants) : 0u;
}

cf_status cf_batch_get_tuning(const cf_batch* b, cf_tuning* out) {
  if (!b || !out || !b->variants) return CF_EINVAL;
  const BatchVariant& v = b->variants[b->variant];
  out->variant = uint32_t(b->variant);
  out->keys_per_thread = uint32_t(v.keys_per_thread);
  out->block = uint32_t(v.block);
  out->frontier = uint32_t(v.frontier);
  out->ms = b->tuned_ms;
  return CF_OK;
}

cf_status cf_batch_autotune(cf_batch* b, void* stream, cf_tuning* chosen) {
  if (!b || b->n_items == 0 || !b->variants) return CF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CFB_CUDA(cudaEventSynchronize(b->done_ev));
  b->pending = false;
  // Save every filter's device state (control block, victim log, table).
  size_t total = 0;
  for (cf_filter* f : b->filters) total += align256(f->mem_bytes);
  char* save = nullptr;
  if (cudaMalloc(&save, total) != cudaSuccess) {
    cudaGetLastError();
    cfk::set_error_text("cf_batch_autotune: no room to save the filters' state");
    return CF_ENOMEM;
  }
  auto copy_all = [&](bool to_save) -> cudaError_t {
    size_t off = 0;
    for (cf_filter* f : b->filters) {
      cudaError_t e = to_save
          ? cudaMemcpyAsync(save + off, f->mem, f->mem_bytes, cudaMemcpyDeviceToDevice, s)
          : cudaMemcpyAsync(f->mem, save + off, f->mem_bytes, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
      off += align256(f->mem_bytes);
    }
    return cudaSuccess;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cf_status st = CF_OK;
  int best = b->variant;
  float best_ms = 1e30f;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = copy_all(true);
  for (int v = 0; v < b->n_variants && e == cudaSuccess && st == CF_OK; ++v) {
    b->variant = v;
    restage(b);
    e = copy_all(false);  // warm-up run on the saved state
    if (e != cudaSuccess) break;
    st = enqueue(b, s, false);
    if (st != CF_OK) break;
    e = cudaStreamSynchronize(s);  // the staging buffer is reused below
    if (e != cudaSuccess) break;
    e = copy_all(false);
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, s);
    st = enqueue(b, s, false);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  if (e == cudaSuccess) e = copy_all(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(save);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cfk::set_error("cf_batch_autotune", e);
    return CF_ECUDA;
  }
  if (st != CF_OK) return st;
  b->variant = best;
  b->tuned_ms = best_ms;
  restage(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[class_of(b)] = best;
  }
  CFB_CUDA(cudaEventRecord(b->done_ev, s));
  mark_filters(b, s);
  if (chosen) return cf_batch_get_tuning(b, chosen);
  return CF_OK;
}

}  // extern "C"
