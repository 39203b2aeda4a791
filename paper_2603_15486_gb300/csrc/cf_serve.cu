// Serving loop with continuous batching (cf_server_* in include/cf.h), the
// trace replayer used to measure it, and the plain one-request-at-a-time
// baseline.
//
// A scheduler thread owns every GPU-side step.  Each pass it
//   1. retires finished waves (cudaEventQuery, never blocking), stamping
//      their requests' completion time and the watchdog verdict;
//   2. closes filters whose removal was requested once their work is done;
//   3. admits waiting filters, oldest first, while they fit the budget;
//   4. fills every free wave slot: round-robin over the live filters with
//      no work in flight, it takes each one's oldest queued requests of one
//      kind, up to the wave's item and key limits, and launches them as one
//      multi-filter launch on the slot's own stream (a wave of one query or
//      delete runs the single-filter kernel instead, which has less to set
//      up than the multi-filter launch).
// Several waves are on the GPU at once, so requests that arrive while
// others run start as soon as a slot frees up, and their kernels overlap.
// Latency: while waves are on the GPU the scheduler polls their events
// without sleeping, and after any activity it keeps polling for new
// requests for kSpinIdle before it sleeps on its condition variable (a
// sleep and wake-up costs tens of microseconds, more than a small
// request's kernels).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cf.h"
#include "cf_internal.h"

namespace {

// How long the scheduler keeps polling for new requests after its last
// activity before it sleeps.
constexpr double kSpinIdle = 2e-3;

double now_s() {
  return std::chrono::duration<double>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t id = 0;
  cf_request r{};
  double submit_s = 0, launch_s = 0;
  uint32_t wave_size = 0;
  int64_t trace_index = -1;
};

struct FSlot {
  uint32_t id = 0;
  cf_config cfg{};
  size_t bytes = 0;
  cf_filter* f = nullptr;
  int32_t state = CF_FILTER_PENDING;
  std::deque<Req*> q;
  bool inflight = false;
  bool remove_requested = false;
};

struct WaveSlot {
  cf_batch* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<Req*> reqs;
  std::vector<uint32_t> fids;
  std::vector<cf_batch_item> items;
  bool busy = false;
  double launch_s = 0;
};

}  // namespace

struct cf_server {
  cf_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler
  std::condition_variable cv_done;  // wakes drain()
  std::unordered_map<uint32_t, FSlot*> filters;
  std::vector<uint32_t> order;      // round-robin order of filter ids
  size_t rr = 0;
  uint32_t next_fid = 1;
  std::deque<uint32_t> admission;
  uint64_t used = 0;
  std::vector<WaveSlot> waves;
  std::deque<cf_completion> done;
  cf_completion* trace_out = nullptr;
  uint64_t next_req = 1, submitted = 0, completed = 0, n_waves = 0, late = 0;
  uint64_t keys_done = 0;
  bool stop = false;
  std::atomic<uint64_t> kicks{0};  // bumped by every submit / add / remove
  std::thread worker;
};

namespace {

void complete(cf_server* s, Req* r, double t, int32_t status) {
  cf_completion c{};
  c.request_id = r->id;
  c.tag = r->r.tag;
  c.status = status;
  c.wave_size = r->wave_size;
  c.submit_s = r->submit_s;
  c.launch_s = r->launch_s;
  c.done_s = t;
  if (r->trace_index >= 0 && s->trace_out)
    s->trace_out[r->trace_index] = c;
  else
    s->done.push_back(c);
  s->completed++;
  s->keys_done += r->r.n;
  delete r;
}

bool retire_waves(cf_server* s) {
  bool any = false;
  for (auto& w : s->waves) {
    if (!w.busy) continue;
    const cudaError_t q = cudaEventQuery(w.done);
    if (q == cudaErrorNotReady) continue;
    const double t = now_s();
    const bool late = s->cfg.watchdog_us &&
                      (t - w.launch_s) * 1e6 > double(s->cfg.watchdog_us);
    if (late) s->late++;
    const int32_t st = q != cudaSuccess ? CF_ECUDA : (late ? CF_ETIMEOUT : CF_OK);
    for (Req* r : w.reqs) complete(s, r, t, st);
    for (uint32_t fid : w.fids) {
      auto it = s->filters.find(fid);
      if (it != s->filters.end()) it->second->inflight = false;
    }
    w.reqs.clear();
    w.fids.clear();
    w.busy = false;
    any = true;
  }
  if (any) s->cv_done.notify_all();
  return any;
}

bool close_filters(cf_server* s) {
  bool any = false;
  for (auto& kv : s->filters) {
    FSlot* fs = kv.second;
    if (!fs->remove_requested || fs->state == CF_FILTER_CLOSED) continue;
    if (fs->inflight || !fs->q.empty()) {
      if (fs->state == CF_FILTER_LIVE) fs->state = CF_FILTER_CLOSING;
      continue;
    }
    if (fs->f) {
      cf_destroy(fs->f);
      fs->f = nullptr;
      s->used -= fs->bytes;
    }
    fs->state = CF_FILTER_CLOSED;
    any = true;
  }
  return any;
}

bool admit(cf_server* s) {
  bool any = false;
  while (!s->admission.empty()) {
    FSlot* fs = s->filters[s->admission.front()];
    // A filter removed before admission still runs the requests queued for
    // it (it closes after them); with none queued it closes unallocated.
    if (fs->state != CF_FILTER_PENDING || (fs->remove_requested && fs->q.empty())) {
      s->admission.pop_front();
      continue;
    }
    if (s->used + fs->bytes > s->cfg.hbm_budget_bytes) break;
    cf_filter* f = nullptr;
    const cf_status st = cf_create_ex(&fs->cfg, &f);
    s->admission.pop_front();
    any = true;
    if (st != CF_OK) {
      // Out of device memory despite the budget: fail its requests.
      fs->state = CF_FILTER_CLOSED;
      const double t = now_s();
      while (!fs->q.empty()) {
        complete(s, fs->q.front(), t, st);
        fs->q.pop_front();
      }
      s->cv_done.notify_all();
      continue;
    }
    // Waves of one query or delete run the single-filter kernels; keep them
    // on the plain path, which needs no scratch memory (no allocation, and
    // so no implicit device synchronisation, inside the scheduler).
    cf_set_slicing(f, 0, 0, 0);
    fs->f = f;
    fs->state = CF_FILTER_LIVE;
    s->used += fs->bytes;
  }
  return any;
}

// Fill one free wave slot; false if nothing could be scheduled.
bool fill_wave(cf_server* s, WaveSlot& w) {
  const size_t nf = s->order.size();
  uint64_t keys = 0;
  for (size_t step = 0; step < nf && w.reqs.size() < s->cfg.max_wave_items; ++step) {
    const uint32_t fid = s->order[(s->rr + step) % nf];
    FSlot* fs = s->filters[fid];
    if (fs->state != CF_FILTER_LIVE && fs->state != CF_FILTER_CLOSING) continue;
    if (fs->inflight || fs->q.empty()) continue;
    const uint32_t op = fs->q.front()->r.op;
    bool took = false;
    while (!fs->q.empty() && w.reqs.size() < s->cfg.max_wave_items) {
      Req* r = fs->q.front();
      if (r->r.op != op) break;
      if (keys + r->r.n > s->cfg.max_wave_keys && !w.reqs.empty()) break;
      keys += r->r.n;
      w.reqs.push_back(r);
      fs->q.pop_front();
      took = true;
    }
    if (took) {
      fs->inflight = true;
      w.fids.push_back(fid);
    }
    if (keys >= s->cfg.max_wave_keys) break;
  }
  if (nf) s->rr = (s->rr + 1) % nf;
  return !w.reqs.empty();
}

cf_status launch_wave(cf_server* s, WaveSlot& w) {
  cf_status st = CF_OK;
  const cf_request& r0 = w.reqs[0]->r;
  if (w.reqs.size() == 1 && r0.op != CF_OP_INSERT) {
    // One query or delete: the single-filter kernel on the slot's stream
    // (the filter's call ordering holds across the two launch forms).
    cf_filter* f = s->filters[r0.filter_id]->f;
    st = r0.op == CF_OP_CONTAINS ? cf_contains(f, r0.keys, r0.n, r0.out_flags, w.stream)
                                 : cf_remove(f, r0.keys, r0.n, r0.out_flags, w.stream);
  } else {
    w.items.resize(w.reqs.size());
    for (size_t i = 0; i < w.reqs.size(); ++i) {
      const cf_request& r = w.reqs[i]->r;
      w.items[i] = cf_batch_item{s->filters[r.filter_id]->f, r.keys, r.n, r.out_flags,
                                 r.op, 0};
    }
    st = cf_batch_set(w.plan, w.items.data(), uint32_t(w.items.size()));
    if (st == CF_OK)
      st = s->cfg.use_graphs ? cf_batch_graph_launch(w.plan, w.stream)
                             : cf_batch_launch(w.plan, w.stream);
  }
  if (st == CF_OK && cudaEventRecord(w.done, w.stream) != cudaSuccess) st = CF_ECUDA;
  const double t = now_s();
  if (st != CF_OK) {
    for (Req* r : w.reqs) complete(s, r, t, st);
    for (uint32_t fid : w.fids) s->filters[fid]->inflight = false;
    w.reqs.clear();
    w.fids.clear();
    s->cv_done.notify_all();
    return st;
  }
  for (Req* r : w.reqs) {
    r->launch_s = t;
    r->wave_size = uint32_t(w.reqs.size());
  }
  w.busy = true;
  w.launch_s = t;
  s->n_waves++;
  return CF_OK;
}

bool has_queued(const cf_server* s) {
  for (const auto& kv : s->filters)
    if (!kv.second->q.empty()) return true;
  return false;
}

void worker_main(cf_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  double last_active = now_s();
  for (;;) {
    const uint64_t kicks = s->kicks.load(std::memory_order_acquire);
    bool progressed = retire_waves(s);
    progressed |= close_filters(s);
    progressed |= admit(s);
    for (auto& w : s->waves) {
      if (w.busy) continue;
      if (!fill_wave(s, w)) break;
      launch_wave(s, w);
      progressed = true;
    }
    bool busy = false;
    for (const auto& w : s->waves) busy = busy || w.busy;
    if (s->stop && !busy && !has_queued(s)) break;
    if (progressed) {
      last_active = now_s();
      continue;
    }
    // Nothing to do right now.  Poll (with the lock released, so that
    // submitters get in) while waves are on the GPU or shortly after the
    // last activity; otherwise sleep until a submit wakes us.
    if (busy || now_s() - last_active < kSpinIdle) {
      lk.unlock();
      for (int i = 0; i < 64 && s->kicks.load(std::memory_order_acquire) == kicks; ++i)
        std::this_thread::yield();
      lk.lock();
      if (busy) last_active = now_s();
    } else {
      s->cv.wait_for(lk, std::chrono::milliseconds(50),
                     [&] { return s->kicks.load(std::memory_order_acquire) != kicks || s->stop; });
      last_active = now_s();
    }
  }
}

cf_status submit_locked(cf_server* s, const cf_request* r, int64_t trace_index,
                        double submit_s, uint64_t* id) {
  auto it = s->filters.find(r->filter_id);
  if (it == s->filters.end() || it->second->state == CF_FILTER_CLOSED ||
      it->second->remove_requested)
    return CF_EINVAL;
  if (r->op > CF_OP_REMOVE || r->n > s->cfg.max_wave_keys) return CF_EINVAL;
  if (r->n && !r->keys) return CF_EINVAL;
  if (r->op == CF_OP_CONTAINS && r->n && !r->out_flags) return CF_EINVAL;
  Req* q = new Req();
  q->id = s->next_req++;
  q->r = *r;
  q->submit_s = submit_s;
  q->trace_index = trace_index;
  it->second->q.push_back(q);
  s->submitted++;
  s->kicks.fetch_add(1, std::memory_order_release);
  if (id) *id = q->id;
  return CF_OK;
}

}  // namespace

extern "C" {

cf_status cf_server_create(const cf_server_config* cfg, cf_server** out) {
  if (!cfg || !out || cfg->max_inflight == 0 || cfg->max_wave_items == 0 ||
      cfg->max_wave_keys == 0)
    return CF_EINVAL;
  *out = nullptr;
  cf_server* s = new cf_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->waves.resize(cfg->max_inflight);
  for (auto& w : s->waves) {
    cf_status st = cf_batch_create(cfg->max_wave_items, cfg->max_wave_keys, &w.plan);
    if (st == CF_OK && cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess)
      st = CF_ECUDA;
    if (st == CF_OK && cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess)
      st = CF_ECUDA;
    if (st != CF_OK) {
      cf_server_destroy(s);
      return st;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return CF_OK;
}

cf_status cf_server_destroy(cf_server* s) {
  if (!s) return CF_OK;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->kicks.fetch_add(1, std::memory_order_release);
    }
    s->cv.notify_all();
    s->worker.join();
  }
  for (auto& w : s->waves) {
    if (w.plan) cf_batch_destroy(w.plan);
    if (w.done) cudaEventDestroy(w.done);
    if (w.stream) cudaStreamDestroy(w.stream);
  }
  for (auto& kv : s->filters) {
    if (kv.second->f) cf_destroy(kv.second->f);
    for (Req* r : kv.second->q) delete r;
    delete kv.second;
  }
  delete s;
  return CF_OK;
}

cf_status cf_server_add_filter(cf_server* s, const cf_config* cfg, uint32_t* filter_id) {
  if (!s || !cfg || !filter_id) return CF_EINVAL;
  const size_t bytes = cf_required_bytes(cfg);
  if (bytes == 0) return CF_EINVAL;
  if (bytes > s->cfg.hbm_budget_bytes) return CF_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  FSlot* fs = new FSlot();
  fs->id = s->next_fid++;
  fs->cfg = *cfg;
  fs->bytes = bytes;
  s->filters[fs->id] = fs;
  s->order.push_back(fs->id);
  s->admission.push_back(fs->id);
  *filter_id = fs->id;
  s->kicks.fetch_add(1, std::memory_order_release);
  s->cv.notify_all();
  return CF_OK;
}

cf_status cf_server_remove_filter(cf_server* s, uint32_t filter_id) {
  if (!s) return CF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->filters.find(filter_id);
  if (it == s->filters.end()) return CF_EINVAL;
  it->second->remove_requested = true;
  s->kicks.fetch_add(1, std::memory_order_release);
  s->cv.notify_all();
  return CF_OK;
}

cf_status cf_server_filter_state(cf_server* s, uint32_t filter_id, int32_t* state) {
  if (!s || !state) return CF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->filters.find(filter_id);
  if (it == s->filters.end()) return CF_EINVAL;
  *state = it->second->state;
  return CF_OK;
}

cf_filter* cf_server_get_filter(cf_server* s, uint32_t filter_id) {
  if (!s) return nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->filters.find(filter_id);
  if (it == s->filters.end() || it->second->state != CF_FILTER_LIVE) return nullptr;
  return it->second->f;
}

cf_status cf_server_submit(cf_server* s, const cf_request* r, uint64_t* request_id) {
  if (!s || !r) return CF_EINVAL;
  cf_status st;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    st = submit_locked(s, r, -1, now_s(), request_id);
  }
  if (st == CF_OK) s->cv.notify_all();
  return st;
}

uint32_t cf_server_poll(cf_server* s, cf_completion* out, uint32_t max) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

cf_status cf_server_drain(cf_server* s, uint32_t timeout_ms) {
  if (!s) return CF_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.notify_all();
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                      [s] { return s->completed == s->submitted; });
  return ok ? CF_OK : CF_ETIMEOUT;
}

cf_status cf_server_stats(cf_server* s, cf_server_stats_t* out) {
  if (!s || !out) return CF_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->waves = s->n_waves;
  out->late_waves = s->late;
  out->keys_completed = s->keys_done;
  out->used_bytes = s->used;
  uint32_t live = 0, pending = 0;
  for (const auto& kv : s->filters) {
    live += kv.second->state == CF_FILTER_LIVE;
    pending += kv.second->state == CF_FILTER_PENDING;
  }
  out->live_filters = live;
  out->pending_filters = pending;
  return CF_OK;
}

cf_status cf_server_run_trace(cf_server* s, const cf_request* reqs,
                              const double* arrival_s, uint32_t n,
                              cf_completion* out) {
  if (!s || (n && (!reqs || !arrival_s || !out))) return CF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->trace_out) return CF_EBUSY;
    if (s->completed != s->submitted) return CF_EBUSY;  // drain first
    s->trace_out = out;
  }
  cf_status st = CF_OK;
  const double t0 = now_s();
  for (uint32_t i = 0; i < n && st == CF_OK; ++i) {
    const double target = t0 + arrival_s[i];
    for (double t = now_s(); t < target; t = now_s()) {
      if (target - t > 200e-6)
        std::this_thread::sleep_for(std::chrono::duration<double>(target - t - 100e-6));
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      st = submit_locked(s, &reqs[i], int64_t(i), target, nullptr);
    }
    s->cv.notify_all();
  }
  const cf_status dr = cf_server_drain(s, 600000);
  std::lock_guard<std::mutex> lk(s->mu);
  s->trace_out = nullptr;
  return st != CF_OK ? st : dr;
}

cf_status cf_plain_run_trace(cf_filter* const* filters, uint32_t n_filters,
                             const cf_request* reqs, const double* arrival_s,
                             uint32_t n, cf_completion* out, void* stream) {
  if (n && (!filters || !reqs || !arrival_s || !out)) return CF_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double t0 = now_s();
  for (uint32_t i = 0; i < n; ++i) {
    const cf_request& r = reqs[i];
    if (r.filter_id >= n_filters || !filters[r.filter_id]) return CF_EINVAL;
    const double target = t0 + arrival_s[i];
    for (double t = now_s(); t < target; t = now_s()) {
      if (target - t > 200e-6)
        std::this_thread::sleep_for(std::chrono::duration<double>(target - t - 100e-6));
    }
    const double launch = now_s();
    cf_status s;
    switch (r.op) {
      case CF_OP_INSERT: s = cf_insert(filters[r.filter_id], r.keys, r.n, r.out_flags, st); break;
      case CF_OP_CONTAINS: s = cf_contains(filters[r.filter_id], r.keys, r.n, r.out_flags, st); break;
      case CF_OP_REMOVE: s = cf_remove(filters[r.filter_id], r.keys, r.n, r.out_flags, st); break;
      default: return CF_EINVAL;
    }
    if (s != CF_OK) return s;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CF_ECUDA;
    cf_completion& c = out[i];
    c.request_id = i;
    c.tag = r.tag;
    c.status = CF_OK;
    c.wave_size = 1;
    c.submit_s = target;
    c.launch_s = launch;
    c.done_s = now_s();
  }
  return CF_OK;
}

}  // extern "C"
