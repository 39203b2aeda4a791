// Launch sequence of the slice-partitioned passes (cf_slice.cuh) and the
// eviction levels (cf_levels.cuh), and the per-geometry table of launchers.
#pragma once

#include "cf_levels.cuh"

namespace cfk {

// ---------------------------------------------------------------------------
// Launch sequence of one chunk.
// ---------------------------------------------------------------------------
// Dynamic shared memory near or above the 48 KB default (static shared
// memory counts against it too) needs the kernel's opt-in.
inline cudaError_t smem_opt_in(const void* fn, size_t bytes) {
  if (bytes <= 40 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

template <class G>
struct SliceLaunch {
  static constexpr int KQ = Tiles<G, false>::K;
  // Keys per round: the query's K for insert (unless CF_SLICE_KMUT caps
  // it), half of it (at most 4) for delete.
  static constexpr int KMS = (CF_SLICE_KMUT > 0 && CF_SLICE_KMUT < KQ) ? CF_SLICE_KMUT : KQ;
  static constexpr int KRM = CF_SLICE_KMUT > 0 ? KMS : (KQ >= 8 ? 4 : KQ);
  static constexpr int U = 16;  // keys per thread of a scatter tile

  template <int OP, int K>
  static cudaError_t probes(const DevFilter& d, const SliceBufs& sb, uint64_t n,
                            int want, uint32_t* queue, cudaStream_t s,
                            KernelTimer* t) {
    constexpr uint32_t T = kSliceBlock * 8;
    const size_t smem = size_t(20) * T + size_t(24) * sb.n_slices + 16;
    const bool rt = d.max_cas != kMaxCas;
    auto p1 = rt ? k_slice_probe1<G, OP, K, true> : k_slice_probe1<G, OP, K>;
    cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(p1), smem);
    if (e != cudaSuccess) return e;
    if (t) t->begin(KK_SLICE_PROBE1, s);
    p1<<<persistent_grid(p1, n, T, kSliceBlock), kSliceBlock, smem, s>>>(d, sb, want);
    if (t) t->end(KK_SLICE_PROBE1, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto p2 = rt ? k_slice_probe2<G, OP, K, true> : k_slice_probe2<G, OP, K>;
    const size_t smem2 = size_t(2) * (sb.n_slices + 1) * sizeof(uint32_t);
    if (t) t->begin(KK_SLICE_PROBE2, s);
    p2<<<persistent_grid(p2, n, kSliceBlock * 8, kSliceBlock), kSliceBlock, smem2, s>>>(
        d, sb, n, want, queue);
    if (t) t->end(KK_SLICE_PROBE2, s);
    return cudaGetLastError();
  }

  // The eviction levels (cf_levels.cuh): counters to zero, the seed and L
  // level launches (timed together as KK_EVICT_LEVEL), and the resume
  // (timed with the eviction loop, KK_INSERT_EVICT).  Each launch decides
  // on the device whether it has work; with the levels off they all return
  // at once and the eviction loop launched after them takes the queue.
  static cudaError_t levels(const DevFilter& d, const SliceBufs& sb, uint32_t* queue,
                            const EvictMap& em, uint8_t* f2, cudaStream_t s, KernelTimer* t) {
    const LevelBufs& lb = em.lv;
    const uint32_t S = sb.n_slices;
    const size_t ctr_bytes = reinterpret_cast<const char*>(lb.ctl + lb.n_levels + 2) -
                             reinterpret_cast<const char*>(lb.fill);
    cudaError_t e = cudaMemsetAsync(lb.fill, 0, ctr_bytes, s);
    if (e != cudaSuccess) return e;
    constexpr uint32_t TS = kBlock * 4;
    auto fs = k_evict_seed<G>;
    const size_t smem_s = lv_split_bytes<TS>(S);
    e = smem_opt_in(reinterpret_cast<const void*>(fs), smem_s);
    if (e != cudaSuccess) return e;
    auto fl = k_evict_level<G>;
    const size_t smem_l = lv_split_bytes<LvTile<G>::T>(S) + size_t(12) * (S + 2);
    e = smem_opt_in(reinterpret_cast<const void*>(fl), smem_l);
    if (e != cudaSuccess) return e;
    const unsigned grid_s = persistent_grid(fs, ~0ull >> 1, 1);
    const unsigned grid_l = persistent_grid(fl, ~0ull >> 1, 1);
    if (t) t->begin(KK_EVICT_LEVEL, s);
    fs<<<grid_s, kBlock, smem_s, s>>>(d, sb.rec2, queue, em.bits, em.min_q, lb, S, sb.shift, f2);
    for (uint32_t k = 0; k < lb.n_levels; ++k)
      fl<<<grid_l, kBlock, smem_l, s>>>(d, em.bits, lb, S, sb.shift, k, f2);
    if (t) t->end(KK_EVICT_LEVEL, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto fr = k_evict_resume<G>;
    if (t) t->begin(KK_INSERT_EVICT, s);
    fr<<<evict_grid(reinterpret_cast<const void*>(fr), true), kBlock,
         size_t(8) * (S + 1), s>>>(d, em.bits, lb, S, f2);
    if (t) t->end(KK_INSERT_EVICT, s);
    return cudaGetLastError();
  }

  // A pass in three parts, so that a pass's keys can arrive in pieces (the
  // host-buffer calls scatter each staging chunk as its copy lands):
  // begin (counters to zero), scatter (any number of times, each for keys
  // [dst_off, dst_off + n) of the pass), finish (everything after the split).
  static cudaError_t begin(const SliceBufs& sb, cudaStream_t s) {
    // fill1 and fill2 (and the tile counters after it) share one range.
    const size_t ctr_bytes = reinterpret_cast<const char*>(
                                 sb.fill2 + (sb.n_slices + kFill2Extra) * kCtrStride) -
                             reinterpret_cast<const char*>(sb.fill1);
    return cudaMemsetAsync(sb.fill1, 0, ctr_bytes, s);
  }

  static cudaError_t scatter(const DevFilter& d, const uint64_t* keys, uint64_t n,
                             uint64_t dst_off, int want, const SliceBufs& sb,
                             cudaStream_t s, KernelTimer* t) {
    auto fs = k_slice_scatter<G, U>;
    const size_t smem = size_t(8) * kBlock * U + size_t(16) * sb.n_slices;
    cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(fs), smem);
    if (e != cudaSuccess) return e;
    if (t) t->begin(KK_SLICE_SPLIT, s);
    fs<<<persistent_grid(fs, n, kBlock * U), kBlock, smem, s>>>(
        d, keys, n, sb, want ? sb.dst + dst_off : nullptr);
    if (t) t->end(KK_SLICE_SPLIT, s);
    return cudaGetLastError();
  }

  static cudaError_t finish(const DevFilter& d, int op, uint64_t n, uint8_t* flags,
                            const SliceBufs& sb, uint32_t* queue, const EvictMap& em,
                            cudaStream_t s, KernelTimer* t) {
    const int want = flags != nullptr;
    const uint32_t S = sb.n_slices;
    cudaError_t e;
    // All three operations take the query's K (8 for 8-byte buckets): the
    // bucket accesses hit L2 here, so the mutating passes are latency-bound
    // and want every key's load and CAS of a tile in flight together.
    if (op == SOP_CONTAINS)
      e = probes<SOP_CONTAINS, KQ>(d, sb, n, want, queue, s, t);
    else if (op == SOP_REMOVE)
      e = probes<SOP_REMOVE, KRM>(d, sb, n, want, queue, s, t);
    else
      e = probes<SOP_INSERT, KMS>(d, sb, n, want, queue, s, t);
    if (e != cudaSuccess) return e;
    if (op == SOP_INSERT) {
      e = Launch<G>::fullmap(d, em, s, t);
      if (e != cudaSuccess) return e;
      const bool lv = em.bits && em.lv.rec[0];
      if (lv) {
        e = levels(d, sb, queue, em, want ? sb.f2 : nullptr, s, t);
        if (e != cudaSuccess) return e;
      }
      auto fe = k_insert_evict<G, true>;
      if (t) t->begin(KK_INSERT_EVICT, s);
      fe<<<evict_grid(reinterpret_cast<const void*>(fe), em.bits != nullptr), kBlock, 0, s>>>(
          d, sb.rec2, want ? sb.f2 : nullptr, nullptr, queue, em.bits, em.min_q,
          lv ? em.lv.ctl : nullptr);
      if (t) t->end(KK_INSERT_EVICT, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    if (!want) return cudaSuccess;
    if (t) t->begin(KK_SLICE_MERGE, s);
    k_slice_merge<<<persistent_grid(k_slice_merge, n, kBlock * 4 * CF_MERGE_V), kBlock,
                    size_t(12) * (S + 2), s>>>(sb);
    k_slice_out<<<persistent_grid(k_slice_out, n, kBlock * 4 * CF_MERGE_V), kBlock, 0, s>>>(
        sb.dst, sb.f1, flags, n);
    if (t) t->end(KK_SLICE_MERGE, s);
    return cudaGetLastError();
  }

  static cudaError_t run(const DevFilter& d, int op, const uint64_t* keys,
                         uint64_t n, uint8_t* flags, const SliceBufs& sb,
                         uint32_t* queue, const EvictMap& em, cudaStream_t s,
                         KernelTimer* t) {
    cudaError_t e = begin(sb, s);
    if (e != cudaSuccess) return e;
    e = scatter(d, keys, n, 0, flags != nullptr, sb, s, t);
    if (e != cudaSuccess) return e;
    return finish(d, op, n, flags, sb, queue, em, s, t);
  }
};

template <class G>
const Ops* ops_for() {
  static const Ops o = {&Launch<G>::contains,     &Launch<G>::remove,
                        &Launch<G>::insert_chunk, &Launch<G>::insert_serial,
                        &Launch<G>::hash,         &Launch<G>::count,
                        &SliceLaunch<G>::run,     &SliceLaunch<G>::begin,
                        &SliceLaunch<G>::scatter, &SliceLaunch<G>::finish,
                        &Launch<G>::touch};
  return &o;
}

}  // namespace cfk
