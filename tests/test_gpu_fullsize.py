"""The insert multiset invariant at full-path sizes, on the two paths that
the small parity tests do not reach at size:

* a 2^25-bucket table (f16 b4, 256 MiB) filled to LF 0.95 in three calls
  through the library's automatic choices: the slice-partitioned path with
  its default 32 MiB slices and default pass size, the full-bucket map and
  the slice-grouped eviction levels;
* a 2^24-bucket table (128 MiB) with slicing off, filled in batches below
  m/8 keys: the plain direct-insert, eviction and delete kernels in their
  DRAM-resident build (the one the serving loop runs on large filters),
  followed by a delete batch judged by the delete checker.

The stored multiset is compared with the keys' classes computed from the
oracle's hashes; the comparison sorts 64-bit class codes on the device with
torch (127 M of them do not sort quickly on the host).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import check_delete, slots_view
from gpu_util import alt_step_table, key_classes_dev, to_dev, xor_classes_dev

pytestmark = pytest.mark.gpu


def _keys_host(seed, n):
    k = torch.empty(n, dtype=torch.int64, device="cuda")
    workloads.keys_dev(k.data_ptr(), n, seed, 0, 0)
    torch.cuda.synchronize()
    return k


def _check_multiset(g, o, keys_dev, m, f, b, flags):
    kh = keys_dev.cpu().numpy().view(np.uint64)
    fp, i1, i2 = o.hash_batch(kh)
    slots = g.table_view().view({8: torch.int8, 16: torch.int16, 32: torch.int32}[f])
    slots = slots.view(m, b).to(torch.int64) & ((1 << f) - 1)
    stored = xor_classes_dev(slots, alt_step_table(o, f))
    vt, vb = g.victims()
    st = g.stats()
    assert st["victims"] == vt.size, "victim log overflowed; cannot judge"
    expect = key_classes_dev(fp, i1, i2)
    if vt.size:
        vstep = np.array([o.alt(0, int(t)) for t in vt], np.int64)
        vb64 = vb.astype(np.int64)
        vlo = np.minimum(vb64, vb64 ^ vstep)
        vcode = torch.from_numpy((vt.astype(np.int64) << 32) | vlo).cuda()
        stored = torch.sort(torch.cat([stored, vcode])).values
    assert stored.numel() == expect.numel()
    assert torch.equal(stored, expect)
    assert st["occupancy"] == int((slots != 0).sum()) == g.count_occupied()
    assert st["insert_fail"] == int((flags != 1).sum()) == vt.size
    assert st["contention"] == 0 and st["error_word"] == 0
    return st


def test_auto_path_at_2_25_buckets_multiset():
    import paper_2603_15486_gb300 as cf
    m, f, b = 1 << 25, 16, 4
    w = workloads.Workload("t", m, f, b, 500, 2, (0.5, 0.8, 0.95), 0, 0, 0)
    keys = _keys_host(2, w.n_insert)
    g = cf.CuckooFilter(m, f, b, 500, victim_capacity=1 << 20)
    g.set_kernel_timing(True)
    flags = torch.empty(w.n_insert, dtype=torch.uint8, device="cuda")
    for lo, hi in w.insert_segments():
        assert hi - lo >= m // 8            # the automatic rule picks slicing
        g.insert(keys[lo:hi], flags=flags[lo:hi])
    torch.cuda.synchronize()
    kt = g.kernel_times()
    assert kt["slice_probe1"][0] >= 3 and kt["insert_evict"][0] >= 3
    assert kt["evict_map"][0] >= 3
    o = oracle.OracleFilter(m, f, b, 500)
    st = _check_multiset(g, o, keys, m, f, b, flags.cpu().numpy())
    assert st["evictions"] > 0
    # The last fills' queues (millions of keys) take the eviction levels.
    assert kt["evict_level"][0] >= 1 and st["level_passes"] > 0


def test_plain_dram_kernels_at_2_24_buckets_multiset_and_delete():
    import paper_2603_15486_gb300 as cf
    m, f, b = 1 << 24, 16, 4
    n = (m * b * 95) // 100
    keys = _keys_host(3, n)
    g = cf.CuckooFilter(m, f, b, 500, victim_capacity=1 << 20)
    g.set_slicing("off")
    g.set_kernel_timing(True)
    flags = torch.empty(n, dtype=torch.uint8, device="cuda")
    step = 1 << 20                          # below m / 8: plain kernels
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        g.insert(keys[lo:hi], flags=flags[lo:hi])
    torch.cuda.synchronize()
    kt = g.kernel_times()
    assert kt["slice_probe1"][0] == 0 and kt["insert_direct"][0] > 0
    o = oracle.OracleFilter(m, f, b, 500)
    _check_multiset(g, o, keys, m, f, b, flags.cpu().numpy())
    # Delete 2^20 stored keys and 2^18 absent ones (plain delete kernel).
    before = slots_view(g.snapshot()[64:], m, f, b)
    dels = np.concatenate([keys[: 1 << 20].cpu().numpy().view(np.uint64),
                           workloads.keys(3, 1 << 18, start=n)])
    dfl = g.remove(to_dev(dels)).cpu().numpy()
    after = slots_view(g.snapshot()[64:], m, f, b)
    dfp, di1, di2 = o.hash_batch(dels)
    probs, n_iso = check_delete(before, after, dfp, di1, di2, dfl, 0, f)
    assert probs == [], probs
    assert n_iso > (1 << 20)
    assert int(dfl[: 1 << 20].sum()) == 1 << 20
    st = g.stats()
    assert st["occupancy"] == int(np.count_nonzero(after)) == g.count_occupied()
