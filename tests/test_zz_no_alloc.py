"""cf_insert_noalloc, the insert entry point for callers that cannot
allocate device memory (its eviction queue is a fixed array inside the
library instead of memory cudaMalloc'd on first use).

It is checked against cf_insert on the same keys, called through the C ABI,
on two calls in a row.  Placement of a parallel insert is not unique, so the
comparison uses the rule of the other insert tests: both tables hold the
same multiset of (tag, {bucket, alternate}) classes, which equals the keys'
classes (no failures at this load), and the counters and query results
agree.  This file is collected last so that a failure here does not stop
the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import AltTable, check_insert, key_classes, multiset_delta, slots_view
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _filter_in_torch_memory(cf, m, f, b):
    nbytes = cf.required_bytes(num_buckets=m, fp_bits=f, slots_per_bucket=b)
    mem = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-mem.data_ptr()) % 256
    filt = cf.CuckooFilter(m, f, b, 500, memory=mem[off: off + nbytes])
    filt._keepalive = mem
    return filt


def test_noalloc_insert_matches_insert_on_two_calls():
    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib

    L = _lib.load()
    m, f, b = 1 << 16, 16, 4
    ref = cf.CuckooFilter(m, f, b, 500)            # cf_insert
    nal = _filter_in_torch_memory(cf, m, f, b)     # cf_insert_noalloc
    o = oracle.OracleFilter(m, f, b, 500)          # hashing only
    stream = torch.cuda.current_stream()
    all_keys = []
    # Two calls in a row, the second on top of the first (LF 0.46, 0.88).
    for start, n in ((0, 120000), (120000, 110000)):
        ks = workloads.keys(71, n, start=start)
        all_keys.append(ks)
        kd = to_dev(ks)
        fa = ref.insert(kd).cpu().numpy()
        fb = torch.empty(n, dtype=torch.uint8, device="cuda")
        rc = L.cf_insert_noalloc(nal.handle, kd.data_ptr(), n, fb.data_ptr(),
                                 stream.cuda_stream)
        assert rc == 0, L.cf_last_error()
        fb = fb.cpu().numpy()
        # Same per-key outcome: every key inserted on both paths.
        assert (fa == 1).all() and (fb == 1).all()
        sa, sb = ref.stats(), nal.stats()
        for k in ("occupancy", "insert_ok", "insert_fail", "victims", "contention"):
            assert sa[k] == sb[k], k
        # Same multiset of stored classes, equal to the keys' classes.
        keys_so_far = np.concatenate(all_keys)
        fp, i1, i2 = o.hash_batch(keys_so_far)
        alt = AltTable(o, fp)
        ta = slots_view(ref.snapshot()[64:], m, f, b)
        tb = slots_view(nal.snapshot()[64:], m, f, b)
        empty = np.zeros_like(ta)
        none_t, none_b = np.empty(0, np.uint32), np.empty(0, np.uint64)
        assert check_insert(alt, empty, ta, fp, i1, i2, none_t, none_b, 0) == []
        assert check_insert(alt, empty, tb, fp, i1, i2, none_t, none_b, 0) == []
        ja, sa_ = np.nonzero(ta)
        jb, sb_ = np.nonzero(tb)
        ca = alt.classes(ja, ta[ja, sa_])
        cb = alt.classes(jb, tb[jb, sb_])
        A, _, _ = multiset_delta([(ca[0], ca[1], 1), (cb[0], cb[1], -1)])
        assert A.size == 0
        # Queries agree on every inserted key (all present on both).
        qa = ref.contains(to_dev(keys_so_far)).cpu().numpy()
        qb = nal.contains(to_dev(keys_so_far)).cpu().numpy()
        assert qa.all() and qb.all()
    # At LF 0.88 some keys found both buckets full: the eviction loop ran
    # on keys queued in the static array.
    assert nal.stats()["evictions"] > 0


def test_noalloc_full_static_queue_batch():
    """A batch of exactly CF_NOALLOC_MAX_KEYS keys on a table pre-filled to
    LF 0.45, ending at LF 0.95, so that a large share of the batch goes
    through the static queue: the insert invariants hold against the
    oracle's hashes, and the counters agree with the table."""
    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib

    L = _lib.load()
    m, f, b = 1 << 19, 16, 4
    nmax = 1 << 20
    n0 = (m * b * 95) // 100 - nmax
    nal = _filter_in_torch_memory(cf, m, f, b)
    pre = workloads.keys(72, n0)
    assert (nal.insert(to_dev(pre)).cpu().numpy() == 1).all()
    st0 = nal.stats()
    before = slots_view(nal.snapshot()[64:], m, f, b)
    ks = workloads.keys(72, nmax, start=n0)
    fl = torch.empty(nmax, dtype=torch.uint8, device="cuda")
    rc = L.cf_insert_noalloc(nal.handle, to_dev(ks).data_ptr(), nmax, fl.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.cf_last_error()
    fl = fl.cpu().numpy()
    st = nal.stats()
    o = oracle.OracleFilter(m, f, b, 500)
    fp, i1, i2 = o.hash_batch(ks)
    pfp, _, _ = o.hash_batch(pre)
    alt = AltTable(o, np.concatenate([fp, pfp]))
    after = slots_view(nal.snapshot()[64:], m, f, b)
    vt, vb = nal.victims()
    vt, vb = vt[st0["victims"]:], vb[st0["victims"]:]
    assert check_insert(alt, before, after, fp, i1, i2, vt, vb, 0) == []
    ev = st["evictions"] - st0["evictions"]
    fails = st["insert_fail"] - st0["insert_fail"]
    assert ev > nmax // 20            # many chains ran from the static queue
    assert fails == int((fl != 1).sum()) == vt.size
    assert st["occupancy"] == int(np.count_nonzero(after))
    assert st["contention"] == 0 and st["error_word"] == 0


def test_noalloc_two_filters_in_a_row_share_the_array():
    """Two filters inserted into one after the other on one stream (the
    ordering the shared array allows): each ends with exactly its own keys."""
    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib

    L = _lib.load()
    stream = torch.cuda.current_stream()
    geo = [(1 << 15, 16, 4, 73), (1 << 14, 8, 8, 74)]
    filts, keysets, flags = [], [], []
    for m, f, b, seed in geo:
        filt = _filter_in_torch_memory(cf, m, f, b)
        ks = workloads.keys(seed, int(0.95 * m * b))
        fl = torch.empty(ks.size, dtype=torch.uint8, device="cuda")
        rc = L.cf_insert_noalloc(filt.handle, to_dev(ks).data_ptr(), ks.size,
                                 fl.data_ptr(), stream.cuda_stream)
        assert rc == 0, L.cf_last_error()
        filts.append(filt)
        keysets.append(ks)
        flags.append(fl)
    torch.cuda.synchronize()
    for (m, f, b, _), filt, ks, fl in zip(geo, filts, keysets, flags):
        o = oracle.OracleFilter(m, f, b, 500)
        fp, i1, i2 = o.hash_batch(ks)
        alt = AltTable(o, fp)
        after = slots_view(filt.snapshot()[64:], m, f, b)
        vt, vb = filt.victims()
        assert check_insert(alt, np.zeros_like(after), after, fp, i1, i2, vt, vb, 0) == []
        st = filt.stats()
        assert st["evictions"] > 0
        assert st["insert_fail"] == int((fl.cpu().numpy() != 1).sum()) == vt.size
        assert st["occupancy"] == int(np.count_nonzero(after))


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib

    L = _lib.load()
    g = cf.CuckooFilter(1 << 20, 16, 4, 500)
    n = (1 << 20) + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    rc = L.cf_insert_noalloc(g.handle, keys.data_ptr(), n, None,
                             torch.cuda.current_stream().cuda_stream)
    assert rc == 1  # CF_EINVAL
    assert b"CF_NOALLOC_MAX_KEYS" in L.cf_last_error()
    assert g.stats()["insert_ok"] == 0
