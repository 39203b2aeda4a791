"""The serving loop (cf_server_*): results of every request are the same
served in the mix as run alone, budget admission, watchdog, drain.

"The same" means: insert and delete flags identical (no capacity pressure,
distinct keys), query flags identical on every key that is present at the
request's turn, and on absent keys only false positives may differ, with
their totals within the Eq. 4 bound on both sides.  The sequential oracle
replays every filter's requests in order as the third witness, and the
final tables hold identical multisets of stored classes.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import AltTable, multiset_delta, slots_view
from workloads.serve import materialize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


def _small_trace(n_requests=600, seed=11):
    return workloads.serve_trace(n_requests, n_filters=8, e_lo=10, e_hi=14,
                                 max_log2=12.0, seed=seed)


def test_served_results_equal_alone_results(cf):
    sizes, plan = _small_trace()
    reqs, keep = materialize(sizes, plan)
    srv = cf.Server(1 << 30, max_inflight=3, max_wave_items=16, max_wave_keys=1 << 14)
    fids = [srv.add_filter(m, 16, 4, 500) for m in sizes]
    plain = [cf.CuckooFilter(m, 16, 4, 500) for m in sizes]
    # Served: everything submitted at once (maximal mixing).
    out_s = srv.run_trace([(fids[f], op, k, fl, i) for i, (f, op, k, fl) in enumerate(reqs)],
                          [0.0] * len(reqs))
    assert (out_s["status"] == 0).all()
    flags_s = [fl.cpu().numpy().copy() for _, _, _, fl in reqs]
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["waves"] < len(reqs)  # batching happened
    assert out_s["wave_size"].max() > 1
    # Alone: one plain call per request, in order.
    for _, _, _, fl in reqs:
        fl.zero_()
    cf.plain_run_trace(plain, [(f, op, k, fl, i) for i, (f, op, k, fl) in enumerate(reqs)],
                       [0.0] * len(reqs))
    flags_p = [fl.cpu().numpy().copy() for _, _, _, fl in reqs]
    # Oracle: each filter's requests in order.
    ors = [oracle.OracleFilter(m, 16, 4, 500) for m in sizes]
    fp_s = fp_p = neg_total = 0
    for (f, op, n, ps, pn, ns, nn), (_, _, k, _), a, b in zip(plan, reqs, flags_s, flags_p):
        kh = k.cpu().numpy().view(np.uint64)
        if op == "insert":
            o = ors[f].insert_batch(kh)
            assert (a == 1).all() and (b == 1).all() and (o == 1).all()
        elif op == "remove":
            o = ors[f].remove_batch(kh)
            assert np.array_equal(a, b) and np.array_equal(a, o)
        else:
            o = ors[f].contains_batch(kh)
            assert (a[:pn] == 1).all() and (b[:pn] == 1).all() and (o[:pn] == 1).all()
            fp_s += int(a[pn:].sum())
            fp_p += int(b[pn:].sum())
            neg_total += nn
    bound = oracle.fpr_bound(neg_total, 16, 4, 0.9)
    assert fp_s <= bound and fp_p <= bound
    # Final states: same multiset of stored classes.
    for f, (m, fid) in enumerate(zip(sizes, fids)):
        g = plain[f]
        h = srv.filter_handle(fid)
        assert h
        from paper_2603_15486_gb300 import _lib
        L = _lib.load()
        buf = np.empty(g.snapshot_bytes(), np.uint8)
        assert L.cf_snapshot(h, buf.ctypes.data, buf.size, 0, None) == 0
        ts = slots_view(buf[64:], m, 16, 4)
        tp = slots_view(g.snapshot()[64:], m, 16, 4)
        allk = workloads.keys(10000 + f, int(np.count_nonzero(tp)) + 100000)
        fp, _, _ = ors[f].hash_batch(allk)
        alt = AltTable(ors[f], fp)
        js, ss = np.nonzero(ts)
        jp, sp = np.nonzero(tp)
        a1, b1, k1 = alt.classes(js, ts[js, ss])
        a2, b2, k2 = alt.classes(jp, tp[jp, sp])
        assert k1.all() and k2.all()
        A, _, _ = multiset_delta([(a1, b1, 1), (a2, b2, -1)])
        assert A.size == 0
        assert ors[f].stats()["occupancy"] == int(np.count_nonzero(ts))
    srv.close()


def test_poisson_arrivals_complete_with_positive_latency(cf):
    sizes, plan = _small_trace(300, seed=12)
    reqs, keep = materialize(sizes, plan)
    srv = cf.Server(1 << 30, max_inflight=2, max_wave_items=8, max_wave_keys=1 << 14)
    fids = [srv.add_filter(m, 16, 4, 500) for m in sizes]
    arr = np.cumsum(np.random.default_rng(1).exponential(50e-6, size=len(reqs)))
    out = srv.run_trace([(fids[f], op, k, fl, i) for i, (f, op, k, fl) in enumerate(reqs)], arr)
    lat = out["done_s"] - out["submit_s"]
    assert (out["status"] == 0).all() and (lat > 0).all()
    assert (out["launch_s"] >= out["submit_s"] - 1e-6).all()
    srv.close()


def test_admission_waits_for_budget(cf):
    m = 1 << 16
    one = cf.required_bytes(num_buckets=m, fp_bits=16, slots_per_bucket=4)
    srv = cf.Server(int(2.5 * one), max_inflight=2, max_wave_items=8, max_wave_keys=1 << 16)
    a, b, c = (srv.add_filter(m) for _ in range(3))
    ks = torch.from_numpy(workloads.keys(5, 50000).view(np.int64)).cuda()
    for fid in (a, b):
        srv.submit(fid, "insert", ks)
    srv.submit(c, "insert", ks)
    out_c = torch.zeros(50000, dtype=torch.uint8, device="cuda")
    srv.submit(c, "contains", ks, out_c)
    # c cannot be admitted while a and b hold the budget.
    assert srv.drain(300) == 4          # CF_ETIMEOUT, nothing stuck on the GPU
    assert srv.filter_state(c) == "pending"
    assert srv.stats()["pending_filters"] == 1
    srv.remove_filter(a)
    assert srv.drain(60000) == 0
    assert srv.filter_state(a) == "closed" and srv.filter_state(c) == "live"
    assert out_c.cpu().numpy().all()
    done = srv.poll()
    assert len(done) == 4 and (done["status"] == 0).all()
    with pytest.raises(RuntimeError):   # a filter larger than the whole budget
        srv.add_filter(1 << 20)
    srv.close()


def test_removed_pending_filter_still_runs_its_requests(cf):
    """A filter removed before the budget admitted it keeps its queued
    requests: it is admitted when room frees up, runs them, then closes.
    A pending filter removed with nothing queued closes unallocated."""
    m = 1 << 16
    one = cf.required_bytes(num_buckets=m, fp_bits=16, slots_per_bucket=4)
    srv = cf.Server(int(1.5 * one), max_inflight=2, max_wave_items=8, max_wave_keys=1 << 16)
    a, b, c = (srv.add_filter(m) for _ in range(3))
    ks = torch.from_numpy(workloads.keys(6, 40000).view(np.int64)).cuda()
    srv.submit(a, "insert", ks)
    srv.submit(b, "insert", ks)
    out_b = torch.zeros(40000, dtype=torch.uint8, device="cuda")
    srv.submit(b, "contains", ks, out_b)
    srv.remove_filter(b)                 # pending, two requests queued
    srv.remove_filter(c)                 # pending, nothing queued
    assert srv.drain(300) == 4           # b waits for a's budget
    assert srv.filter_state(b) == "pending"
    srv.remove_filter(a)
    assert srv.drain(60000) == 0
    assert srv.filter_state(a) == "closed"
    assert srv.filter_state(b) == "closed" and srv.filter_state(c) == "closed"
    assert out_b.cpu().numpy().all()
    done = srv.poll()
    assert len(done) == 3 and (done["status"] == 0).all()
    assert srv.stats()["used_bytes"] == 0
    srv.close()


def test_watchdog_marks_late_waves(cf):
    srv = cf.Server(1 << 30, max_inflight=2, max_wave_items=8, max_wave_keys=1 << 20,
                    watchdog_us=1)
    fid = srv.add_filter(1 << 18)
    ks = torch.from_numpy(workloads.keys(6, 400000).view(np.int64)).cuda()
    fl = torch.zeros(400000, dtype=torch.uint8, device="cuda")
    srv.submit(fid, "insert", ks, fl)
    assert srv.drain(60000) == 0
    done = srv.poll()
    assert (done["status"] == 4).all()          # late, reported as CF_ETIMEOUT
    assert fl.cpu().numpy().all()               # results are still written
    assert srv.stats()["late_waves"] >= 1
    srv.close()


def test_submit_validation(cf):
    srv = cf.Server(1 << 30, max_inflight=1, max_wave_items=4, max_wave_keys=1000)
    fid = srv.add_filter(1 << 10)
    k = torch.zeros(10, dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        srv.submit(fid + 100, "insert", k)            # unknown filter
    with pytest.raises(RuntimeError):
        srv.submit(fid, "contains", k, None)          # query without flags
    with pytest.raises(RuntimeError):
        srv.submit(fid, "insert", torch.zeros(2000, dtype=torch.int64, device="cuda"))
    srv.submit(fid, "insert", k)
    assert srv.drain(60000) == 0
    srv.close()
