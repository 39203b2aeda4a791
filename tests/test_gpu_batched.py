"""The multi-filter launch (cf_batch_*) against the oracle and against the
single-filter calls.  Same rules as the single-filter parity tests: query
bit-exact, insert by the multiset invariant, delete by the validity checker
with bit-exact agreement where the outcome is forced."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import AltTable, check_delete, check_insert, key_classes, slots_view
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


def _sizes(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    return [1 << int(e) for e in rng.integers(lo, hi + 1, size=n)]


def _oracle_filters(ms, f, b, alpha, seed):
    out = []
    for i, m in enumerate(ms):
        o = oracle.OracleFilter(m, f, b, 500)
        ks = workloads.keys(seed + i, int(alpha * m * b))
        o.insert_batch(ks)
        out.append((o, ks))
    return out


@pytest.mark.parametrize("f,b", [(16, 4), (16, 16), (8, 8), (32, 4)])
def test_batched_query_bit_exact_every_variant(cf, f, b):
    ms = _sizes(24, 4, 12, 1)
    ors = _oracle_filters(ms, f, b, 0.9, 100)
    gfs, items, expect = [], [], []
    for i, (o, ks) in enumerate(ors):
        g = cf.CuckooFilter(o.m, f, b, 500)
        g.load(o.snapshot())
        q = np.concatenate([ks, workloads.keys(100 + i, 777 + 13 * i, start=ks.size)])
        qd = to_dev(q)
        out = torch.full((q.size,), 7, dtype=torch.uint8, device="cuda")
        gfs.append(g)
        items.append((g, "contains", qd, out))
        expect.append(o.contains_batch(q))
    bt = cf.Batch(64, 1 << 22)
    bt.set(items)
    assert bt.variant_count() >= 1
    for v in range(bt.variant_count()):
        bt.set_variant(v)
        for graph in (False, True):
            for _, _, _, out in items:
                out.fill_(7)
            bt.launch(graph=graph)
            torch.cuda.synchronize()
            for (_, _, _, out), e in zip(items, expect):
                assert np.array_equal(out.cpu().numpy(), e), (v, graph)


def test_batched_insert_invariants_many_sizes(cf):
    f, b = 16, 4
    ms = _sizes(40, 4, 14, 2)
    rng = np.random.default_rng(3)
    gfs, items, keysets = [], [], []
    for i, m in enumerate(ms):
        n = int(min(10 ** rng.uniform(1, 4.5), 0.9 * m * b))
        ks = workloads.keys(300 + i, n)
        g = cf.CuckooFilter(m, f, b, 500)
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        gfs.append(g)
        keysets.append(ks)
        items.append((g, "insert", to_dev(ks), fl))
    bt = cf.Batch(64, sum(k.size for k in keysets))
    bt.set(items)
    bt.launch()
    torch.cuda.synchronize()
    for (g, _, _, fl), ks, m in zip(items, keysets, ms):
        o = oracle.OracleFilter(m, f, b, 500)
        fp, i1, i2 = o.hash_batch(ks)
        slots = slots_view(g.snapshot()[64:], m, f, b)
        vt, vb = g.victims()
        probs = check_insert(AltTable(o, fp), np.zeros_like(slots), slots, fp, i1, i2,
                             vt, vb, 0)
        assert probs == [], probs
        st = g.stats()
        flags = fl.cpu().numpy()
        assert st["occupancy"] == int(np.count_nonzero(slots))
        assert st["insert_fail"] == int((flags != 1).sum()) == st["victims"]
        assert st["insert_ok"] == int((flags == 1).sum())
        q = g.contains(to_dev(ks)).cpu().numpy()
        if vt.size == 0:
            assert q.all()


def test_batched_remove_parity_on_oracle_tables(cf):
    f, b = 16, 8
    ms = _sizes(16, 6, 12, 4)
    ors = _oracle_filters(ms, f, b, 0.9, 500)
    items, befores, dels = [], [], []
    gfs = []
    for i, (o, ks) in enumerate(ors):
        g = cf.CuckooFilter(o.m, f, b, 500)
        g.load(o.snapshot())
        d = np.concatenate([ks[: ks.size // 2], workloads.keys(500 + i, 300, start=ks.size),
                            ks[:20]])
        befores.append(slots_view(o.table_words(), o.m, f, b).copy())
        fl = torch.empty(d.size, dtype=torch.uint8, device="cuda")
        items.append((g, "remove", to_dev(d), fl))
        dels.append(d)
        gfs.append(g)
    bt = cf.Batch(32, 1 << 20)
    bt.set(items)
    bt.launch(graph=True)
    torch.cuda.synchronize()
    for (o, ks), (g, _, _, fl), d, before in zip(ors, items, dels, befores):
        ofl = o.remove_batch(d)
        fp, i1, i2 = o.hash_batch(d)
        after = slots_view(g.snapshot()[64:], o.m, f, b)
        probs, n_iso = check_delete(before, after, fp, i1, i2, fl.cpu().numpy(), 0, f,
                                    oracle_after=slots_view(o.table_words(), o.m, f, b),
                                    oracle_flags=ofl)
        assert probs == [], probs


def test_batched_mixed_ops_and_graph_replay_with_new_items(cf):
    f, b = 16, 4
    m = 1 << 12
    A = [cf.CuckooFilter(m, f, b, 500) for _ in range(3)]
    ks = [workloads.keys(600 + i, 12000) for i in range(3)]
    bt = cf.Batch(8, 1 << 20)
    # First batch: insert into all three (graph captured here).
    bt.set([(A[i], "insert", to_dev(ks[i]), None) for i in range(3)])
    bt.launch(graph=True)
    # Second batch, same graph replayed: query A0, remove half of A1, insert more into A2.
    out0 = torch.empty(ks[0].size, dtype=torch.uint8, device="cuda")
    rm1 = torch.empty(6000, dtype=torch.uint8, device="cuda")
    more = workloads.keys(603, 2000)
    bt.set([(A[0], "contains", to_dev(ks[0]), out0),
            (A[1], "remove", to_dev(ks[1][:6000]), rm1),
            (A[2], "insert", to_dev(more), None)])
    bt.launch(graph=True)
    torch.cuda.synchronize()
    assert out0.cpu().numpy().all()
    assert rm1.cpu().numpy().all()
    assert A[1].stats()["occupancy"] == 12000 - 6000
    assert A[2].stats()["occupancy"] == 14000
    assert A[2].contains(to_dev(np.concatenate([ks[2], more]))).cpu().numpy().all()


def test_batched_rejects_bad_batches(cf):
    g = cf.CuckooFilter(1 << 10, 16, 4, 500)
    h = cf.CuckooFilter(1 << 10, 16, 8, 500)
    k = to_dev(workloads.keys(1, 100))
    out = torch.empty(100, dtype=torch.uint8, device="cuda")
    bt = cf.Batch(4, 1000)
    with pytest.raises(RuntimeError):   # query and mutation of one filter
        bt.set([(g, "insert", k, None), (g, "contains", k, out)])
    with pytest.raises(RuntimeError):   # two geometries
        bt.set([(g, "insert", k, None), (h, "insert", k, None)])
    with pytest.raises(RuntimeError):   # query without output
        bt.set([(g, "contains", k, None)])
    with pytest.raises(RuntimeError):   # too many keys
        bt.set([(g, "insert", to_dev(workloads.keys(1, 2000)), None)])
    bt.set([(g, "insert", k, None), (g, "insert", k, None)])  # two inserts: fine
    bt.launch()
    torch.cuda.synchronize()
    assert g.stats()["occupancy"] == 200


def test_autotune_leaves_state_and_results_correct(cf):
    f, b = 16, 4
    ms = _sizes(32, 8, 14, 7)
    rng = np.random.default_rng(8)
    items, keysets, gfs = [], [], []
    for i, m in enumerate(ms):
        n = int(min(10 ** rng.uniform(2, 4.3), 0.9 * m * b))
        ks = workloads.keys(700 + i, n)
        g = cf.CuckooFilter(m, f, b, 500)
        g.insert(to_dev(ks[: n // 3]))            # some prior state
        keysets.append(ks)
        gfs.append(g)
        items.append((g, "insert", to_dev(ks[n // 3:]), None))
    torch.cuda.synchronize()
    before = [g.snapshot() for g in gfs]
    bt = cf.Batch(64, 1 << 21)
    bt.set(items)
    t = bt.autotune()
    assert 0 <= t["variant"] < bt.variant_count() and t["ms"] > 0
    for g, s in zip(gfs, before):
        assert np.array_equal(g.snapshot(), s)     # trials were undone
    bt.launch()
    torch.cuda.synchronize()
    for g, ks in zip(gfs, keysets):
        st = g.stats()
        assert st["occupancy"] + st["insert_fail"] == ks.size
        assert g.contains(to_dev(ks)).cpu().numpy().sum() >= ks.size - st["victims"]
    # A later plan of the same class picks the tuned variant without tuning.
    bt2 = cf.Batch(64, 1 << 21)
    bt2.set(items)
    assert bt2.tuning()["variant"] == t["variant"]


def test_batched_equals_plain_calls_on_queries(cf):
    """Queries through the batch and through one cf_contains per filter give
    identical flags on the same tables."""
    f, b = 16, 4
    ms = _sizes(20, 6, 13, 9)
    ors = _oracle_filters(ms, f, b, 0.85, 900)
    items, plain = [], []
    for i, (o, ks) in enumerate(ors):
        g = cf.CuckooFilter(o.m, f, b, 500)
        g.load(o.snapshot())
        q = to_dev(np.concatenate([ks, workloads.keys(900 + i, 5000, start=ks.size)]))
        out = torch.empty(q.numel(), dtype=torch.uint8, device="cuda")
        items.append((g, "contains", q, out))
        plain.append(g.contains(q))
    bt = cf.Batch(32, 1 << 20)
    bt.set(items)
    bt.launch()
    torch.cuda.synchronize()
    for (_, _, _, out), p in zip(items, plain):
        assert torch.equal(out, p)
