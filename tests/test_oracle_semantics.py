"""Pins for the oracle's insert / query / delete semantics (Alg. 1-3).

Special case f = 32 with few keys: a false positive needs a 32-bit
fingerprint collision inside a shared bucket, which these seeds never hit,
so the filter must behave exactly like a multiset of keys.
"""
import collections

import numpy as np
import pytest

import oracle
import workloads
from cfcheck import AltTable, check_delete, check_insert, slots_view


def _collision_free(o, universe):
    fp, i1, i2 = o.hash_batch(universe)
    seen = {}
    for k, f_, a, b in zip(universe, fp, i1, i2):
        for j in (int(a), int(b)):
            if (j, int(f_)) in seen and seen[(j, int(f_))] != int(k):
                return False
            seen[(j, int(f_))] = int(k)
    return True


@pytest.mark.parametrize("b", [4, 8, 16])
@pytest.mark.parametrize("policy", [0, 1])
def test_f32_behaves_as_multiset(b, policy):
    m = 1 << 8 if policy == 0 else 300
    o = oracle.OracleFilter(m, 32, b, 500, policy=policy)
    universe = workloads.keys(21 + b, 200)
    assert _collision_free(o, universe)
    ms = collections.Counter()
    rng = np.random.default_rng(b + 10 * policy)
    cap = m * b
    for step in range(6000):
        k = int(universe[rng.integers(0, universe.size)])
        r = rng.random()
        if r < 0.4 and sum(ms.values()) < cap // 2 and ms[k] < 2:
            ok, _ = o.insert(k)
            assert ok
            ms[k] += 1
        elif r < 0.7:
            got = o.remove(k)
            assert got == (ms[k] > 0), (step, k)
            if got:
                ms[k] -= 1
        else:
            assert o.contains(k) == (ms[k] > 0), (step, k)
    assert o.stats()["occupancy"] == sum(ms.values())
    # No false negatives, no false positives at the end.
    for k in universe:
        assert o.contains(int(k)) == (ms[int(k)] > 0)


def test_delete_then_absent():
    o = oracle.OracleFilter(1 << 10, 32, 4, 100)
    ks = workloads.keys(31, 2000)
    assert o.insert_batch(ks).all()
    assert o.remove_batch(ks[:1000]).all()
    assert not o.contains_batch(ks[:1000]).any()
    assert o.contains_batch(ks[1000:]).all()
    assert not o.remove_batch(ks[:1000]).any()


@pytest.mark.parametrize("f,b,alpha", [(16, 4, 0.95), (8, 8, 0.97), (16, 16, 0.98),
                                       (32, 4, 0.9)])
@pytest.mark.parametrize("eviction", [0, 1])
def test_insert_invariants(f, b, alpha, eviction):
    """Every stored tag sits in i1 or i2 of a key with that fingerprint; the
    stored multiset equals keys minus victims; counters agree."""
    m = 1 << 12
    o = oracle.OracleFilter(m, f, b, 60, eviction=eviction)
    n = int(alpha * m * b)
    ks = workloads.keys(41 + f + b, n)
    flags, ev = o.insert_batch(ks, want_evictions=True)
    st = o.stats()
    vt, vb = o.victims()
    slots = slots_view(o.table_words(), m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    alt = AltTable(o, fp)
    empty = np.zeros_like(slots)
    assert check_insert(alt, empty, slots, fp, i1, i2, vt, vb, 0) == []
    assert st["occupancy"] == int(np.count_nonzero(slots))
    assert st["insert_fail"] == int((flags == 0).sum()) == st["victims"] == vt.size
    assert st["evictions"] == int(ev.sum())
    # Zero false negatives apart from keys whose class lost a victim.
    q = o.contains_batch(ks)
    vclass = set()
    if vt.size:
        va, vb2, _ = alt.classes(vb, vt)
        vclass = set(zip(va.tolist(), vb2.tolist()))
    from cfcheck import key_classes
    ka, kb = key_classes(fp, i1, i2, 0)
    for idx in np.flatnonzero(q == 0):
        assert (int(ka[idx]), int(kb[idx])) in vclass


def test_checker_catches_planted_mistakes():
    """Plant mistakes in an oracle result and check that the invariant
    checker flags each one."""
    m, f, b = 1 << 10, 16, 4
    o = oracle.OracleFilter(m, f, b, 100)
    ks = workloads.keys(55, int(0.9 * m * b))
    o.insert_batch(ks)
    slots = slots_view(o.table_words(), m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    alt = AltTable(o, fp)
    vt, vb = o.victims()
    empty = np.zeros_like(slots)
    assert check_insert(alt, empty, slots, fp, i1, i2, vt, vb, 0) == []
    j, s = map(int, np.argwhere(slots)[17])
    # 1. a dropped tag
    bad = slots.copy(); bad[j, s] = 0
    assert check_insert(alt, empty, bad, fp, i1, i2, vt, vb, 0)
    # 2. a tag moved to a bucket that is not one of its two
    bad = slots.copy(); t = bad[j, s]; bad[j, s] = 0
    other = (j + 1) % m
    e = np.flatnonzero(bad[other] == 0)
    if e.size == 0:
        bad[other, 0] = t
    else:
        bad[other, e[0]] = t
    assert check_insert(alt, empty, bad, fp, i1, i2, vt, vb, 0)
    # 3. a wrong tag value
    bad = slots.copy(); bad[j, s] ^= 1
    assert check_insert(alt, empty, bad, fp, i1, i2, vt, vb, 0)


def test_delete_checker_on_oracle_results_and_planted_mistakes():
    m, f, b = 1 << 10, 16, 4
    o = oracle.OracleFilter(m, f, b, 100)
    ks = workloads.keys(66, int(0.9 * m * b))
    o.insert_batch(ks)
    before = slots_view(o.table_words(), m, f, b).copy()
    # Delete a prefix, some absent keys and a duplicate.
    dels = np.concatenate([ks[:1500], workloads.keys(66, 300, start=10**6), ks[:5]])
    fl = o.remove_batch(dels)
    after = slots_view(o.table_words(), m, f, b)
    fp, i1, i2 = o.hash_batch(dels)
    probs, n_iso = check_delete(before, after, fp, i1, i2, fl, 0, f,
                                oracle_after=after, oracle_flags=fl)
    assert probs == [] and n_iso > 1000
    # A success reported on an absent key.
    bad = fl.copy(); bad[1500 + np.flatnonzero(fl[1500:1800] == 0)[0]] = 1
    assert check_delete(before, after, fp, i1, i2, bad, 0, f)[0]
    # A failure reported on a present key.
    bad = fl.copy(); bad[3] = 0
    assert check_delete(before, after, fp, i1, i2, bad, 0, f)[0]
    # A lane cleared that nobody asked for.
    j = int(np.flatnonzero((after != 0).any(1))[0])
    s = int(np.flatnonzero(after[j])[0])
    bad_after = after.copy(); bad_after[j, s] = 0
    assert check_delete(before, bad_after, fp, i1, i2, fl, 0, f)[0]


@pytest.mark.parametrize("seed", range(6))
def test_delete_order_only_matters_within_contended_groups(seed):
    """Run the same delete batch in several orders: isolated deleters always
    get the same outcome, and every order passes the validity checker."""
    m, f, b = 1 << 6, 8, 4   # tiny and f = 8: plenty of shared (bucket, tag)
    base = oracle.OracleFilter(m, f, b, 100)
    ks = workloads.keys(100 + seed, int(0.9 * m * b))
    base.insert_batch(ks)
    snap = base.snapshot()
    before = slots_view(snap[64:], m, f, b).copy()
    rng = np.random.default_rng(seed)
    dels = np.concatenate([ks[rng.permutation(ks.size)[:120]],
                           workloads.keys(7, 40, start=500)])
    fp, i1, i2 = base.hash_batch(dels)
    ref_flags = None
    for trial in range(8):
        perm = rng.permutation(dels.size)
        o = oracle.OracleFilter(m, f, b, 100)
        o.load(snap)
        fl = np.empty(dels.size, np.uint8)
        fl[perm] = o.remove_batch(dels[perm])
        after = slots_view(o.table_words(), m, f, b)
        probs, n_iso = check_delete(before, after, fp, i1, i2, fl, 0, f)
        assert probs == []
        if ref_flags is None:
            ref_flags, ref_after = fl, after
        else:
            p2, _ = check_delete(before, after, fp, i1, i2, fl, 0, f,
                                 oracle_after=ref_after, oracle_flags=ref_flags)
            assert p2 == []
