"""Pins for the oracle against facts fixed by the mathematics and the paper:
capacity (exact maximum b-matching on tiny tables), the FPR model (Eq. 4),
the paper's printed FPR, and the eviction-depth shape of Fig. 5."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_points.json")))


def max_b_matching(i1, i2, m, b):
    """Largest number of keys that can be placed, each in one of its two
    buckets, with at most b per bucket (Kuhn's augmenting paths over
    bucket slots).  Brute-force sized: m * b <= 64."""
    owner = [-1] * (m * b)

    def slots_of(j):
        return range(j * b, j * b + b)

    def augment(k, seen):
        for j in {int(i1[k]), int(i2[k])}:
            for s in slots_of(j):
                if s in seen:
                    continue
                seen.add(s)
                if owner[s] < 0 or augment(owner[s], seen):
                    owner[s] = k
                    return True
        return False

    return sum(augment(k, set()) for k in range(len(i1)))


@pytest.mark.parametrize("m", [2, 4, 8, 16])
@pytest.mark.parametrize("eviction", [0, 1])
def test_stored_never_exceeds_max_matching(m, eviction):
    b = 4
    for seed in range(5):
        o = oracle.OracleFilter(m, 8, b, 200, eviction=eviction)
        ks = workloads.keys(1000 + seed, m * b + 6)
        fp, i1, i2 = o.hash_batch(ks)
        M = max_b_matching(i1, i2, m, b)
        flags = o.insert_batch(ks)
        st = o.stats()
        assert st["occupancy"] <= M
        assert st["insert_fail"] >= ks.size - M
        assert st["occupancy"] + st["insert_fail"] == ks.size
        assert int((flags == 0).sum()) == st["insert_fail"]


def _fpr_count(f, b, m, alpha, n_neg, policy=0, low32=False):
    o = oracle.OracleFilter(m, f, b, 500, policy=policy)
    n = int(alpha * m * b)
    if low32:
        pos = workloads.low32_keys(7, n)
        neg = workloads.high_keys(8, n_neg)
    else:
        pos = workloads.keys(1, n)
        neg = workloads.keys(1, n_neg, start=n)
    flags = o.insert_batch(pos)
    assert flags.all(), int((flags == 0).sum())
    alpha_real = o.stats()["occupancy"] / (m * b)
    return int(o.contains_batch(neg).sum()), alpha_real


@pytest.mark.parametrize("f,b,m_log,n_neg_log", [(8, 4, 14, 18), (8, 16, 12, 18),
                                                 (16, 4, 18, 20)])
def test_fpr_matches_eq4(f, b, m_log, n_neg_log):
    """Measured false positives lie within five Poisson standard deviations
    of Eq. 4 on both sides (a query that skips a bucket halves the rate, a
    wrong tag comparison inflates it)."""
    m, N = 1 << m_log, 1 << n_neg_log
    fp_count, a = _fpr_count(f, b, m, 0.95, N)
    e = N * oracle.fpr_expected(f, b, a)
    assert abs(fp_count - e) <= 5 * math.sqrt(e) + 1, (fp_count, e)
    assert fp_count <= oracle.fpr_bound(N, f, b, a)


def test_fpr_single_filter_workload_within_stated_bound():
    """2^18 buckets x 4 slots, 16-bit fingerprints, LF 0.95, 2^20 disjoint
    negatives: count <= E + 5 sqrt(E) + 1 (about 178, FPR <= 1.7e-4)."""
    fp_count, a = _fpr_count(16, 4, 1 << 18, 0.95, 1 << 20)
    bound = oracle.fpr_bound(1 << 20, 16, 4, a)
    assert 170 < bound < 185
    assert fp_count <= bound


def test_fpr_paper_point_f16_b16():
    """The paper prints about 0.045% for f = 16, b = 16 at 95% load, with
    positives from [0, 2^32) and negatives from [2^32, 2^64)."""
    g = GOLD["fpr_f16_b16_lf095"]
    N = 1 << 21
    cnt, a = _fpr_count(g["f"], g["b"], 1 << 16, g["alpha"], N, low32=True)
    rate = cnt / N
    assert abs(rate - g["fpr"]) < 0.00008, rate
    assert abs(rate - oracle.fpr_expected(16, 16, a)) < 0.00008


def test_fpr_offset_policy_within_eq4_with_one_bit_less():
    """Offset policy: the choice bit costs one fingerprint bit, so the rate
    stays below Eq. 4 evaluated with f - 1 bits."""
    N = 1 << 18
    cnt, a = _fpr_count(8, 4, 12345, 0.9, N, policy=1)
    e_hi = N * oracle.fpr_expected(8, 4, a, policy=1)
    assert cnt <= e_hi + 5 * math.sqrt(e_hi) + 1
    e_lo = N * oracle.fpr_expected(8, 4, a)
    assert cnt >= e_lo * 0.5


def _tail_evictions(eviction, alpha, m=1 << 14, b=16):
    """Fig. 5 protocol: pre-fill 3/4 of the target, record the evictions of
    the last quarter."""
    o = oracle.OracleFilter(m, 16, b, 500, eviction=eviction)
    n = int(alpha * m * b)
    ks = workloads.keys(2, n)
    q = (3 * n) // 4
    o.insert_batch(ks[:q])
    flags, ev = o.insert_batch(ks[q:], want_evictions=True)
    return np.percentile(ev, [90, 95, 99]), flags


def test_bfs_tail_evictions_shape():
    g = GOLD["bfs_tail_evictions"]
    p, flags = _tail_evictions(0, 0.90)
    assert p[0] <= g["bfs_p90_until_0.90"] + 0 and p[2] <= g["bfs_p99_until_0.95"] + 1
    p, flags = _tail_evictions(0, 0.95)
    assert p[2] <= g["bfs_p99_until_0.95"] + 1
    assert flags.all()


def test_dfs_tail_exceeds_bfs_near_full():
    pb, _ = _tail_evictions(0, 0.99)
    pd, _ = _tail_evictions(1, 0.99)
    assert pd[2] >= pb[2]
    assert pd[2] > 2
