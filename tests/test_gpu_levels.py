"""The slice-grouped eviction levels of the sliced insert
(cf_set_eviction_levels).

The levels change the order in which the eviction chains of one batch take
their steps (all chains one step per level, grouped by table slice), not
the steps themselves (Alg. 1 phase 2 with the BFS heuristic of Sec. 4.6.1,
asked of the full-bucket map).  So:

  * a batch whose only queued key is one chain (one key inserted into a
    table the oracle filled) leaves the table, the flag, the eviction count
    and the victims exactly as the sequential oracle does, whether the
    chain ends inside the levels or in the run of the remaining chains;
  * parallel inserts through the levels satisfy the insert invariants on
    every geometry and both bucket policies, with failure counts within
    the usual margin of the oracle's;
  * a batch skewed into one slice overflows a level's buffer: those chains
    run to their end at once, and the invariants still hold;
  * the levels run only when switched on, for BFS, with the map, and for
    queues of at least min_queue keys; host-buffer inserts and filters
    with buckets wider than 8 bytes take them only in the "always" mode
    (the tests below use that mode to cover every geometry).
"""
import numpy as np
import pytest

import oracle
import workloads
from cfcheck import AltTable, check_insert, slots_view
from gpu_util import m_for, oracle_policy, to_dev

pytestmark = pytest.mark.gpu

GEOMS = [(8, 4), (8, 8), (8, 16), (16, 4), (16, 8), (16, 16), (32, 4), (32, 8), (32, 16)]


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


def _levels_filter(cf, m, f, b, policy="xor", n_levels=24, stop_queue=1, max_ev=500,
                   victim_capacity=1 << 16):
    g = cf.CuckooFilter(m, f, b, max_ev, policy=policy, victim_capacity=victim_capacity)
    g.set_eviction_map("always")
    g.set_slicing("always", 1024)
    g.set_eviction_levels("always", n_levels, 1, stop_queue)
    g.set_kernel_timing(True)
    return g


@pytest.mark.parametrize("f,b", [(8, 4), (16, 4), (16, 16), (32, 8)])
@pytest.mark.parametrize("policy", ["xor", "offset"])
@pytest.mark.parametrize("n_levels", [1, 24])
def test_single_chain_through_levels_bit_exact(cf, f, b, policy, n_levels):
    m = m_for(policy, 1 << 9)
    o = oracle.OracleFilter(m, f, b, 100, policy=oracle_policy(policy))
    o.insert_batch(workloads.keys(300 + f + b, int(0.97 * m * b)))
    g = _levels_filter(cf, m, f, b, policy, n_levels=n_levels, max_ev=100)
    snap = g.snapshot()
    snap[64:] = o.table_words()
    g.load(snap)
    ot0 = o.victims()[0].size
    chains = 0
    for k in workloads.keys(400 + f + b, 48):
        ev0 = g.stats()["evictions"]
        fl = g.insert(to_dev(np.array([k], np.uint64))).cpu().numpy()
        ok, oev = o.insert(int(k))
        st = g.stats()
        assert int(fl[0]) == int(ok)
        assert st["evictions"] - ev0 == oev
        assert np.array_equal(g.snapshot()[64:], o.table_words())
        chains += oev > 0
    ot, ob = o.victims()
    gt, gb = g.victims()
    assert np.array_equal(gt, ot[ot0:]) and np.array_equal(gb, ob[ot0:])
    st = g.stats()
    assert chains > 0 and st["level_passes"] > 0 and st["level_runout"] == 0
    assert st["contention"] == 0 and st["error_word"] == 0
    assert g.kernel_times()["evict_level"][0] > 0


def _check(cf, g, o, ks, flags, policy, m, f, b):
    slots = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    vt, vb = g.victims()
    st = g.stats()
    probs = check_insert(AltTable(o, fp), np.zeros_like(slots), slots, fp, i1, i2, vt, vb,
                         oracle_policy(policy))
    assert probs == [], probs
    assert st["occupancy"] == int(np.count_nonzero(slots)) == g.count_occupied()
    assert st["insert_fail"] == int((flags != 1).sum()) == st["victims"] == vt.size
    assert st["contention"] == 0 and st["error_word"] == 0
    return st


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", ["xor", "offset"])
def test_parallel_insert_through_levels_invariants(cf, f, b, policy):
    m = m_for(policy, 1 << 12)
    n = int(0.96 * m * b) + 5
    ks = workloads.keys(517 + f + b, n)
    o = oracle.OracleFilter(m, f, b, 500, policy=oracle_policy(policy))
    g = _levels_filter(cf, m, f, b, policy)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    st = _check(cf, g, o, ks, flags, policy, m, f, b)
    assert st["level_passes"] > 0 and st["level_steps"] > 0 and st["evictions"] > 0
    ofl = o.insert_batch(ks)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + max(5, n // 100)


@pytest.mark.parametrize("n_levels,stop_queue", [(1, 1), (2, 64), (4, 1 << 30)])
def test_levels_hand_over_to_the_run_of_the_rest(cf, n_levels, stop_queue):
    """Few levels, or a stop threshold that ends the levels early: the
    chains left run to their end; invariants and counts as before."""
    m, f, b = 1 << 14, 16, 4
    n = int(0.97 * m * b)
    ks = workloads.keys(611, n)
    o = oracle.OracleFilter(m, f, b, 500)
    g = _levels_filter(cf, m, f, b, n_levels=n_levels, stop_queue=stop_queue)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    st = _check(cf, g, o, ks, flags, "xor", m, f, b)
    # Level 0 always runs once the seed switched the levels on; a stop
    # threshold above any count leaves every later level idle.
    assert 1 <= st["level_passes"] <= n_levels
    if stop_queue > n:
        assert st["level_passes"] == 1
    ofl = o.insert_batch(ks)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + max(5, n // 100)


def test_levels_in_three_calls(cf):
    """Fill 0 -> 0.5 -> 0.8 -> 0.95 in three calls (the benchmark's
    protocol) through the levels, on a table of 2^16 buckets."""
    m, f, b = 1 << 16, 16, 4
    w = workloads.Workload("t", m, f, b, 500, 2, (0.5, 0.8, 0.95), 0, 0, 0)
    ks = workloads.keys(2, w.n_insert)
    g = _levels_filter(cf, m, f, b)
    o = oracle.OracleFilter(m, f, b, 500)
    flags = np.concatenate([g.insert(to_dev(ks[lo:hi])).cpu().numpy()
                            for lo, hi in w.insert_segments()])
    st = _check(cf, g, o, ks, flags, "xor", m, f, b)
    assert st["level_passes"] >= 2


def test_skewed_batch_overflows_a_level(cf):
    """Keys whose two buckets both lie in slice 0 of 32 (slice_bytes 1024
    over 8-byte buckets: 128 buckets per slice): every chain stays in that
    slice, overflows its region and the spill region of level 0's buffer,
    and runs to its end at once; the invariants still hold."""
    m, f, b = 1 << 12, 16, 4
    o = oracle.OracleFilter(m, f, b, 50)
    cand = workloads.keys(707, 1 << 22)
    _, i1, i2 = o.hash_batch(cand)
    ks = cand[(i1 < 128) & (i2 < 128)]
    assert 3000 < ks.size < 5000
    g = _levels_filter(cf, m, f, b, max_ev=50, victim_capacity=1 << 16)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    st = _check(cf, g, o, ks, flags, "xor", m, f, b)
    assert st["level_passes"] > 0 and st["level_runout"] > 0


def test_levels_rules(cf):
    m, f, b = 1 << 12, 16, 4
    ks = to_dev(workloads.keys(808, int(0.96 * m * b)))
    # Off: no level runs.
    g = _levels_filter(cf, m, f, b)
    g.set_eviction_levels("off")
    g.insert(ks)
    assert g.stats()["level_passes"] == 0
    # A queue threshold above any queue: the seed leaves them off.
    g = _levels_filter(cf, m, f, b)
    g.set_eviction_levels("on", 0, 1 << 31, 0)
    fl = g.insert(ks).cpu().numpy()
    st = g.stats()
    assert st["level_passes"] == 0 and st["evictions"] > 0
    assert st["occupancy"] == g.count_occupied() == int((fl == 1).sum())
    # Without the map (and so for DFS) the levels never run.
    g = _levels_filter(cf, m, f, b)
    g.set_eviction_map("off")
    g.insert(ks)
    assert g.stats()["level_passes"] == 0
    g = cf.CuckooFilter(m, f, b, 500, eviction="dfs")
    g.set_slicing("always", 1024)
    g.set_eviction_map("always")
    g.set_eviction_levels("on", 0, 1, 1)
    g.insert(ks)
    assert g.stats()["level_passes"] == 0
    with pytest.raises(Exception):
        g.set_eviction_levels("bogus")
    with pytest.raises(Exception):
        g.set_eviction_levels("on", 257)


def test_automatic_levels_only_for_narrow_buckets(cf):
    """The default mode takes the levels for buckets of up to 8 bytes, not
    for wider ones (where they measured slower than the loop); "always"
    takes them for both."""
    for (f, b), mode, runs in (((16, 4), "on", True), ((16, 16), "on", False),
                               ((16, 16), "always", True)):
        m = 1 << 10 if b == 16 else 1 << 12
        ks = workloads.keys(911 + b, int(0.96 * m * b))
        o = oracle.OracleFilter(m, f, b, 500)
        g = _levels_filter(cf, m, f, b)
        g.set_eviction_levels(mode, 0, 1, 1)
        flags = g.insert(to_dev(ks)).cpu().numpy()
        st = _check(cf, g, o, ks, flags, "xor", m, f, b)
        assert (st["level_passes"] > 0) == runs, (f, b, mode)


@pytest.mark.parametrize("mode,runs", [("on", False), ("always", True)])
def test_levels_on_host_buffer_calls(cf, mode, runs):
    """Host-buffer inserts keep the eviction loop in the default mode (the
    levels slow the copies beside them) and take the levels in "always";
    the results are valid either way."""
    m, f, b = 1 << 12, 16, 4
    ks = workloads.keys(909, int(0.96 * m * b))
    o = oracle.OracleFilter(m, f, b, 500)
    g = _levels_filter(cf, m, f, b)
    g.set_eviction_levels(mode, 0, 1, 1)
    g.set_staging_chunk(4096)
    flags = g.insert_host(ks)
    st = _check(cf, g, o, ks, flags, "xor", m, f, b)
    assert (st["level_passes"] > 0) == runs and st["evictions"] > 0
