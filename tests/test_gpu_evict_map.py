"""The full-bucket map of the eviction loop (cf_set_eviction_map).

The map changes where a BFS round (Sec. 4.6.1) learns whether a candidate's
alternate bucket is open (one bit per bucket instead of the bucket's words),
not what the round does.  So:

  * one GPU thread with an exact map reproduces the sequential oracle bit
    for bit (table, flags, eviction counts, victims) on every geometry and
    both bucket policies;
  * parallel inserts with the map forced on satisfy the insert invariants,
    on the plain and on the slice-partitioned path, and their failure
    counts stay within the usual margin of the oracle's;
  * the automatic rule builds the map only for tables larger than 64 MiB,
    and only for eviction queues of at least m/16 keys.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_util import m_for, oracle_policy, to_dev

pytestmark = pytest.mark.gpu

GEOMS = [(8, 4), (8, 8), (8, 16), (16, 4), (16, 8), (16, 16), (32, 4), (32, 8), (32, 16)]


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", ["xor", "offset"])
def test_serial_insert_with_map_bit_exact(cf, f, b, policy):
    m = m_for(policy, 1 << 9)
    n = int(0.985 * m * b)
    ks = workloads.keys(105 + f + b, n)
    o = oracle.OracleFilter(m, f, b, 100, policy=oracle_policy(policy))
    ofl, oev = o.insert_batch(ks, want_evictions=True)
    g = cf.CuckooFilter(m, f, b, 100, policy=policy)
    g.set_eviction_map("always")
    g.set_kernel_timing(True)
    gfl, gev = g.insert_serial(to_dev(ks))
    assert np.array_equal(g.snapshot()[64:], o.table_words())
    assert np.array_equal(gfl.cpu().numpy(), ofl)
    assert np.array_equal(gev.cpu().numpy().view(np.uint32), oev)
    ot, ob = o.victims()
    gt, gb = g.victims()
    assert np.array_equal(gt, ot) and np.array_equal(gb, ob)
    st, ost = g.stats(), o.stats()
    for k in ("occupancy", "insert_ok", "insert_fail", "evictions", "victims"):
        assert st[k] == ost[k], k
    assert oev.max() > 1


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", ["xor", "offset"])
@pytest.mark.parametrize("path", ["plain", "sliced"])
def test_parallel_insert_with_map_invariants(cf, f, b, policy, path):
    from test_gpu_parity import _check_parallel_insert
    m = m_for(policy, 1 << 12)
    n = int(0.96 * m * b) + 5
    ks = workloads.keys(117 + f, n)
    o = oracle.OracleFilter(m, f, b, 500, policy=oracle_policy(policy))
    g = cf.CuckooFilter(m, f, b, 500, policy=policy)
    g.set_eviction_map("always")
    g.set_kernel_timing(True)
    if path == "sliced":
        g.set_slicing("always", 1024)
        flags = g.insert(to_dev(ks)).cpu().numpy()
    else:
        ev = torch.empty(n, dtype=torch.int32, device="cuda")
        flags = g.insert(to_dev(ks), evictions=ev).cpu().numpy()
    kt = g.kernel_times()
    assert kt["evict_map"][0] == 1
    st = _check_parallel_insert(cf, g, o, ks, flags, f, b, policy, m)
    assert st["evictions"] > 0
    if path == "plain":
        assert st["evictions"] == int(ev.sum())
    ofl = o.insert_batch(ks)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + max(5, n // 100)


def test_map_rule(cf):
    # 2^22 buckets of 8 bytes = 32 MiB: below the automatic size rule.
    m, f, b = 1 << 22, 16, 4
    ks = to_dev(workloads.keys(131, int(0.95 * m * b)))
    g = cf.CuckooFilter(m, f, b, 500)
    g.set_kernel_timing(True)
    g.insert(ks)
    assert g.kernel_times()["evict_map"][0] == 0
    # Forced on, with a queue threshold above any queue: the map kernel is
    # launched but neither it nor the eviction loop uses the map; results
    # stay valid either way.
    g2 = cf.CuckooFilter(m, f, b, 500)
    g2.set_eviction_map("always", 1 << 31)
    g2.set_kernel_timing(True)
    fl = g2.insert(ks).cpu().numpy()
    assert g2.kernel_times()["evict_map"][0] == 1
    st = g2.stats()
    assert st["occupancy"] == g2.count_occupied() == int((fl == 1).sum())
    # DFS filters never take the map.
    g3 = cf.CuckooFilter(1 << 4, 16, 4, 50, eviction="dfs")
    g3.set_eviction_map("always")
    g3.set_kernel_timing(True)
    g3.insert(to_dev(workloads.keys(132, 60)))
    assert g3.kernel_times()["evict_map"][0] == 0
    with pytest.raises(Exception):
        g3.set_eviction_map("bogus")
