"""Slice-partitioned execution (cf_set_slicing): each key still runs Alg. 1 /
2 / 3 on its own, so

  * query flags are bit-exact with the oracle on the same table, and with
    the plain kernels;
  * delete results pass the same checker as the plain path (bit-exact for
    keys whose class has no competing deleter, exact success counts per
    class, a valid final table);
  * insert results satisfy the plain path's invariants (stored multiset =
    inserted keys minus victims, counters, no false negatives).

Small slices (1 KiB) give tens to hundreds of slices on these tables, so
every pass crosses slice boundaries; duplicate-heavy batches overflow the
per-slice capacity of the second pass into its spill region; small chunk
limits run a batch as several passes with ragged tails.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import check_delete, slots_view
from gpu_util import m_for, oracle_policy, to_dev
from test_gpu_parity import EDGE_KEYS, GEOMS, POLICIES, _check_parallel_insert, _oracle_table

pytestmark = pytest.mark.gpu

SLICE = 1024


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


def _sliced(g, slice_bytes=SLICE, chunk=0):
    g.set_slicing("always", slice_bytes, chunk)
    return g


def _ran_sliced(g):
    kt = g.kernel_times()
    return kt["slice_split"][0] > 0 and kt["slice_probe1"][0] > 0


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
def test_sliced_query_bit_exact(cf, f, b, policy):
    m = m_for(policy, 1 << 12)
    o, ks = _oracle_table(f, b, policy, m)
    neg = workloads.keys(3, 3 * 8192 + 37, start=ks.size)
    q = np.concatenate([ks, neg, EDGE_KEYS, neg[:50].repeat(40)])
    g = _sliced(cf.CuckooFilter(m, f, b, 500, policy=policy))
    g.load(o.snapshot())
    g.set_kernel_timing(True)
    got = g.contains(to_dev(q)).cpu().numpy()
    assert _ran_sliced(g)
    assert np.array_equal(got, o.contains_batch(q))
    assert g.stats()["error_word"] == 0
    assert np.array_equal(g.snapshot(), o.snapshot())      # a query writes nothing
    g.set_slicing("off")
    assert np.array_equal(g.contains(to_dev(q)).cpu().numpy(), got)


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
def test_sliced_delete_parity(cf, f, b, policy):
    m = m_for(policy, 1 << 12)
    o, ks = _oracle_table(f, b, policy, m, seed=4)
    rng = np.random.default_rng(f * b + 1)
    dels = np.concatenate([ks[rng.permutation(ks.size)[: ks.size // 2]],
                           workloads.keys(4, 5000, start=ks.size),
                           ks[:300]])
    before = slots_view(o.table_words(), m, f, b).copy()
    g = _sliced(cf.CuckooFilter(m, f, b, 500, policy=policy))
    g.load(o.snapshot())
    g.set_kernel_timing(True)
    gfl = g.remove(to_dev(dels)).cpu().numpy()
    assert _ran_sliced(g)
    after = slots_view(g.snapshot()[64:], m, f, b)
    ofl = o.remove_batch(dels)
    oafter = slots_view(o.table_words(), m, f, b)
    fp, i1, i2 = o.hash_batch(dels)
    probs, n_iso = check_delete(before, after, fp, i1, i2, gfl, oracle_policy(policy), f,
                                oracle_after=oafter, oracle_flags=ofl)
    assert probs == [], probs
    assert n_iso > dels.size // 2
    st = g.stats()
    assert st["remove_ok"] == int((gfl == 1).sum())
    assert st["remove_fail"] == int((gfl != 1).sum())
    assert st["occupancy"] == int(np.count_nonzero(after))


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("eviction", ["bfs", "dfs"])
def test_sliced_insert_invariants(cf, f, b, policy, eviction):
    m = m_for(policy, 1 << 12)
    n = int(0.95 * m * b) + 3
    ks = workloads.keys(7 + f, n)
    o = oracle.OracleFilter(m, f, b, 500, policy=oracle_policy(policy))
    g = _sliced(cf.CuckooFilter(m, f, b, 500, policy=policy, eviction=eviction))
    g.set_kernel_timing(True)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    kt = g.kernel_times()
    assert kt["slice_probe2"][0] > 0 and kt["insert_direct"][0] == 0
    assert set(np.unique(flags)) <= {0, 1}
    st = _check_parallel_insert(cf, g, o, ks, flags, f, b, policy, m)
    ofl = o.insert_batch(ks)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + max(5, n // 100)


def _fill_query_delete(cf, m, f, b, slice_bytes):
    """The benchmark's protocol with the sliced path forced: fill 0 -> 0.5
    -> 0.8 -> 0.95 in three calls, query all keys plus negatives, delete
    half; every step checked as on the plain path."""
    w = workloads.Workload("t", m, f, b, 500, 2, (0.5, 0.8, 0.95), 0, 0, 0)
    ks = workloads.keys(2, w.n_insert)
    g = _sliced(cf.CuckooFilter(m, f, b, 500), slice_bytes=slice_bytes)
    g.set_kernel_timing(True)
    o = oracle.OracleFilter(m, f, b, 500)
    flags = np.concatenate([g.insert(to_dev(ks[lo:hi])).cpu().numpy()
                            for lo, hi in w.insert_segments()])
    assert _ran_sliced(g)
    st = _check_parallel_insert(cf, g, o, ks, flags, f, b, "xor", m)
    assert st["insert_fail"] <= 5
    neg = workloads.keys(2, 1 << 18, start=ks.size)
    table = g.snapshot()
    o2 = oracle.OracleFilter(m, f, b, 500)
    o2.load(table)
    q = np.concatenate([ks, neg])
    got = g.contains(to_dev(q)).cpu().numpy()
    assert np.array_equal(got, o2.contains_batch(q))
    dels = ks[: ks.size // 2]
    before = slots_view(table[64:], m, f, b).copy()
    gfl = g.remove(to_dev(dels)).cpu().numpy()
    ofl = o2.remove_batch(dels)
    fp, i1, i2 = o2.hash_batch(dels)
    probs, _ = check_delete(before, slots_view(g.snapshot()[64:], m, f, b), fp, i1, i2, gfl,
                            0, f, oracle_after=slots_view(o2.table_words(), m, f, b),
                            oracle_flags=ofl)
    assert probs == [], probs
    assert g.stats()["occupancy"] == g.count_occupied()
    assert g.stats()["error_word"] == 0


def test_sliced_insert_in_several_batches_then_query_and_delete(cf):
    """2^16 buckets in slices of 8 KiB (64 slices)."""
    _fill_query_delete(cf, 1 << 16, 16, 4, 8192)


@pytest.mark.parametrize("f,b", [(16, 4), (16, 8)])
def test_sliced_at_the_maximum_slice_count(cf, f, b):
    """Slices of one bucket's size ask for more slices than the maximum:
    the table gets 1024 slices of 64 buckets, the largest shared-memory
    footprint of the split and bucket passes."""
    _fill_query_delete(cf, 1 << 16, f, b, f * b // 8)


def test_sliced_spill_with_duplicates(cf):
    """Batches dominated by a few repeated keys overflow the per-slice
    capacity of the second pass: the overflow goes through the spill region
    and every result is still exact."""
    m, f, b = 1 << 12, 16, 4
    o, ks = _oracle_table(f, b, "xor", m, alpha=0.9, seed=8)
    neg = workloads.keys(8, 64, start=ks.size)
    q = np.concatenate([neg.repeat(600), ks[:2000], neg])
    np.random.default_rng(3).shuffle(q)
    g = _sliced(cf.CuckooFilter(m, f, b, 500))
    g.load(o.snapshot())
    assert np.array_equal(g.contains(to_dev(q)).cpu().numpy(), o.contains_batch(q))
    # Zipf-duplicated inserts into an empty filter: hot keys overflow their
    # buckets, fail, and log victims; the invariants still hold.
    zk = workloads.zipf_keys(int(0.9 * m * b), universe=2000, s=1.1)
    g2 = _sliced(cf.CuckooFilter(m, f, b, 100, victim_capacity=1 << 16))
    fl = g2.insert(to_dev(zk)).cpu().numpy()
    from cfcheck import AltTable, check_insert
    o3 = oracle.OracleFilter(m, f, b, 100)
    fp, i1, i2 = o3.hash_batch(zk)
    slots = slots_view(g2.snapshot()[64:], m, f, b)
    vt, vb = g2.victims()
    st = g2.stats()
    assert st["victims"] == vt.size == st["insert_fail"] == int((fl != 1).sum()) > 0
    assert check_insert(AltTable(o3, fp), np.zeros_like(slots), slots, fp, i1, i2,
                        vt, vb, 0) == []
    assert st["occupancy"] == int(np.count_nonzero(slots))


@pytest.mark.parametrize("f,b", [(16, 4), (8, 8)])
@pytest.mark.parametrize("chunk", [0, 9000])
def test_sliced_first_split_spill(cf, f, b, chunk):
    """One key repeated over most of a batch overflows its slice's region in
    the first split (the expected share plus six standard deviations), so
    most records take the spill region after the slices; with the chunk
    limit the batch runs as passes whose spill starts empty each time.
    Every result is still exact."""
    m = 1 << 12
    o, ks = _oracle_table(f, b, "xor", m, alpha=0.9, seed=11)
    neg = workloads.keys(11, 4000, start=ks.size)
    q = np.concatenate([ks[7:8].repeat(20000), ks[:4000], neg, neg[:3].repeat(700)])
    np.random.default_rng(5).shuffle(q)
    g = _sliced(cf.CuckooFilter(m, f, b, 500), chunk=chunk)
    g.load(o.snapshot())
    g.set_kernel_timing(True)
    got = g.contains(to_dev(q)).cpu().numpy()
    assert _ran_sliced(g)
    assert np.array_equal(got, o.contains_batch(q))
    assert g.stats()["error_word"] == 0


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 4099 * 3 + 7])
def test_sliced_chunks_tails_and_alignment(cf, n):
    """Batches split into passes of at most 4099 keys, sizes that leave
    ragged tails in every four-key loop, and flag arrays at odd addresses."""
    m, f, b = 1 << 12, 16, 4
    o, ks = _oracle_table(f, b, "xor", m, seed=9)
    q = np.concatenate([ks, workloads.keys(9, ks.size, start=ks.size)])[:n]
    g = _sliced(cf.CuckooFilter(m, f, b, 500), chunk=4099)
    g.load(o.snapshot())
    buf = torch.full((n + 1,), 7, dtype=torch.uint8, device="cuda")
    g.contains(to_dev(q), out=buf[1:])
    got = buf.cpu().numpy()
    assert got[0] == 7 and np.array_equal(got[1:], o.contains_batch(q))
    # Insert and delete through misaligned flags as well.
    g2 = _sliced(cf.CuckooFilter(m, f, b, 500), chunk=4099)
    kk = workloads.keys(10, n)
    fb = torch.full((n + 3,), 7, dtype=torch.uint8, device="cuda")
    g2.insert(to_dev(kk), flags=fb[3:])
    fl = fb.cpu().numpy()
    assert (fl[:3] == 7).all() and (fl[3:] == 1).all()
    db = torch.full((n + 1,), 7, dtype=torch.uint8, device="cuda")
    g2.remove(to_dev(kk), out=db[1:])
    dl = db.cpu().numpy()
    assert dl[0] == 7 and (dl[1:] == 1).all()
    st = g2.stats()
    assert st["occupancy"] == 0 == g2.count_occupied()


def test_sliced_without_flags(cf):
    """Insert and delete without flag arrays skip the result passes; the
    counters and the table are still right."""
    m, f, b = 1 << 12, 16, 4
    ks = workloads.keys(11, int(0.9 * m * b))
    g = _sliced(cf.CuckooFilter(m, f, b, 500))
    g.set_kernel_timing(True)
    g.insert(to_dev(ks), want_flags=False)
    torch.cuda.synchronize()
    kt = g.kernel_times()
    assert kt["slice_merge"][0] == 0 and kt["slice_probe1"][0] == 1
    st = g.stats()
    assert st["insert_ok"] == ks.size and st["insert_fail"] == 0
    assert st["occupancy"] == g.count_occupied() == ks.size
    assert g.contains(to_dev(ks)).cpu().numpy().all()
    g.remove(to_dev(ks), want_flags=False)
    torch.cuda.synchronize()
    st2 = g.stats()
    assert st2["remove_ok"] == st["insert_ok"] and st2["occupancy"] == 0 == g.count_occupied()


def test_sliced_one_slice_and_large_slices(cf):
    """slice_bytes at least the table: one slice (every record in slice 0);
    the query is still exact."""
    m, f, b = 1 << 12, 16, 4
    o, ks = _oracle_table(f, b, "xor", m, seed=12)
    q = np.concatenate([ks, workloads.keys(12, 9000, start=ks.size)])
    for sb in (1 << 20, 8, 64):
        g = _sliced(cf.CuckooFilter(m, f, b, 500), slice_bytes=sb)
        g.load(o.snapshot())
        assert np.array_equal(g.contains(to_dev(q)).cpu().numpy(), o.contains_batch(q)), sb


def test_slicing_modes_and_validation(cf):
    m, f, b = 1 << 12, 16, 4
    ks = workloads.keys(13, 5000)
    g = cf.CuckooFilter(m, f, b, 500)
    g.set_kernel_timing(True)
    g.contains(to_dev(ks))                  # auto on a 32 KiB table: plain kernels
    kt = g.kernel_times()
    assert kt["contains"][0] == 1 and kt["slice_split"][0] == 0
    g.set_slicing("always", SLICE)
    g.contains(to_dev(ks))
    assert _ran_sliced(g)
    g.set_slicing("off")
    g.contains(to_dev(ks))
    assert g.kernel_times()["slice_split"][0] == 0
    # Per-key eviction counts need the plain insert.
    g.set_slicing("always", SLICE)
    ev = torch.empty(ks.size, dtype=torch.int32, device="cuda")
    g.insert(to_dev(ks), evictions=ev)
    kt = g.kernel_times()
    assert kt["insert_direct"][0] == 1 and kt["slice_split"][0] == 0
    with pytest.raises(RuntimeError):
        g.set_slicing("always", 4)           # smaller than one 8-byte bucket
    with pytest.raises(RuntimeError):
        g.set_slicing("always", 0, (1 << 30) + 1)
