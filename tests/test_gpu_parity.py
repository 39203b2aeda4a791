"""GPU path (through the C ABI) against the CPU oracle.

Sizes span many warp tiles and end on a ragged tail.  Rules:
  hash, query: bit-exact;
  one-thread insert: bit-exact table, flags, eviction counts and victims;
  parallel insert: multiset invariant + counters + no false negatives;
  delete: validity checker + bit-exact where the outcome is forced.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
import workloads
from cfcheck import AltTable, check_delete, check_insert, key_classes, slots_view
from gpu_util import m_for, oracle_policy, to_dev, to_host_u32, to_host_u64

pytestmark = pytest.mark.gpu

GEOMS = [(8, 4), (8, 8), (8, 16), (16, 4), (16, 8), (16, 16), (32, 4), (32, 8), (32, 16)]
POLICIES = ["xor", "offset"]


@pytest.fixture(scope="module")
def cf():
    import paper_2603_15486_gb300 as cf
    return cf


EDGE_KEYS = np.array([0, 1, 2, 0xFF, 2**32 - 1, 2**32, 2**63, 2**64 - 1,
                      0x0123456789ABCDEF], dtype=np.uint64)


# ---------------------------------------------------------------------------
# Hash (Eq. 1-3, Sec. 4.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("f", [8, 16, 32])
@pytest.mark.parametrize("policy,m", [("xor", 1), ("xor", 2), ("xor", 1 << 10),
                                      ("xor", 1 << 18), ("xor", 1 << 28),
                                      ("xor", 1 << 32), ("offset", 2), ("offset", 3),
                                      ("offset", 12345), ("offset", (1 << 31) + 11),
                                      ("offset", (1 << 32) - 1)])
def test_hash_bit_exact(cf, f, policy, m):
    keys = np.concatenate([EDGE_KEYS, workloads.keys(17, (1 << 18) + 123)])
    fp, i1, i2 = cf.hash_debug(to_dev(keys), f, m, policy)
    ofp, oi1, oi2 = oracle.hash_params(keys, m, f, oracle_policy(policy))
    assert np.array_equal(to_host_u32(fp), ofp)
    assert np.array_equal(to_host_u64(i1), oi1)
    assert np.array_equal(to_host_u64(i2), oi2)


def test_hash_zero_fingerprint_remap(cf):
    """Keys whose 8-bit fingerprint bits are zero get fingerprint 1 on both
    sides."""
    keys = np.arange(200000, dtype=np.uint64)
    fp, _, _ = cf.hash_debug(to_dev(keys), 8, 1 << 10)
    ofp, _, _ = oracle.hash_params(keys, 1 << 10, 8)
    g = to_host_u32(fp)
    assert np.array_equal(g, ofp)
    raw0 = np.array([(oracle.xxh64_u64(int(k)) >> 32) & 0xFF == 0 for k in keys[:20000]])
    assert raw0.sum() > 10 and (g[:20000][raw0] == 1).all()


# ---------------------------------------------------------------------------
# Query (Alg. 2) and delete (Alg. 3) on an oracle-built table
# ---------------------------------------------------------------------------
def _oracle_table(f, b, policy, m, alpha=0.9, seed=3):
    o = oracle.OracleFilter(m, f, b, 500, policy=oracle_policy(policy))
    n = int(alpha * m * b)
    ks = workloads.keys(seed, n)
    o.insert_batch(ks)
    return o, ks


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
def test_query_bit_exact(cf, f, b, policy):
    m = m_for(policy, 1 << 12)
    o, ks = _oracle_table(f, b, policy, m)
    neg = workloads.keys(3, 3 * 8192 + 37, start=ks.size)
    q = np.concatenate([ks, neg, EDGE_KEYS])
    g = cf.CuckooFilter(m, f, b, 500, policy=policy)
    g.load(o.snapshot())
    assert g.stats()["occupancy"] == o.stats()["occupancy"]
    got = g.contains(to_dev(q)).cpu().numpy()
    assert np.array_equal(got, o.contains_batch(q))
    # The table round-trips bit for bit (header occupancy recounted on GPU).
    assert np.array_equal(g.snapshot(), o.snapshot())


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
def test_delete_parity(cf, f, b, policy):
    m = m_for(policy, 1 << 12)
    o, ks = _oracle_table(f, b, policy, m, seed=4)
    rng = np.random.default_rng(f * b)
    dels = np.concatenate([ks[rng.permutation(ks.size)[: ks.size // 2]],
                           workloads.keys(4, 5000, start=ks.size),
                           ks[:300]])  # some keys twice
    before = slots_view(o.table_words(), m, f, b).copy()
    g = cf.CuckooFilter(m, f, b, 500, policy=policy)
    g.load(o.snapshot())
    gfl = g.remove(to_dev(dels)).cpu().numpy()
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
    assert st["occupancy"] == int(np.count_nonzero(after))


# ---------------------------------------------------------------------------
# Insert (Alg. 1 + BFS of Sec. 4.6.1 / DFS of Alg. 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("eviction", ["bfs", "dfs"])
def test_serial_insert_bit_exact(cf, f, b, policy, eviction):
    """One GPU thread running the same insert code over the keys in order
    reproduces the sequential oracle exactly, eviction chains included."""
    m = m_for(policy, 1 << 9)
    n = int(0.985 * m * b)
    ks = workloads.keys(5 + f + b, n)
    o = oracle.OracleFilter(m, f, b, 100, policy=oracle_policy(policy),
                            eviction=0 if eviction == "bfs" else 1)
    ofl, oev = o.insert_batch(ks, want_evictions=True)
    g = cf.CuckooFilter(m, f, b, 100, policy=policy, eviction=eviction)
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
    assert oev.max() > 1  # the chains really ran


def _check_parallel_insert(cf, g, o, ks, flags, f, b, policy, m):
    """Invariants of a parallel insert of ks into an empty GPU filter g (o is
    an oracle filter with the same parameters, used for hashing only)."""
    slots = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    alt = AltTable(o, fp)
    vt, vb = g.victims()
    st = g.stats()
    before = np.zeros_like(slots)
    probs = check_insert(alt, before, slots, fp, i1, i2, vt, vb, oracle_policy(policy))
    assert probs == [], probs
    assert st["occupancy"] == int(np.count_nonzero(slots)) == g.count_occupied()
    assert st["insert_fail"] == int((flags != 1).sum()) == st["victims"] == vt.size
    assert st["contention"] == 0 and st["error_word"] == 0
    # No false negatives, except keys whose class lost a victim.
    q = g.contains(to_dev(ks)).cpu().numpy()
    miss = np.flatnonzero(q == 0)
    if miss.size:
        va, vb2, _ = alt.classes(vb, vt)
        vcls = set(zip(va.tolist(), vb2.tolist()))
        ka, kb = key_classes(fp, i1, i2, oracle_policy(policy))
        for i in miss:
            assert (int(ka[i]), int(kb[i])) in vcls
    return st


@pytest.mark.parametrize("f,b", GEOMS)
@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("eviction", ["bfs", "dfs"])
def test_parallel_insert_invariants(cf, f, b, policy, eviction):
    m = m_for(policy, 1 << 12)
    n = int(0.95 * m * b) + 3
    ks = workloads.keys(7 + f, n)
    o = oracle.OracleFilter(m, f, b, 500, policy=oracle_policy(policy))
    g = cf.CuckooFilter(m, f, b, 500, policy=policy, eviction=eviction)
    ev = torch.empty(n, dtype=torch.int32, device="cuda")
    flags = g.insert(to_dev(ks), evictions=ev).cpu().numpy()
    st = _check_parallel_insert(cf, g, o, ks, flags, f, b, policy, m)
    assert st["evictions"] == int(ev.sum())
    # Expected zero failures at LF 0.95 with 500 evictions; allow a few.
    ofl = o.insert_batch(ks)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + max(5, n // 100)


def test_parallel_insert_in_several_batches(cf):
    """Fill 0 -> 0.5 -> 0.8 -> 0.95 in three calls (the benchmark's
    protocol), on a table of 2^16 buckets."""
    m, f, b = 1 << 16, 16, 4
    w = workloads.Workload("t", m, f, b, 500, 2, (0.5, 0.8, 0.95), 0, 0, 0)
    ks = workloads.keys(2, w.n_insert)
    g = cf.CuckooFilter(m, f, b, 500)
    o = oracle.OracleFilter(m, f, b, 500)
    flags = np.concatenate([g.insert(to_dev(ks[lo:hi])).cpu().numpy()
                            for lo, hi in w.insert_segments()])
    _check_parallel_insert(cf, g, o, ks, flags, f, b, "xor", m)


# ---------------------------------------------------------------------------
# The single-filter workload: 2^18 x 4, f = 16, LF 0.95 (996,147 keys)
# ---------------------------------------------------------------------------
def test_single_filter_workload(cf):
    W = workloads.SINGLE
    m, f, b = W.m, W.f, W.b
    pos = workloads.keys(W.key_seed, W.n_insert)
    neg = workloads.keys(W.key_seed, 1 << 20, start=W.n_insert)
    o = oracle.OracleFilter(m, f, b, W.max_evictions)
    ofl = o.insert_batch(pos)
    g = cf.CuckooFilter(m, f, b, W.max_evictions)
    gfl = g.insert(to_dev(pos)).cpu().numpy()
    st = _check_parallel_insert(cf, g, o, pos, gfl, f, b, "xor", m)
    assert st["insert_fail"] <= int((ofl == 0).sum()) + 5
    # FPR on 2^20 disjoint negatives within Eq. 4 + 5 sigma.
    alpha = st["occupancy"] / (m * b)
    fpc = int(g.contains(to_dev(neg)).sum())
    assert fpc <= oracle.fpr_bound(neg.size, f, b, alpha), fpc
    # Delete the first half; the GPU's own before/after must be valid.
    before = slots_view(g.snapshot()[64:], m, f, b).copy()
    half = pos[: pos.size // 2]
    dfl = g.remove(to_dev(half)).cpu().numpy()
    after = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(half)
    probs, _ = check_delete(before, after, fp, i1, i2, dfl, 0, f)
    assert probs == [], probs
    # Re-query everything: the kept half is still there except false
    # deletions (a deleter clearing an equal tag of another key).
    kept = g.contains(to_dev(pos[pos.size // 2:])).cpu().numpy()
    assert (kept == 0).sum() <= 20
    gone = int(g.contains(to_dev(half)).sum())
    assert gone <= oracle.fpr_bound(half.size, f, b, alpha) + 20


def test_single_filter_delete_parity_on_oracle_table(cf):
    W = workloads.SINGLE
    m, f, b = W.m, W.f, W.b
    pos = workloads.keys(W.key_seed, W.n_insert)
    o = oracle.OracleFilter(m, f, b, W.max_evictions)
    o.insert_batch(pos)
    g = cf.CuckooFilter(m, f, b, W.max_evictions)
    g.load(o.snapshot())
    neg = workloads.keys(W.key_seed, 1 << 20, start=W.n_insert)
    allq = np.concatenate([pos, neg])
    assert np.array_equal(g.contains(to_dev(allq)).cpu().numpy(), o.contains_batch(allq))
    before = slots_view(o.table_words(), m, f, b).copy()
    half = pos[: pos.size // 2]
    gfl = g.remove(to_dev(half)).cpu().numpy()
    ofl = o.remove_batch(half)
    fp, i1, i2 = o.hash_batch(half)
    probs, n_iso = check_delete(before, slots_view(g.snapshot()[64:], m, f, b),
                                fp, i1, i2, gfl, 0, f,
                                oracle_after=slots_view(o.table_words(), m, f, b),
                                oracle_flags=ofl)
    assert probs == [] and n_iso > 0.99 * half.size
    assert np.array_equal(g.contains(to_dev(allq)).cpu().numpy(), o.contains_batch(allq))


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------
def test_empty_and_tiny_batches(cf):
    g = cf.CuckooFilter(1 << 8, 16, 4, 500)
    e = torch.empty(0, dtype=torch.int64, device="cuda")
    assert g.insert(e).numel() == 0
    assert g.contains(e).numel() == 0
    assert g.remove(e).numel() == 0
    one = to_dev(np.array([42], np.uint64))
    assert g.insert(one).item() == 1
    assert g.contains(one).item() == 1
    assert g.remove(one).item() == 1
    assert g.contains(one).item() == 0
    assert g.stats()["occupancy"] == 0
    g.insert(one, want_flags=False)
    torch.cuda.synchronize()
    assert g.stats()["occupancy"] == 1


@pytest.mark.parametrize("m", [1, 2, 4, 16])
@pytest.mark.parametrize("eviction", ["bfs", "dfs"])
def test_contention_stress_tiny_tables(cf, m, eviction):
    """Tiny tables, large batches with many duplicate keys: CAS races, BFS
    rollbacks, many failures.  The invariants must still hold."""
    f, b = 8, 4
    base = workloads.keys(900 + m, 8 * m)
    ks = np.concatenate([base] * 40 + [workloads.keys(901, 5000)])
    g = cf.CuckooFilter(m, f, b, 50, eviction=eviction, victim_capacity=1 << 16)
    o = oracle.OracleFilter(m, f, b, 50)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    slots = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    vt, vb = g.victims()
    st = g.stats()
    assert st["victims"] <= (1 << 16)
    probs = check_insert(AltTable(o, fp), np.zeros_like(slots), slots, fp, i1, i2,
                         vt, vb, 0)
    assert probs == [], (probs, st)
    assert st["occupancy"] == int(np.count_nonzero(slots))
    assert st["insert_fail"] == int((flags != 1).sum()) == st["victims"]
    assert st["occupancy"] <= m * b
    # CAS-retry histogram: forty copies of every key race for a few buckets,
    # so first attempts fail; a loop that failed at depth r failed at every
    # depth below it, so bin 0 >= bin 1, and bin 2 (depths 2-3) <= 2 x bin 1.
    h = st["cas_retry"]
    assert h[0] > 0 and h[0] >= h[1] and h[2] <= 2 * h[1]
    assert all(x >= 0 for x in h)


@pytest.mark.parametrize("m", [1 << 4, 1 << 6])
@pytest.mark.parametrize("eviction", ["bfs", "dfs"])
@pytest.mark.parametrize("slicing", ["off", "always"])
def test_cas_limit_runs_out(cf, m, eviction, slicing):
    """With the CAS retry bound lowered to one attempt, the duplicate-heavy
    stress makes the bounded loops run out: those keys end with
    CF_FLAG_CONTENTION and a logged victim, the counter and error-word bit 0
    report it, every kernel returns, and the invariants still hold."""
    f, b = 8, 4
    base = workloads.keys(900 + m, 8 * m)
    ks = np.concatenate([base] * 40 + [workloads.keys(901, 5000)])
    g = cf.CuckooFilter(m, f, b, 50, eviction=eviction, victim_capacity=1 << 16)
    g.set_cas_limit(1)
    if slicing == "always":
        g.set_slicing("always", 16)
    o = oracle.OracleFilter(m, f, b, 50)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    st = g.stats()
    n_cont = int((flags == 2).sum())
    assert n_cont > 0
    assert st["contention"] == n_cont
    assert st["error_word"] & 1
    # With one attempt allowed, every failed CAS was a loop's first attempt
    # (bin 0) and every loop that ran out had one: bins above 0 stay empty.
    assert st["cas_retry"][0] >= n_cont and sum(st["cas_retry"][1:]) == 0
    slots = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    vt, vb = g.victims()
    assert vt.size == st["victims"] == st["insert_fail"] == int((flags != 1).sum())
    probs = check_insert(AltTable(o, fp), np.zeros_like(slots), slots, fp, i1, i2,
                         vt, vb, 0)
    assert probs == [], (probs, st)
    assert st["occupancy"] == int(np.count_nonzero(slots))
    # The default bound restored: a fresh batch on a fresh filter has none.
    g.set_cas_limit(0)
    g2 = cf.CuckooFilter(1 << 10, f, b, 50)
    g2.insert(to_dev(workloads.keys(902, 3000)))
    assert g2.stats()["contention"] == 0
    with pytest.raises(Exception):
        g.set_cas_limit(5000)


def test_max_evictions_zero(cf):
    m, f, b = 1 << 6, 16, 4
    ks = workloads.keys(77, 2 * m * b)
    g = cf.CuckooFilter(m, f, b, 0)
    o = oracle.OracleFilter(m, f, b, 0)
    flags = g.insert(to_dev(ks)).cpu().numpy()
    st = g.stats()
    assert st["evictions"] == 0
    assert st["occupancy"] + st["insert_fail"] == ks.size
    slots = slots_view(g.snapshot()[64:], m, f, b)
    fp, i1, i2 = o.hash_batch(ks)
    vt, vb = g.victims()
    assert check_insert(AltTable(o, fp), np.zeros_like(slots), slots, fp, i1, i2,
                        vt, vb, 0) == []
    # Serial form: identical to the oracle.
    gs = cf.CuckooFilter(m, f, b, 0)
    gfl, _ = gs.insert_serial(to_dev(ks))
    assert np.array_equal(gfl.cpu().numpy(), o.insert_batch(ks))
    assert np.array_equal(gs.snapshot()[64:], o.table_words())


def test_cross_stream_calls_are_ordered(cf):
    """An insert on one stream followed by a query on another, with no
    user synchronisation: the library orders them (Sec. 4.4: no query may
    overlap a mutation)."""
    m, f, b = 1 << 20, 16, 4
    ks = workloads.keys(88, int(0.9 * m * b))
    k = to_dev(ks)
    g = cf.CuckooFilter(m, f, b, 500)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        g.insert(k, want_flags=False, stream=s1)
    out = torch.empty(ks.size, dtype=torch.uint8, device="cuda")
    g.contains(k, out=out, stream=s2)
    s2.synchronize()
    assert int(out.sum()) >= ks.size - g.stats()["insert_fail"]


def test_host_buffer_api_matches_device_api(cf):
    m, f, b = 1 << 14, 16, 8
    ks = workloads.keys(55, int(0.9 * m * b))
    neg = workloads.keys(55, 40000, start=ks.size)
    o = oracle.OracleFilter(m, f, b, 500)
    g = cf.CuckooFilter(m, f, b, 500)
    g.set_staging_chunk(7777)  # many chunks, ragged last one
    flags = g.insert_host(ks)
    _check_parallel_insert(cf, g, o, ks, flags, f, b, "xor", m)
    q = np.concatenate([ks, neg])
    hq = g.contains_host(q)
    dq = g.contains(to_dev(q)).cpu().numpy()
    assert np.array_equal(hq, dq)
    pinned = torch.from_numpy(q.view(np.int64)).pin_memory()
    out = torch.empty(q.size, dtype=torch.uint8).pin_memory()
    g.contains_host(pinned, out=out)
    assert np.array_equal(out.numpy(), dq)
    rf = g.remove_host(ks[:5000])
    assert rf.all()
    assert g.stats()["remove_ok"] == 5000


@pytest.mark.parametrize("reads", ["staged", "in_place"])
@pytest.mark.parametrize("slicing", ["off", "always"])
def test_async_host_calls_match_device_calls(cf, slicing, reads):
    """The asynchronous host-buffer calls, issued back to back without a
    synchronisation in between (insert, query, delete, query), give what
    the device calls give on the same table.  With slicing forced, passes of
    5000 keys gather their keys in staging chunks of 1777, so every pass is
    split across several chunks and the chunks across passes; or, with
    in-place reads, the scatter reads the pinned keys over the host link
    (no key copies at all)."""
    m, f, b = 1 << 12, 16, 4
    ks = workloads.keys(57, int(0.9 * m * b))
    neg = workloads.keys(57, 9000, start=ks.size)
    q = np.concatenate([ks, neg])
    g = cf.CuckooFilter(m, f, b, 500)
    g.set_staging_chunk(1777)
    g.set_host_reads(reads)
    g.set_kernel_timing(True)
    if slicing == "always":
        g.set_slicing("always", 1024, 5000)
    hk = torch.from_numpy(ks.view(np.int64)).pin_memory()
    hq = torch.from_numpy(q.view(np.int64)).pin_memory()
    fi = torch.empty(ks.size, dtype=torch.uint8).pin_memory()
    fq = torch.empty(q.size, dtype=torch.uint8).pin_memory()
    fd = torch.empty(4000, dtype=torch.uint8).pin_memory()
    fq2 = torch.empty(q.size, dtype=torch.uint8).pin_memory()
    st = torch.cuda.Stream()
    g.insert_host_async(hk, out=fi, stream=st)
    g.contains_host_async(hq, out=fq, stream=st)
    g.remove_host_async(hk[:4000], out=fd, stream=st)
    g.contains_host_async(hq, out=fq2, stream=st)
    st.synchronize()
    h2d = g.kernel_times()["copy_h2d"][0]
    assert (h2d == 0) == (reads == "in_place" and slicing == "always")
    flags = fi.numpy()
    # The inserts: the invariants on the table as it stood after them are
    # checked through the first query (every key found) and the counters.
    assert (flags == 1).all()
    assert fq.numpy()[: ks.size].all()
    assert fd.numpy().all()
    # Device calls on the final table agree with the last async query.
    dq = g.contains(to_dev(q)).cpu().numpy()
    assert np.array_equal(fq2.numpy(), dq)
    st_ = g.stats()
    assert st_["insert_ok"] == ks.size and st_["remove_ok"] == 4000
    assert st_["occupancy"] == ks.size - 4000 == g.count_occupied()
    # The last query equals Alg. 2 evaluated by the oracle on the table the
    # calls left.
    ot = oracle.OracleFilter(m, f, b, 500)
    ot.load(g.snapshot())
    assert np.array_equal(ot.contains_batch(q), fq2.numpy())


def test_in_place_reads_fall_back_to_copies_for_pageable_keys(cf):
    """In-place reads take only pinned keys; a pageable numpy buffer keeps
    the staged copies, with the same results."""
    m, f, b = 1 << 12, 16, 4
    ks = workloads.keys(59, int(0.9 * m * b))
    g = cf.CuckooFilter(m, f, b, 500)
    g.set_slicing("always", 1024, 5000)
    g.set_host_reads("in_place")
    g.set_kernel_timing(True)
    fl = g.insert_host(ks)
    assert (fl == 1).all() and g.kernel_times()["copy_h2d"][0] > 0
    assert g.contains_host(ks).all()
    with pytest.raises(Exception):
        g.set_host_reads("bogus")


def test_create_at_caller_memory(cf):
    m, f, b = 1 << 12, 32, 8
    nbytes = cf.required_bytes(num_buckets=m, fp_bits=f, slots_per_bucket=b)
    mem = torch.full((nbytes + 256,), 0xAB, dtype=torch.uint8, device="cuda")
    off = (-mem.data_ptr()) % 256
    g = cf.CuckooFilter(m, f, b, 500, memory=mem[off: off + nbytes])
    ks = workloads.keys(66, 5000)
    assert g.insert(to_dev(ks)).all()
    assert g.contains(to_dev(ks)).all()
    g.close()
    with pytest.raises(RuntimeError):
        cf.CuckooFilter(m, f, b, 500, memory=mem[:nbytes // 2])


def test_snapshot_device_round_trip_and_bad_header(cf):
    m, f, b = 1 << 12, 16, 4
    g = cf.CuckooFilter(m, f, b, 500)
    ks = workloads.keys(12, 10000)
    g.insert(to_dev(ks))
    snap = g.snapshot(device=True)
    h = cf.CuckooFilter(m, f, b, 500)
    h.load(snap)
    assert np.array_equal(h.snapshot(), g.snapshot())
    assert h.stats()["occupancy"] == g.stats()["occupancy"]
    other = cf.CuckooFilter(m, f, 8, 500)
    with pytest.raises(RuntimeError):
        other.load(snap)
    g.clear()
    assert g.stats()["occupancy"] == 0 and g.count_occupied() == 0
