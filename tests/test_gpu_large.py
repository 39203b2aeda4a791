"""The large-filter workload at full size (2^28 buckets x 4, f16, fill to
LF 0.95 in three calls, 2^30 queries at a 50% positive mix, 2^28 deletes),
in the launch configuration bench.py times (the slice-partitioned path,
which the library picks for a table of this size).  The oracle cannot
replay a billion inserts, so outputs are checked on samples it can compute
one by one, and by properties that hold at any size:

  * hash: (fp, i1, i2) of 2^20 sampled keys bit-exact with the oracle;
  * query: for sampled queries, the flag equals the definition of Alg. 2
    ("fp is in bucket i1 or i2") evaluated on the table the GPU built, with
    the oracle's (fp, i1, i2); every sampled inserted key is present;
  * counters: occupancy = nonzero slots (device recount) = inserts - fails;
  * FPR: false positives over all 2^29 negatives within Eq. 4 + 5 sigma;
  * delete: occupancy drops by exactly the successes; sampled kept keys
    stay present up to the false deletions fingerprint collisions allow.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

W = workloads.LARGE


def _table_slots(g):
    t = g.table_view()
    return t.view(torch.int16).view(W.m, W.b)


def _definition(slots, fp, i1, i2):
    """Alg. 2 on sampled keys: any slot of i1 or i2 equal to fp."""
    fpt = torch.from_numpy(fp.astype(np.int64)).cuda()
    b1 = slots[torch.from_numpy(i1.view(np.int64)).cuda()].to(torch.int64) & 0xFFFF
    b2 = slots[torch.from_numpy(i2.view(np.int64)).cuda()].to(torch.int64) & 0xFFFF
    return ((b1 == fpt[:, None]).any(1) | (b2 == fpt[:, None]).any(1)).cpu().numpy()


def test_large_workload_full_size():
    import paper_2603_15486_gb300 as cf

    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    keys = torch.empty(W.n_insert, dtype=torch.int64, device=dev)
    workloads.keys_dev(keys.data_ptr(), W.n_insert, W.key_seed, 0, sh)
    queries = torch.empty(W.n_queries, dtype=torch.int64, device=dev)
    workloads.query_mix_dev(queries.data_ptr(), W.n_queries, keys.data_ptr(), W.n_insert,
                            W.query_pos_seed, W.key_seed, W.n_insert, sh)
    stream.synchronize()
    g = cf.CuckooFilter(W.m, W.f, W.b, W.max_evictions)
    ins_flags = torch.empty(W.n_insert, dtype=torch.uint8, device=dev)
    # Same calls as bench.py: one cf_insert per load-factor segment.
    for lo, hi in W.insert_segments():
        g.insert(keys[lo:hi], flags=ins_flags[lo:hi], stream=stream)
    stream.synchronize()
    st = g.stats()
    fails = int((ins_flags != 1).sum())
    assert fails == st["insert_fail"] == st["victims"] <= 5
    assert st["contention"] == 0 and st["error_word"] == 0
    occ = g.count_occupied()
    assert occ == st["occupancy"] == W.n_insert - fails

    rng = np.random.default_rng(2028)
    # Hash parity on sampled keys.
    pick = np.sort(rng.choice(W.n_insert, size=1 << 20, replace=False))
    sk = keys[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint64)
    gfp, gi1, gi2 = cf.hash_debug(torch.from_numpy(sk.view(np.int64)).cuda(), W.f, W.m)
    ofp, oi1, oi2 = oracle.hash_params(sk, W.m, W.f)
    assert np.array_equal(gfp.cpu().numpy().view(np.uint32), ofp)
    assert np.array_equal(gi1.cpu().numpy().view(np.uint64), oi1)
    assert np.array_equal(gi2.cpu().numpy().view(np.uint64), oi2)

    # Queries (bench launch: one cf_contains over 2^30 keys; the 2 GiB table
    # takes the slice-partitioned path by default).
    qf = g.contains(queries, stream=stream)
    stream.synchronize()
    # The plain kernels give the same 2^30 flags.
    g.set_slicing("off")
    qf_plain = g.contains(queries, stream=stream)
    stream.synchronize()
    assert torch.equal(qf, qf_plain)
    del qf_plain
    g.set_slicing("auto")
    slots = _table_slots(g)
    qpick = np.sort(rng.choice(W.n_queries, size=1 << 20, replace=False))
    qk = queries[torch.from_numpy(qpick).cuda()].cpu().numpy().view(np.uint64)
    fp, i1, i2 = oracle.hash_params(qk, W.m, W.f)
    expect = _definition(slots, fp, i1, i2)
    got = qf[torch.from_numpy(qpick).cuda()].cpu().numpy()
    assert np.array_equal(got, expect.astype(np.uint8))
    pos = (qpick % 2) == 0
    assert got[pos].all()                                   # no false negatives
    assert int(qf[0::2].sum()) == W.n_queries // 2
    alpha = occ / (W.m * W.b)
    n_neg = W.n_queries // 2
    fpc = int(qf[1::2].sum())
    assert fpc <= oracle.fpr_bound(n_neg, W.f, W.b, alpha)
    # Also the other side: at most 5 sigma below Eq. 4 (a query that
    # skipped the second bucket would halve the rate).
    e = n_neg * oracle.fpr_expected(W.f, W.b, alpha)
    assert fpc >= e - 5 * e ** 0.5

    # Deletes (bench launch: one cf_remove of the first 2^28 keys).
    before = g.stats()["occupancy"]
    df = g.remove(keys[: W.n_deletes], stream=stream)
    stream.synchronize()
    st2 = g.stats()
    ok = int(df.sum())
    assert st2["remove_ok"] == ok and before - st2["occupancy"] == ok
    assert g.count_occupied() == st2["occupancy"]
    # Every delete of an inserted key succeeds unless a concurrent deleter
    # took its fingerprint from a shared bucket first (false deletion);
    # each such event needs an equal fingerprint in a shared bucket, about
    # 2 * b * alpha / 2^16 per delete.
    steal_bound = W.n_deletes * 2 * W.b / 65535.0
    assert W.n_deletes - ok <= steal_bound
    kept = np.sort(rng.choice(np.arange(W.n_deletes, W.n_insert), size=1 << 20, replace=False))
    kq = g.contains(keys[torch.from_numpy(kept).cuda()]).cpu().numpy()
    assert (kq == 0).sum() <= (1 << 20) * 2 * 2 * W.b / 65535.0
