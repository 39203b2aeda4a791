"""Pins for the oracle's table layout (Sec. 4.2, Fig. 2) and snapshot format."""
import json
import os

import numpy as np
import pytest

import oracle
from cfcheck import slots_view

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig2_layout.json")


def test_fig2_word_packing():
    cases = json.load(open(GOLD))["cases"]
    for c in cases:
        o = oracle.OracleFilter(4, c["f"], c["b"], 10)
        for s, v in enumerate(c["slots"]):
            o.set_slot(2, s, v)
        table = o.table_words()
        wbytes = 8
        bucket_bytes = c["f"] * c["b"] // 8
        word = table[2 * bucket_bytes: 2 * bucket_bytes + wbytes].view(np.uint64)[0]
        assert f"{int(word):016x}" == c["word_hex"]
        # The other buckets stay empty.
        assert int(table[:2 * bucket_bytes].sum()) == 0


@pytest.mark.parametrize("f,b", [(8, 4), (8, 8), (8, 16), (16, 4), (16, 8),
                                 (16, 16), (32, 4), (32, 8), (32, 16)])
def test_slot_addressing_matches_element_view(f, b):
    """Slot s of bucket j sits in word s div tpw at lane s mod tpw; on a
    little-endian machine this is element j*b + s of an f-bit array."""
    m = 16
    o = oracle.OracleFilter(m, f, b, 10)
    rng = np.random.default_rng(f * 100 + b)
    ref = rng.integers(1, 1 << f, size=(m, b), dtype=np.uint64).astype(np.uint32)
    for j in range(m):
        for s in range(b):
            o.set_slot(j, s, int(ref[j, s]))
    assert o.table_bytes() == m * b * f // 8
    got = slots_view(o.table_words(), m, f, b)
    assert np.array_equal(got, ref)
    assert np.array_equal(o.slots(), ref)
    # Words are 64-bit except the 32-bit bucket f=8, b=4.
    if f * b == 32:
        w = o.table_words().view(np.uint32)
        assert int(w[0]) == sum(int(ref[0, s]) << (8 * s) for s in range(4))
    else:
        w = o.table_words().view(np.uint64)
        tpw = 64 // f
        for s in range(b):
            word = int(w[s // tpw])
            assert (word >> ((s % tpw) * f)) & ((1 << f) - 1) == int(ref[0, s])


def test_snapshot_round_trip_and_header():
    o = oracle.OracleFilter(1 << 10, 16, 8, 33)
    import workloads
    o.insert_batch(workloads.keys(3, 6000))
    snap = o.snapshot()
    assert snap.size == 64 + o.table_bytes()
    hdr = snap[:64]
    assert hdr[:4].tobytes() == b"CFG1"
    assert int(hdr[8:16].view(np.uint64)[0]) == 1 << 10
    assert int(hdr[16:20].view(np.uint32)[0]) == 16
    assert int(hdr[20:24].view(np.uint32)[0]) == 8
    assert int(hdr[24:28].view(np.uint32)[0]) == 33
    assert int(hdr[32:40].view(np.uint64)[0]) == o.stats()["occupancy"]
    o2 = oracle.OracleFilter(1 << 10, 16, 8, 33)
    o2.load(snap)
    assert np.array_equal(o2.snapshot(), snap)
    assert o2.stats()["occupancy"] == int(np.count_nonzero(slots_view(
        snap[64:], 1 << 10, 16, 8)))
    bad = oracle.OracleFilter(1 << 10, 16, 4, 33)
    with pytest.raises(RuntimeError):
        bad.load(snap)
