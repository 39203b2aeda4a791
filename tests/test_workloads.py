"""Pins for the input generators (not part of the method)."""
import numpy as np

import workloads


def test_splitmix64_reference_value():
    # splitmix64 started from state 0 yields 0xE220A8397B1DCDAF first
    # (published reference output of the generator).
    assert int(workloads.keys(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_streams_are_counter_based():
    a = workloads.keys(3, 1000)
    b = workloads.keys(3, 400, start=600)
    assert np.array_equal(a[600:], b)


def test_first_outputs_distinct_and_ranges_disjoint():
    a = workloads.keys(1, 1 << 20)
    assert np.unique(a).size == a.size
    neg = workloads.keys(1, 1 << 18, start=1 << 20)
    assert not np.isin(neg, a).any()


def test_query_mix_structure():
    pos = workloads.keys(2, 5000)
    q = workloads.query_mix(4000, pos, 12, 2, 5000)
    assert np.isin(q[0::2], pos).all()
    assert not np.isin(q[1::2], pos).any()
    assert np.array_equal(q[1::2], workloads.keys(2, 2000, start=5000))


def test_low_and_high_ranges():
    lo = workloads.low32_keys(7, 1 << 16)
    hi = workloads.high_keys(8, 1 << 16)
    assert (lo < (1 << 32)).all() and np.unique(lo).size == lo.size
    assert (hi >= (1 << 32)).all()


def test_load_factor_counts():
    assert workloads.lf_count(1 << 18, 4, 0.95) == 996147
    assert workloads.lf_count(1 << 28, 4, 0.95) == 1020054732
    assert workloads.lf_count(1 << 28, 4, 0.8) == 858993459
    assert workloads.LARGE.insert_segments()[-1] == (858993459, 1020054732)


def test_zipf_keys_are_skewed_and_from_the_universe():
    z = workloads.zipf_keys(200000, 50000, 1.1)
    uni = workloads.keys(3, 50000)
    assert np.isin(z, uni).all()
    vals, counts = np.unique(z, return_counts=True)
    counts = np.sort(counts)[::-1]
    # Rank 1 is the most frequent key: P(r=1) is about 1 - 2^(-0.1) of the
    # continuous law's mass on [1, 2), far above uniform.
    assert counts[0] > 20 * 200000 / 50000
    assert int((z == uni[0]).sum()) == int(counts[0])  # rank 1 = first key
