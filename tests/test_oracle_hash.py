"""Pins for the oracle's hashing (Sec. 2.1 Eq. 1-3, Sec. 4.3 step 1).

The oracle's XXH64 is checked against an independent implementation: the
system's libxxhash (the reference xxHash library), called through ctypes.
"""
import ctypes
import ctypes.util
import struct

import numpy as np
import pytest

import oracle
import workloads


def _libxxhash():
    for name in ("libxxhash.so.0", ctypes.util.find_library("xxhash")):
        if not name:
            continue
        try:
            L = ctypes.CDLL(name)
        except OSError:
            continue
        L.XXH64.restype = ctypes.c_uint64
        L.XXH64.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
        return L
    return None


XX = _libxxhash()
needs_xx = pytest.mark.skipif(XX is None, reason="libxxhash not installed")

EDGE = [0, 1, 2, 0xFF, 2**32 - 1, 2**32, 2**63, 2**64 - 1, 0x0123456789ABCDEF]


def ref_xxh64(key: int, seed: int = 0) -> int:
    b = struct.pack("<Q", key)
    return int(XX.XXH64(b, 8, seed))


@needs_xx
def test_xxh64_matches_reference_library():
    ks = list(EDGE) + [int(k) for k in workloads.keys(77, 20000)]
    for k in ks:
        assert oracle.xxh64_u64(k) == ref_xxh64(k), hex(k)


@needs_xx
def test_xxh64_seeded_matches_reference_library():
    for seed in (1, 0x9E3779B97F4A7C15, 2**64 - 1):
        for k in EDGE:
            assert oracle.xxh64_u64(k, seed) == ref_xxh64(k, seed)


@needs_xx
@pytest.mark.parametrize("f", [8, 16, 32])
@pytest.mark.parametrize("m_log", [0, 4, 18, 28, 32])
def test_hash_split_xor(f, m_log):
    """fp from the upper 32 bits (zero mapped to 1), i1 from the lower 32
    bits, i2 = i1 xor H(fp), all masked to m - 1."""
    m = 1 << m_log
    o = oracle.OracleFilter(m, f, 4, 10) if m_log <= 20 else None
    if o is None:
        # Large m: only hash, never allocate a table that size here.
        o = _HashOnly(m, f)
    mask = m - 1
    fmask = (1 << f) - 1
    for k in EDGE + [int(x) for x in workloads.keys(5, 500)]:
        h = ref_xxh64(k)
        fp = (h >> 32) & fmask
        fp = fp or 1
        i1 = (h & 0xFFFFFFFF) & mask
        i2 = i1 ^ (ref_xxh64(fp) & 0xFFFFFFFF & mask)
        assert o.hash(k) == (fp, i1, i2)


class _HashOnly:
    """Hash-only check for m too large to allocate: the split is a pure
    function of (key, f, m), so a 2^20-bucket filter's i1 is compared after
    widening the mask by hand."""

    def __init__(self, m, f):
        self.m, self.f = m, f
        self.small = oracle.OracleFilter(1 << 20, f, 4, 10)

    def hash(self, k):
        h = oracle.xxh64_u64(k)
        fp, _, _ = self.small.hash(k)
        i1 = (h & 0xFFFFFFFF) & (self.m - 1)
        i2 = i1 ^ (oracle.xxh64_u64(fp) & 0xFFFFFFFF & (self.m - 1))
        return fp, i1, i2


def test_fingerprint_zero_maps_to_one():
    """Zero is EMPTY (Alg. 3), so a key whose fingerprint bits are all zero
    gets fingerprint 1.  Find such keys by brute force for f = 8."""
    o = oracle.OracleFilter(1 << 10, 8, 4, 10)
    found = 0
    for k in range(20000):
        h = oracle.xxh64_u64(k)
        if (h >> 32) & 0xFF == 0:
            fp, i1, i2 = o.hash(k)
            assert fp == 1
            found += 1
    assert found > 10


@pytest.mark.parametrize("m_log", [1, 3, 10, 20])
def test_alternate_is_involution(m_log):
    """Eq. 3: i1 = i2 xor H(fp), so alt(alt(j, fp), fp) == j."""
    m = 1 << m_log
    o = oracle.OracleFilter(m, 16, 4, 10)
    rng = np.random.default_rng(3)
    for _ in range(3000):
        j = int(rng.integers(0, m))
        fp = int(rng.integers(1, 1 << 16))
        a = o.alt(j, fp)
        assert 0 <= a < m
        assert o.alt(a, fp) == j


def test_key_buckets_are_each_others_alternate():
    o = oracle.OracleFilter(1 << 16, 16, 4, 10)
    fp, i1, i2 = o.hash_batch(workloads.keys(9, 5000))
    for f_, a, b in zip(fp[:2000], i1[:2000], i2[:2000]):
        assert o.alt(int(a), int(f_)) == int(b)
        assert o.alt(int(b), int(f_)) == int(a)


@pytest.mark.parametrize("m", [2, 3, 1000, 12345, 1 << 16])
def test_offset_policy_alternate_round_trip(m):
    """Sec. 4.6.2: choice bit 0 -> forward by offset(fp), choice bit 1 ->
    back by offset(fp); the bit flips with the move, and the two candidate
    buckets always differ."""
    o = oracle.OracleFilter(m, 16, 4, 10, policy=oracle.CFO_POLICY_OFFSET)
    fp, i1, i2 = o.hash_batch(workloads.keys(4, 3000))
    assert (fp < (1 << 15)).all() and (fp > 0).all()
    assert (i1 < m).all() and (i2 < m).all()
    assert (i1 != i2).all()
    cb = 1 << 15
    for f_, a, b in zip(fp[:500], i1[:500], i2[:500]):
        assert o.alt(int(a), int(f_)) == int(b)
        assert o.alt(int(b), int(f_) | cb) == int(a)
        h = oracle.xxh64_u64(int(f_)) & 0xFFFFFFFF
        assert int(b) == (int(a) + 1 + h % (m - 1)) % m


def test_hash_batch_equals_single():
    o = oracle.OracleFilter(1 << 12, 16, 8, 10)
    ks = workloads.keys(11, 1000)
    fp, i1, i2 = o.hash_batch(ks)
    for k, a, b, c in zip(ks, fp, i1, i2):
        assert o.hash(int(k)) == (int(a), int(b), int(c))
