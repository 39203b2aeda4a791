"""The named synthetic workloads, with their sizes and seeds.

Load-factor counts use floor(alpha * m * b).  All key streams are
splitmix64 outputs of one seed, so positives and negatives taken from
disjoint index ranges of the same seed are disjoint sets.
"""
from __future__ import annotations

from dataclasses import dataclass


def lf_count(m: int, b: int, alpha: float) -> int:
    """floor(alpha * m * b), computed exactly for the decimal alphas used."""
    num = round(alpha * 10**6)
    return (m * b * num) // 10**6


@dataclass(frozen=True)
class Workload:
    name: str
    m: int              # buckets
    f: int              # fingerprint bits
    b: int              # slots per bucket
    max_evictions: int
    key_seed: int
    alphas: tuple       # load factors the insert phase passes through
    n_queries: int
    query_pos_seed: int
    n_deletes: int

    @property
    def n_insert(self) -> int:
        return lf_count(self.m, self.b, self.alphas[-1])

    @property
    def table_bytes(self) -> int:
        return self.m * self.b * self.f // 8

    def insert_segments(self):
        """[(lo, hi)] key-index ranges filling 0 -> alphas[0] -> ... ."""
        out, lo = [], 0
        for a in self.alphas:
            hi = lf_count(self.m, self.b, a)
            out.append((lo, hi))
            lo = hi
        return out

    def ops_per_step(self) -> int:
        return self.n_insert + self.n_queries + self.n_deletes


# Single filter, 2^18 buckets x 4 slots, 16-bit fingerprints (2 MiB table):
# insert floor(0.95 * 2^20) keys, query them plus 2^20 disjoint negatives,
# delete the first half and query everything again.
SINGLE = Workload(name="single_2^18x4_f16", m=1 << 18, f=16, b=4,
                  max_evictions=500, key_seed=1, alphas=(0.95,),
                  n_queries=0, query_pos_seed=0, n_deletes=0)

# Single large filter, 2^28 buckets x 4 slots, 16-bit fingerprints (2 GiB):
# fill through load factors 0.5 / 0.8 / 0.95, then 2^30 queries at a 50%
# positive mix, then delete 2^28 inserted keys.
LARGE = Workload(name="large_2^28x4_f16_lf0.95", m=1 << 28, f=16, b=4,
                 max_evictions=500, key_seed=2, alphas=(0.5, 0.8, 0.95),
                 n_queries=1 << 30, query_pos_seed=12, n_deletes=1 << 28)

# The same structure at 2^24 buckets (128 MiB table, larger than L2): the
# profiling-size case of the large filter.
MEDIUM = Workload(name="medium_2^24x4_f16_lf0.95", m=1 << 24, f=16, b=4,
                  max_evictions=500, key_seed=2, alphas=(0.5, 0.8, 0.95),
                  n_queries=1 << 26, query_pos_seed=12, n_deletes=1 << 24)

# The CPU scale model of the large filter (2^22 buckets): same load-factor
# path, query mix and delete fraction; used to time the oracle and to count
# the buckets each operation touches.
SCALE = Workload(name="scale_2^22x4_f16_lf0.95", m=1 << 22, f=16, b=4,
                 max_evictions=500, key_seed=2, alphas=(0.5, 0.8, 0.95),
                 n_queries=1 << 24, query_pos_seed=12, n_deletes=1 << 22)

REF_STEP = Workload(name="ref_2^20x4_f16_lf0.95", m=1 << 20, f=16, b=4,
                    max_evictions=500, key_seed=2, alphas=(0.5, 0.8, 0.95),
                    n_queries=1 << 22, query_pos_seed=12, n_deletes=1 << 20)

# The same structure at 2^25 buckets (256 MiB table, twice L2; about 3 GB on
# the device in all): the size at which kernels are profiled with ncu.
PROFILE = Workload(name="profile_2^25x4_f16_lf0.95", m=1 << 25, f=16, b=4,
                   max_evictions=500, key_seed=2, alphas=(0.5, 0.8, 0.95),
                   n_queries=1 << 27, query_pos_seed=12, n_deletes=1 << 25)

BY_NAME = {w.name: w for w in (SINGLE, LARGE, MEDIUM, SCALE, REF_STEP, PROFILE)}


def multi_filter_layout(n_filters: int = 512, e_lo: int = 8, e_hi: int = 22,
                        u_lo: float = 2.0, u_hi: float = 6.0, b: int = 4,
                        alpha: float = 0.95, seed: int = 4):
    """The many-filters workload: filter i has m_i = 2^e_i buckets with e_i
    uniform in [e_lo, e_hi] and a key batch of round(10^u_i) keys with u_i
    uniform in [u_lo, u_hi], clipped to floor(alpha * m_i * b).  Draws come
    from splitmix64 streams `seed` (sizes) and `seed + 40` (batch sizes)."""
    from .gen import keys as _stream
    r1 = _stream(seed, n_filters)
    r2 = _stream(seed + 40, n_filters)
    out = []
    for i in range(n_filters):
        e = e_lo + int(r1[i] % (e_hi - e_lo + 1))
        u = u_lo + (u_hi - u_lo) * float(int(r2[i]) >> 11) / float(1 << 53)
        m = 1 << e
        n = min(int(round(10 ** u)), lf_count(m, b, alpha))
        out.append((m, n))
    return out


def serve_trace(n_requests: int, n_filters: int = 64, e_lo: int = 16, e_hi: int = 26,
                max_log2: float = 20.0, mix=(1, 8, 1), b: int = 4, fill: float = 0.9,
                seed: int = 5):
    """The serving workload's request sequence (host-side plan, no keys).

    Filter f has 2^e_f buckets, e_f uniform in [e_lo, e_hi]; its keys are
    splitmix64 stream 10000+f (inserted in order) and its query negatives
    stream 20000+f.  Request r picks a filter uniformly, an op with weights
    `mix` (insert : query : delete) and n = round(2^(max_log2 * u)), u
    uniform in [0, 1).  Inserts take the filter's next keys (never beyond
    `fill` of its capacity), deletes its oldest live keys, queries n/2 live
    keys (the oldest ones) then negatives; an insert or delete with nothing
    to do becomes a query.  Returns (bucket counts, requests) where each
    request is (filter, op, n, pos_start, pos_n, neg_start, neg_n): keys
    [pos_start, pos_start+pos_n) of the filter's key stream followed by
    negatives [neg_start, neg_start+neg_n)."""
    from .gen import keys as _stream
    rf = _stream(seed, n_filters)
    sizes = [1 << (e_lo + int(rf[i] % (e_hi - e_lo + 1))) for i in range(n_filters)]
    caps = [lf_count(m, b, fill) for m in sizes]
    ins = [0] * n_filters
    dele = [0] * n_filters
    neg = [0] * n_filters
    r1 = _stream(seed + 1, n_requests)
    r2 = _stream(seed + 2, n_requests)
    r3 = _stream(seed + 3, n_requests)
    tot = sum(mix)
    reqs = []
    for r in range(n_requests):
        f = int(r1[r] % n_filters)
        w = int(r2[r] % tot)
        op = "insert" if w < mix[0] else ("contains" if w < mix[0] + mix[1] else "remove")
        u = float(int(r3[r]) >> 11) / float(1 << 53)
        n = max(1, int(round(2.0 ** (max_log2 * u))))
        if op == "insert":
            n = min(n, caps[f] - ins[f])
            if n <= 0:
                op, n = "contains", max(1, int(round(2.0 ** (max_log2 * u))))
            else:
                reqs.append((f, op, n, ins[f], n, 0, 0))
                ins[f] += n
                continue
        if op == "remove":
            n = min(n, ins[f] - dele[f])
            if n <= 0:
                op, n = "contains", max(1, int(round(2.0 ** (max_log2 * u))))
            else:
                reqs.append((f, op, n, dele[f], n, 0, 0))
                dele[f] += n
                continue
        pos_n = min(n // 2, ins[f] - dele[f])
        neg_n = n - pos_n
        reqs.append((f, "contains", n, dele[f], pos_n, neg[f], neg_n))
        neg[f] += neg_n
    return sizes, reqs
