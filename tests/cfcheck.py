"""Invariant checkers for cuckoo-filter results (test infrastructure).

Concurrent inserts and deletes have no single correct outcome, so the tests
judge them by properties that every correct interleaving satisfies:

* insert: the multiset of stored (tag, candidate-bucket pair) classes equals
  the classes before the batch, plus one class per key in the batch, minus one
  class per logged victim; plus counter identities.
* delete: every changed lane was cleared; each successful deleter owns one
  cleared lane holding its tag in one of its buckets (a perfect matching);
  a failed deleter's tag is absent from both its buckets afterwards; deleters
  that share no (bucket, tag) with any other deleter agree bit for bit with
  the sequential oracle, and so do the buckets only they touch.

The expected classes are computed from the keys with the oracle's hash; the
alternate bucket of a stored tag comes from a table of H(fp) that the oracle
computes for the fingerprints of the KEYS, never from a GPU value.
"""
from __future__ import annotations

import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)


def slots_view(table: np.ndarray, m: int, f: int, b: int) -> np.ndarray:
    """(m, b) view of a raw table.  Slot s of bucket j is lane s mod tpw of
    word s div tpw; in little-endian memory that is element j*b + s of an
    array of f-bit integers (pinned by tests/test_oracle_layout.py)."""
    dt = {8: np.uint8, 16: np.uint16, 32: np.uint32}[f]
    t = np.ascontiguousarray(table, dtype=np.uint8)
    assert t.size == m * b * f // 8, (t.size, m, b, f)
    return t.view(dt).reshape(m, b).astype(np.uint32)


class AltTable:
    """H(fp) for a fixed set of fingerprints, computed by the oracle."""

    def __init__(self, oracle_filter, fps: np.ndarray):
        self.o = oracle_filter
        self.m = oracle_filter.m
        self.policy = oracle_filter.policy
        self.cb = (1 << (oracle_filter.f - 1)) if self.policy == 1 else 0
        self.fps = np.unique(np.asarray(fps, dtype=np.uint32))
        # alt of each fingerprint seen from bucket 0 (XOR: H(fp) & (m-1);
        # Offset: the forward offset of the fingerprint).
        alt0 = np.array([oracle_filter.alt(0, int(t)) for t in self.fps],
                        dtype=np.uint64)
        self.step = alt0

    def lookup(self, fp: np.ndarray):
        fp = np.asarray(fp, dtype=np.uint32)
        idx = np.searchsorted(self.fps, fp)
        idx = np.minimum(idx, max(self.fps.size - 1, 0))
        ok = self.fps.size > 0 and True
        ok = (self.fps[idx] == fp) if self.fps.size else np.zeros(fp.shape, bool)
        return self.step[idx], ok

    def classes(self, buckets: np.ndarray, tags: np.ndarray):
        """Canonical class (a, b) of each stored (bucket, tag).  Returns
        (a, b, known) where known is False for tags outside the key set."""
        buckets = np.asarray(buckets, dtype=np.uint64)
        tags = np.asarray(tags, dtype=np.uint32)
        if self.policy == 0:
            step, known = self.lookup(tags)
            other = buckets ^ step
            lo = np.minimum(buckets, other)
            hi = np.maximum(buckets, other)
            fp = tags.astype(np.uint64)
        else:
            fp32 = tags & np.uint32(self.cb - 1)
            off, known = self.lookup(fp32)
            in_alt = (tags & np.uint32(self.cb)) != 0
            m = np.uint64(self.m)
            lo = np.where(in_alt, (buckets + m - off) % m, buckets)
            hi = np.where(in_alt, buckets, (buckets + off) % m)
            fp = fp32.astype(np.uint64)
        a = (fp << np.uint64(32)) | lo
        return a, hi, known


def key_classes(fp, i1, i2, policy: int):
    fp = np.asarray(fp, dtype=np.uint64)
    i1 = np.asarray(i1, dtype=np.uint64)
    i2 = np.asarray(i2, dtype=np.uint64)
    if policy == 0:
        lo, hi = np.minimum(i1, i2), np.maximum(i1, i2)
    else:
        lo, hi = i1, i2
    return (fp << np.uint64(32)) | lo, hi


def multiset_delta(parts):
    """parts: list of (a, b, sign).  Returns the classes whose signed counts
    do not cancel, as (a, b, count) arrays."""
    A = np.concatenate([np.asarray(p[0], np.uint64) for p in parts])
    B = np.concatenate([np.asarray(p[1], np.uint64) for p in parts])
    W = np.concatenate([np.full(len(p[0]), p[2], np.int64) for p in parts])
    if A.size == 0:
        return A, B, W
    order = np.lexsort((B, A))
    A, B, W = A[order], B[order], W[order]
    new = np.ones(A.size, bool)
    new[1:] = (A[1:] != A[:-1]) | (B[1:] != B[:-1])
    starts = np.flatnonzero(new)
    sums = np.add.reduceat(W, starts)
    bad = sums != 0
    return A[starts][bad], B[starts][bad], sums[bad]


def check_insert(alt: AltTable, slots_before: np.ndarray, slots_after: np.ndarray,
                 fp, i1, i2, victim_tags, victim_buckets, policy: int):
    """Multiset invariant of an insert batch.  Returns a list of problems."""
    probs = []
    jb, sb = np.nonzero(slots_before)
    ja, sa = np.nonzero(slots_after)
    a0, b0, k0 = alt.classes(jb, slots_before[jb, sb])
    a1, b1, k1 = alt.classes(ja, slots_after[ja, sa])
    if not k1.all():
        probs.append(f"{int((~k1).sum())} stored tags are no key's fingerprint")
    if not k0.all():
        probs.append(f"{int((~k0).sum())} pre-existing tags unknown")
    ak, bk = key_classes(fp, i1, i2, policy)
    vt = np.asarray(victim_tags, np.uint32)
    av, bv, kv = alt.classes(np.asarray(victim_buckets, np.uint64), vt)
    if not kv.all():
        probs.append(f"{int((~kv).sum())} victims are no key's fingerprint")
    A, B, C = multiset_delta([(a0, b0, 1), (ak, bk, 1), (av, bv, -1), (a1, b1, -1)])
    if A.size:
        probs.append(f"{A.size} classes off (first: fp={int(A[0] >> np.uint64(32))} "
                     f"lo={int(A[0] & MASK32)} hi={int(B[0])} delta={int(C[0])})")
    return probs


def _resource(bucket, tag):
    return (np.asarray(bucket, np.uint64) << np.uint64(32)) | np.asarray(tag, np.uint64)


def check_delete(slots_before, slots_after, fp, i1, i2, flags, policy: int,
                 f: int, oracle_after=None, oracle_flags=None):
    """Validity of a concurrent delete batch (see module docstring).
    Returns (problems, n_isolated)."""
    probs = []
    cb = np.uint32(1 << (f - 1)) if policy == 1 else np.uint32(0)
    fp = np.asarray(fp, np.uint32)
    t1, t2 = fp, fp | cb
    i1 = np.asarray(i1, np.uint64)
    i2 = np.asarray(i2, np.uint64)
    flags = np.asarray(flags, np.uint8)
    if not np.isin(flags, (0, 1)).all():
        probs.append("flags outside {0,1}")
    ok = flags == 1
    changed = slots_before != slots_after
    if np.any(slots_after[changed] != 0):
        probs.append("a lane changed to a nonzero value")
    zj, zs = np.nonzero(changed)
    zt = slots_before[zj, zs]
    if zj.size != int(ok.sum()):
        probs.append(f"{zj.size} lanes cleared but {int(ok.sum())} successes")
    # Failed deleters: their tag must be gone from both buckets.
    fail = np.flatnonzero(~ok)
    if fail.size:
        s1 = slots_after[i1[fail].astype(np.int64)]
        s2 = slots_after[i2[fail].astype(np.int64)]
        still = (s1 == t1[fail, None]).any(1) | (s2 == t2[fail, None]).any(1)
        if still.any():
            probs.append(f"{int(still.sum())} failed deleters still have a copy")
    # Resource nodes (bucket, tag) and who wants them.
    r1 = _resource(i1, t1)
    r2 = _resource(i2, t2)
    rz = _resource(zj, zt)
    allr = np.concatenate([r1, r2[r2 != r1]])
    u, cnt = np.unique(allr, return_counts=True)

    def count_of(r):
        idx = np.searchsorted(u, r)
        return cnt[np.minimum(idx, u.size - 1)]

    iso = (count_of(r1) == 1) & (count_of(r2) == 1)
    # Cleared lanes per resource.
    zu, zc = np.unique(rz, return_counts=True)
    zmap = dict(zip(zu.tolist(), zc.tolist()))
    # Every cleared resource must be wanted by some successful deleter.
    okr = np.unique(np.concatenate([r1[ok], r2[ok]]))
    if zu.size and not np.isin(zu, okr).all():
        probs.append("a cleared lane matches no successful deleter")
    # Isolated successful deleters own exactly one cleared lane.
    for idx in np.flatnonzero(iso & ok):
        a, b = int(r1[idx]), int(r2[idx])
        got = zmap.get(a, 0) + (zmap.get(b, 0) if b != a else 0)
        if got != 1:
            probs.append(f"isolated deleter {idx} owns {got} cleared lanes")
            break
    # Contended deleters: bipartite matching per component (Kuhn).
    cont = np.flatnonzero(~iso)
    if cont.size:
        cap = {}
        for r in set(r1[cont].tolist()) | set(r2[cont].tolist()):
            cap[r] = zmap.get(r, 0)
        succ = [int(i) for i in cont if ok[i]]
        slots = []  # expand capacities into unit slots
        slot_of = {}
        for r, c in cap.items():
            for _ in range(c):
                slot_of.setdefault(r, []).append(len(slots))
                slots.append(r)
        if len(slots) != len(succ):
            probs.append(f"contended: {len(succ)} successes vs {len(slots)} cleared")
        else:
            match = [-1] * len(slots)

            def try_assign(d, seen):
                for r in {int(r1[d]), int(r2[d])}:
                    for s in slot_of.get(r, []):
                        if s in seen:
                            continue
                        seen.add(s)
                        if match[s] < 0 or try_assign(match[s], seen):
                            match[s] = d
                            return True
                return False

            for d in succ:
                if not try_assign(d, set()):
                    probs.append(f"contended deleter {d} has no cleared lane")
                    break
    # Bit-exact agreement with the oracle where the outcome is forced.
    if oracle_flags is not None:
        of = np.asarray(oracle_flags, np.uint8)
        bad = iso & (of != flags)
        if bad.any():
            probs.append(f"{int(bad.sum())} isolated deleters differ from oracle")
    if oracle_after is not None:
        touched = np.zeros(slots_before.shape[0], bool)
        touched[i1[cont].astype(np.int64)] = True
        touched[i2[cont].astype(np.int64)] = True
        diff = np.any(oracle_after != slots_after, axis=1) & ~touched
        if diff.any():
            probs.append(f"{int(diff.sum())} uncontended buckets differ from oracle")
    return probs, int(iso.sum())
