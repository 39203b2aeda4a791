"""Hand-worked pins for the parts of the oracle that the multiset, capacity
and FPR pins cannot see:

1. the slot that TryInsert (Alg. 1) fills and the copy that TryRemove
   (Alg. 3) clears: the scan starts at word (tag mod b) / tagsPerWord, wraps
   around the bucket's words, and takes the lowest lane of the first word
   that has a candidate (FindFirstSet on the SWAR mask);
2. the BFS window of Sec. 4.6.1 (reading A5): b/2 consecutive slots from
   the round's random start; the first candidate whose alternate bucket has
   room moves there; if none has, the last of the b/2 is evicted (and, for
   comparison, the one random slot of the DFS chain of Alg. 1);
3. the bucket-touch counters that the roofline's algorithmic bytes are
   built from, counted by hand for short sequences.

Each scenario is built slot by slot with set_slot on tiny tables; keys are
picked (by searching a key stream with the oracle's hash, itself pinned to
the system xxHash library) so that their fingerprint lands on the wanted
start word or their random draw on the wanted start slot.  Every expected
slot below is a literal worked out by hand in the comment beside it.

The same checks are then run against copies of the oracle with one planted
mistake each (start word 0, start word tag mod wordsPerBucket, highest lane
first, no wrap-around, all b candidates, first candidate evicted, window
walked backwards, a bucket counted twice, a query's second probe not
counted): each copy must fail at least one of them.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads

M64 = (1 << 64) - 1
HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "cf_oracle.c")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _mk(library=None):
    def make(m, f, b, max_ev=500, eviction=oracle.CFO_EVICT_BFS):
        return oracle.OracleFilter(m, f, b, max_ev, eviction=eviction, library=library)
    return make


def _find_key(o, pred, seed=900, batch=1 << 16, tries=64):
    """First key of a splitmix64 stream whose (fp, i1, i2, key) satisfies
    pred; the hash comes from the oracle filter o."""
    for t in range(tries):
        ks = workloads.keys(seed, batch, start=t * batch)
        fp, i1, i2 = o.hash_batch(ks)
        for j in range(ks.size):
            if pred(int(fp[j]), int(i1[j]), int(i2[j]), int(ks[j])):
                return int(ks[j]), int(fp[j]), int(i1[j]), int(i2[j])
    raise AssertionError("no key found")


def _filler(fp, f, k=0):
    """A nonzero tag different from fp (k-th choice)."""
    mask = (1 << f) - 1
    t = ((fp + 1 + 7 * k) & mask) or 1
    return t if t != fp else ((t + 1) & mask) or 1


def _bucket(o, j):
    return [o.get_slot(j, s) for s in range(o.b)]


def _splitmix(state):
    """splitmix64 (Steele, Lea, Flood 2014): returns (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def _draws(key, n):
    """The first n draws of a key's eviction stream (reading A6: splitmix64
    seeded with the key's 64-bit hash)."""
    s = oracle.xxh64_u64(key)
    out = []
    for _ in range(n):
        s, z = _splitmix(s)
        out.append(z)
    return out


def _fp_hash(tag):
    """H(fp) of Eq. 3 under reading A3: low 32 bits of XXH64(tag)."""
    return oracle.xxh64_u64(tag) & 0xFFFFFFFF


def _tag_with_alt(cur, target, m, f, avoid):
    """A tag t (not in avoid) whose alternate from bucket cur is target under
    the XOR policy: cur ^ (H(t) mod m) == target."""
    want = cur ^ target
    for t in range(1, 1 << min(f, 20)):
        if t not in avoid and (_fp_hash(t) & (m - 1)) == want:
            return t
    raise AssertionError("no tag")


# ---------------------------------------------------------------------------
# 1. start word, wrap-around and lane order (Alg. 1 TryInsert, Alg. 3)
# ---------------------------------------------------------------------------
# (f, b, fp mod b, pre-filled slots of bucket i1, slot the insert must fill)
# Slot s is lane s mod tpw of word s div tpw; tpw = 64/f (32/f for f8 b4).
INSERT_CASES = [
    # f16 b16: tpw 4, wpb 4.  fp mod 16 = 9 -> start word 9 div 4 = 2; word 2
    # holds slots 8..11, slot 8 is taken, so the lowest empty lane is slot 9.
    # (Scanning from word 0 gives 0, from word 9 mod 4 = 1 gives 4, the
    # highest lane first gives 11.)
    (16, 16, 9, [8], 9),
    # fp mod 16 = 13 -> start word 3 (slots 12..15) is full; the scan wraps
    # to word 0 (slots 0..3) where only slot 2 is free -> slot 2.  Words 1
    # and 2 also have room (slots 4, 9): a scan that walks backwards from
    # word 3 would take word 2 (slot 9); one that does not wrap would find
    # no room in i1 and move on to i2.
    (16, 16, 13, [12, 13, 14, 15, 0, 1, 3, 5, 6, 7, 8, 10, 11], 2),
    # fp mod 16 = 4 -> start word 1 (slots 4..7); slots 4 and 6 taken, so the
    # lowest empty lane is slot 5 (highest lane first would give 7).
    (16, 16, 4, [4, 6], 5),
    # fp mod 16 = 3 -> start word 3 div 4 = 0 -> slot 0 (taking fp mod b
    # mod wpb = 3 would give word 3, slot 12).
    (16, 16, 3, [], 0),
    # f8 b16: tpw 8, wpb 2.  fp mod 16 = 11 -> start word 1 (slots 8..15),
    # empty bucket -> slot 8.
    (8, 16, 11, [], 8),
    # fp mod 16 = 15 -> start word 1, full; wrap to word 0 where slots 0..4
    # are taken -> slot 5.
    (8, 16, 15, [8, 9, 10, 11, 12, 13, 14, 15, 0, 1, 2, 3, 4], 5),
    # f32 b16: tpw 2, wpb 8.  fp mod 16 = 13 -> start word 6 (slots 12, 13)
    # -> slot 12.
    (32, 16, 13, [], 12),
    # fp mod 16 = 15 -> start word 7 (slots 14, 15) full -> wrap to word 0
    # -> slot 0.
    (32, 16, 15, [14, 15], 0),
    # f16 b8: tpw 4, wpb 2.  fp mod 8 = 5 -> start word 1 (slots 4..7) ->
    # slot 4.
    (16, 8, 5, [], 4),
    # f16 b4: one word per bucket, start word 0 always (reading A4): slots
    # 0 and 1 taken -> slot 2.
    (16, 4, 3, [0, 1], 2),
    # f8 b4: one 32-bit word per bucket; slot 0 taken -> slot 1.
    (8, 4, 2, [0], 1),
]

# (f, b, fp mod b, slots of i1 holding a copy of fp, slot the remove must clear)
REMOVE_CASES = [
    # f16 b16, start word 2 (slots 8..11): copies in slots 1, 10, 11, 14 ->
    # the lowest match of word 2 is slot 10 (from word 0: 1; highest: 11).
    (16, 16, 9, [1, 10, 11, 14], 10),
    # start word 3 (slots 12..15) has no copy; wrap to word 0 -> slot 2
    # (walking backwards would reach word 2 first: slot 9).
    (16, 16, 13, [2, 6, 9], 2),
    # f8 b16, start word 1 (slots 8..15): copies in 3 and 12 -> slot 12.
    (8, 16, 11, [3, 12], 12),
    # f32 b16, start word 7 (slots 14, 15) has none; wrap to word 0 -> the
    # copies in slots 1 and 4: slot 1.
    (32, 16, 15, [4, 1], 1),
    # f16 b4 (one word): copies in slots 1 and 3 -> slot 1.
    (16, 4, 2, [3, 1], 1),
]


def check_insert_slot(make, f, b, r, filled, expect):
    m = 16
    o = make(m, f, b)
    key, fp, i1, i2 = _find_key(o, lambda fp, i1, i2, k: fp % b == r and i1 != i2)
    for s in filled:
        o.set_slot(i1, s, _filler(fp, f, s))
    before1, before2 = _bucket(o, i1), _bucket(o, i2)
    ok, ev = o.insert(key)
    assert ok and ev == 0
    after1 = _bucket(o, i1)
    changed = [s for s in range(b) if after1[s] != before1[s]]
    assert changed == [expect], (f, b, r, changed)
    assert after1[expect] == fp
    assert _bucket(o, i2) == before2


def check_remove_slot(make, f, b, r, copies, expect):
    m = 16
    o = make(m, f, b)
    key, fp, i1, i2 = _find_key(o, lambda fp, i1, i2, k: fp % b == r and i1 != i2)
    for s in copies:
        o.set_slot(i1, s, fp)
    before = _bucket(o, i1)
    assert o.remove(key)
    after = _bucket(o, i1)
    changed = [s for s in range(b) if after[s] != before[s]]
    assert changed == [expect], (f, b, r, changed)
    assert after[expect] == 0


def check_remove_falls_back_to_i2(make):
    # Alg. 3: TryRemove(i1) or TryRemove(i2).  fp absent from i1, present
    # in i2 at slots 9 and 14 (f16 b16, fp mod 16 = 13: start word 3 ->
    # slots 12..15 -> slot 14).  A copy in i1 always wins over one in i2.
    o = make(16, 16, 16)
    key, fp, i1, i2 = _find_key(o, lambda fp, i1, i2, k: fp % 16 == 13 and i1 != i2)
    o.set_slot(i2, 9, fp)
    o.set_slot(i2, 14, fp)
    assert o.remove(key)
    assert _bucket(o, i2)[14] == 0 and _bucket(o, i2)[9] == fp
    o.set_slot(i1, 0, fp)
    assert o.remove(key)
    assert _bucket(o, i1)[0] == 0 and _bucket(o, i2)[9] == fp


@pytest.mark.parametrize("case", INSERT_CASES, ids=lambda c: f"f{c[0]}b{c[1]}r{c[2]}")
def test_try_insert_start_word_wrap_and_lane(case):
    check_insert_slot(_mk(), *case)


@pytest.mark.parametrize("case", REMOVE_CASES, ids=lambda c: f"f{c[0]}b{c[1]}r{c[2]}")
def test_try_remove_start_word_wrap_and_lane(case):
    check_remove_slot(_mk(), *case)


def test_remove_falls_back_to_i2():
    check_remove_falls_back_to_i2(_mk())


# ---------------------------------------------------------------------------
# 2. the BFS window (Sec. 4.6.1, reading A5) and the DFS slot (Alg. 1)
# ---------------------------------------------------------------------------
M_EV, F_EV, B_EV = 16, 16, 8   # b/2 = 4 candidates out of 8 slots


def _eviction_scene(make, start, max_ev, eviction=oracle.CFO_EVICT_BFS):
    """A 16-bucket f16 b8 table, every bucket full, and a key whose two
    buckets are full and whose first eviction round starts at slot `start`.
    Returns the filter, the key, its fp, the bucket cur its chain starts
    from, and the buckets that are neither i1 nor i2."""
    o = make(M_EV, F_EV, B_EV, max_ev, eviction)

    def pred(fp, i1, i2, k):
        if i1 == i2:
            return False
        d = _draws(k, 2)
        return d[1] % B_EV == start

    key, fp, i1, i2 = _find_key(o, pred, seed=901)
    d = _draws(key, 2)
    cur = i1 if (d[0] & 1) == 0 else i2     # first draw picks the bucket
    others = [j for j in range(M_EV) if j not in (i1, i2)]
    for j in range(M_EV):
        for s in range(B_EV):
            o.set_slot(j, s, _filler(fp, F_EV, 3 * j + s + 1))
    return o, key, fp, cur, others


def _set_candidate(o, cur, slot, target, fp, used):
    t = _tag_with_alt(cur, target, M_EV, F_EV, used | {fp})
    used.add(t)
    o.set_slot(cur, slot, t)
    return t


def check_bfs_relocates_first_open_candidate(make):
    # Start slot 6 -> the b/2 = 4 candidates are slots 6, 7, 0, 1 (wrapping).
    # Alternates: slot 6 -> full bucket A, slot 7 -> bucket O1 with one free
    # slot, slot 0 -> bucket O2 with one free slot, slot 1 -> full bucket B;
    # slot 2 (outside the window) -> O2 as well.  The first candidate with
    # an open alternate is slot 7: its tag moves to O1's free slot and the
    # key's fingerprint takes slot 7.  One eviction, success.
    o, key, fp, cur, others = _eviction_scene(make, start=6, max_ev=500)
    A, O1, O2, B = others[:4]
    used = set()
    _set_candidate(o, cur, 6, A, fp, used)
    t7 = _set_candidate(o, cur, 7, O1, fp, used)
    _set_candidate(o, cur, 0, O2, fp, used)
    _set_candidate(o, cur, 1, B, fp, used)
    _set_candidate(o, cur, 2, O2, fp, used)
    o.set_slot(O1, 5, 0)   # f16 b8: fp-independent start word; one hole only
    o.set_slot(O2, 3, 0)
    before = {j: _bucket(o, j) for j in range(M_EV)}
    ok, ev = o.insert(key)
    assert ok and ev == 1
    after = {j: _bucket(o, j) for j in range(M_EV)}
    assert after[cur][7] == fp
    assert after[O1][5] == t7
    diff = sorted((j, s) for j in range(M_EV) for s in range(B_EV)
                  if after[j][s] != before[j][s])
    assert diff == sorted([(cur, 7), (O1, 5)]), diff
    st = o.stats()
    # Buckets touched: read i1 and i2 (direct attempts; cur is one of
    # them), then A (slot 6's alternate, full) and O1 (slot 7's, open):
    # 4 distinct reads; written: O1 and cur: 2.
    assert (st["ins_bucket_reads"], st["ins_bucket_writes"]) == (4, 2)
    assert (st["ins_direct_reads"], st["ins_direct_writes"]) == (2, 0)
    assert st["ins_evict_keys"] == 1 and st["evictions"] == 1


def check_bfs_evicts_last_candidate(make):
    # Start slot 5 -> candidates 5, 6, 7, 0, all with full alternates: slots
    # 5 and 6 -> bucket A, slot 7 -> B, slot 0 -> C.  Slot 1 (just after
    # the window) and slot 4 (just before it) have open alternates, which a
    # window of all b slots, or one walked backwards, would find.  With
    # max_evictions 1 the round evicts the last candidate, slot 0: the key's
    # fingerprint takes slot 0, slot 0's old tag goes to C, C is full, the
    # loop ends, and that tag is the victim, logged with bucket C.
    o, key, fp, cur, others = _eviction_scene(make, start=5, max_ev=1)
    A, B, C, O = others[:4]
    used = set()
    _set_candidate(o, cur, 5, A, fp, used)
    _set_candidate(o, cur, 6, A, fp, used)
    _set_candidate(o, cur, 7, B, fp, used)
    t0 = _set_candidate(o, cur, 0, C, fp, used)
    _set_candidate(o, cur, 1, O, fp, used)
    _set_candidate(o, cur, 4, O, fp, used)
    o.set_slot(O, 2, 0)
    before = {j: _bucket(o, j) for j in range(M_EV)}
    ok, ev = o.insert(key)
    assert not ok and ev == 1
    after = {j: _bucket(o, j) for j in range(M_EV)}
    diff = [(j, s) for j in range(M_EV) for s in range(B_EV) if after[j][s] != before[j][s]]
    assert diff == [(cur, 0)], diff
    assert after[cur][0] == fp
    vt, vb = o.victims()
    assert vt.tolist() == [t0] and vb.tolist() == [C]
    st = o.stats()
    # Reads: i1, i2, A (twice, counted once), B, C -> 5; writes: cur -> 1.
    assert (st["ins_bucket_reads"], st["ins_bucket_writes"]) == (5, 1)
    assert st["victims"] == 1 and st["insert_fail"] == 1 and st["occupancy"] == 0


def check_dfs_swaps_random_slot(make):
    # DFS (Alg. 1 phase 2): the round's draw picks slot 3; the key's
    # fingerprint takes it, slot 3's tag goes to its alternate C (full) and
    # with max_evictions 1 becomes the victim.  Slot 3's neighbours have
    # open alternates, which DFS never inspects.
    o, key, fp, cur, others = _eviction_scene(make, start=3, max_ev=1,
                                              eviction=oracle.CFO_EVICT_DFS)
    C, O = others[:2]
    used = set()
    t3 = _set_candidate(o, cur, 3, C, fp, used)
    _set_candidate(o, cur, 2, O, fp, used)
    _set_candidate(o, cur, 4, O, fp, used)
    o.set_slot(O, 0, 0)
    ok, ev = o.insert(key)
    assert not ok and ev == 1
    assert _bucket(o, cur)[3] == fp
    vt, vb = o.victims()
    assert vt.tolist() == [t3] and vb.tolist() == [C]


def test_bfs_relocates_first_open_candidate():
    check_bfs_relocates_first_open_candidate(_mk())


def test_bfs_evicts_last_candidate():
    check_bfs_evicts_last_candidate(_mk())


def test_dfs_swaps_random_slot():
    check_dfs_swaps_random_slot(_mk())


# ---------------------------------------------------------------------------
# 3. bucket-touch counters (the algorithmic bytes of the roofline)
# ---------------------------------------------------------------------------
def check_counters(make):
    m, f, b = 16, 16, 4
    o = make(m, f, b)
    key, fp, i1, i2 = _find_key(o, lambda fp, i1, i2, k: i1 != i2, seed=902)

    def st():
        return o.stats()

    # Insert into i1 (empty table): read i1, write i1.
    assert o.insert(key)[0]
    s = st()
    assert (s["ins_bucket_reads"], s["ins_bucket_writes"]) == (1, 1)
    assert (s["ins_direct_reads"], s["ins_direct_writes"], s["ins_evict_keys"]) == (1, 1, 0)
    # Query found in i1: one bucket probed (Alg. 2 short-circuits).
    assert o.contains(key)
    assert st()["qry_bucket_reads"] == 1
    # Delete found in i1: read i1, write i1.
    assert o.remove(key)
    s = st()
    assert (s["rem_bucket_reads"], s["rem_bucket_writes"]) == (1, 1)
    # Query of an absent key: both buckets probed (1 + 2 = 3 so far).
    assert not o.contains(key)
    assert st()["qry_bucket_reads"] == 3
    # Failed delete: both buckets read, nothing written (1 + 2 = 3, 1).
    assert not o.remove(key)
    s = st()
    assert (s["rem_bucket_reads"], s["rem_bucket_writes"]) == (3, 1)
    # Fill i1 with other tags: the insert reads i1 (full), reads i2, writes
    # i2: 2 reads + 1 write (totals 1 + 2 = 3 and 1 + 1 = 2).
    for sl in range(b):
        o.set_slot(i1, sl, _filler(fp, f, sl))
    assert o.insert(key)[0]
    s = st()
    assert (s["ins_bucket_reads"], s["ins_bucket_writes"]) == (3, 2)
    # Query found in i2: 2 probes (3 + 2 = 5); delete found in i2: 2 reads,
    # 1 write (3 + 2 = 5, 1 + 1 = 2).
    assert o.contains(key)
    assert st()["qry_bucket_reads"] == 5
    assert o.remove(key)
    s = st()
    assert (s["rem_bucket_reads"], s["rem_bucket_writes"]) == (5, 2)


def test_bucket_touch_counters():
    check_counters(_mk())


# ---------------------------------------------------------------------------
# planted mistakes: each mutated copy of the oracle fails a check above
# ---------------------------------------------------------------------------
START = "uint32_t start = (tag % F->b) / F->tpw;"
SCAN = "uint32_t w = (start + i) % F->wpb;"
MUTANTS = {
    "start_word_zero": [(START, "uint32_t start = 0;")],
    "start_word_mod_wpb": [(START, "uint32_t start = tag % F->wpb;")],
    "highest_lane_first": [("uint32_t s = w * F->tpw + lane;",
                            "uint32_t s = w * F->tpw + (F->tpw - 1 - lane);")],
    "no_wrap_around": [(SCAN, "uint32_t w = start + i; if (w >= F->wpb) break;")],
    "backward_wrap": [(SCAN, "uint32_t w = (start + F->wpb - i) % F->wpb;")],
    "all_b_candidates": [("const uint32_t half = F->b / 2;", "const uint32_t half = F->b;")],
    "first_candidate_evicted": [("uint32_t c = (start + half - 1) % F->b;",
                                 "uint32_t c = start % F->b;")],
    "window_backwards": [("uint32_t c = (start + k) % F->b;",
                          "uint32_t c = (start + F->b - k) % F->b;")],
    "bucket_counted_twice": [("if (set[i] == j) return;", "if (0) return;")],
    "second_probe_uncounted": [("  F->st.qry_bucket_reads++;\n  return find(",
                                "  return find(")],
}

ALL_CHECKS = (
    [lambda mk, c=c: check_insert_slot(mk, *c) for c in INSERT_CASES]
    + [lambda mk, c=c: check_remove_slot(mk, *c) for c in REMOVE_CASES]
    + [check_remove_falls_back_to_i2, check_bfs_relocates_first_open_candidate,
       check_bfs_evicts_last_candidate, check_dfs_swaps_random_slot, check_counters]
)


def _build_mutant(name, edits, tmp_path):
    src = open(ORACLE_SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-w",
                    f"-I{os.path.dirname(ORACLE_SRC)}", "-o", str(so), str(c)],
                   check=True)
    import ctypes
    return oracle.oracle.bind(ctypes.CDLL(str(so)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    L = _build_mutant(name, MUTANTS[name], tmp_path)
    mk = _mk(L)
    failed = 0
    for chk in ALL_CHECKS:
        try:
            chk(mk)
        except AssertionError:
            failed += 1
    assert failed > 0, f"planted mistake {name} passed every pin"


def test_unmutated_copy_passes_every_check(tmp_path):
    """The mutation harness itself: the oracle source built the same way,
    unchanged, passes every check."""
    L = _build_mutant("unchanged", [], tmp_path)
    mk = _mk(L)
    for chk in ALL_CHECKS:
        chk(mk)
