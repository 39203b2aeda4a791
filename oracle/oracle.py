"""ctypes wrapper around the C oracle (TEST INFRASTRUCTURE ONLY).

See ``cf_oracle.h`` for what each call computes and which part of the paper it
follows.  Arrays are numpy; every batch runs strictly in key order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFO_POLICY_XOR = 0
CFO_POLICY_OFFSET = 1
CFO_EVICT_BFS = 0
CFO_EVICT_DFS = 1

_lock = threading.Lock()
_lib = None


def _elf_matches_host(path: str) -> bool:
    """True if `path` is an ELF file built for this machine's architecture
    (x86-64 objects can travel to an Arm host with the source tree)."""
    import platform
    want = {"x86_64": 0x3E, "amd64": 0x3E, "aarch64": 0xB7, "arm64": 0xB7}.get(
        platform.machine().lower())
    try:
        with open(path, "rb") as fh:
            hdr = fh.read(20)
    except OSError:
        return False
    if len(hdr) < 20 or hdr[:4] != b"\x7fELF":
        return False
    return want is None or int.from_bytes(hdr[18:20], "little") == want


def build(force: bool = False) -> str:
    """Compile ``cf_oracle.c`` into ``liboracle.so`` next to it (plain gcc,
    no architecture-specific flags, so it builds the same on x86 and Arm)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(_SRC[:-1] + "h"))
            and _elf_matches_host(_LIB)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared",
                    "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "occupancy", "insert_ok", "insert_fail", "remove_ok", "remove_fail",
        "evictions", "victims", "ins_bucket_reads", "ins_bucket_writes",
        "qry_bucket_reads", "rem_bucket_reads", "rem_bucket_writes",
        "ins_direct_reads", "ins_direct_writes", "ins_evict_keys")]


def bind(L):
    """Set the ctypes signatures of an oracle library handle."""
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    L.cfo_create.restype = vp
    L.cfo_create.argtypes = [u64, u32, u32, u32, u32, u32]
    L.cfo_destroy.argtypes = [vp]
    L.cfo_clear.argtypes = [vp]
    L.cfo_xxh64_u64.restype = u64
    L.cfo_xxh64_u64.argtypes = [u64, u64]
    L.cfo_hash.argtypes = [vp, u64, vp, vp, vp]
    L.cfo_alt.restype = u64
    L.cfo_alt.argtypes = [vp, u64, u32]
    L.cfo_insert.restype = ctypes.c_int
    L.cfo_insert.argtypes = [vp, u64, vp]
    L.cfo_contains.restype = ctypes.c_int
    L.cfo_contains.argtypes = [vp, u64]
    L.cfo_remove.restype = ctypes.c_int
    L.cfo_remove.argtypes = [vp, u64]
    for name in ("cfo_insert_batch",):
        getattr(L, name).argtypes = [vp, vp, u64, vp, vp]
    for name in ("cfo_contains_batch", "cfo_remove_batch"):
        getattr(L, name).argtypes = [vp, vp, u64, vp]
    L.cfo_hash_batch.argtypes = [vp, vp, u64, vp, vp, vp]
    L.cfo_hash_params_batch.restype = ctypes.c_int
    L.cfo_hash_params_batch.argtypes = [u64, u32, u32, vp, u64, vp, vp, vp]
    L.cfo_get_slot.restype = u32
    L.cfo_get_slot.argtypes = [vp, u64, u32]
    L.cfo_set_slot.argtypes = [vp, u64, u32, u32]
    L.cfo_table_bytes.restype = u64
    L.cfo_table_bytes.argtypes = [vp]
    L.cfo_snapshot_bytes.restype = u64
    L.cfo_snapshot_bytes.argtypes = [vp]
    L.cfo_snapshot.restype = ctypes.c_int
    L.cfo_snapshot.argtypes = [vp, vp, u64]
    L.cfo_load.restype = ctypes.c_int
    L.cfo_load.argtypes = [vp, vp, u64]
    L.cfo_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    L.cfo_victims.restype = u64
    L.cfo_victims.argtypes = [vp, vp, vp, u64]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(ctypes.CDLL(_LIB))
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def xxh64_u64(key: int, seed: int = 0) -> int:
    return int(lib().cfo_xxh64_u64(int(key) & (2**64 - 1), seed))


def hash_params(keys, m: int, f: int, policy: int = CFO_POLICY_XOR):
    """(fp, i1, i2) of every key for a filter with m buckets, f-bit
    fingerprints and the given policy (no table is allocated)."""
    k = _u64(keys)
    fp = np.empty(k.size, np.uint32)
    i1 = np.empty(k.size, np.uint64)
    i2 = np.empty(k.size, np.uint64)
    rc = lib().cfo_hash_params_batch(int(m), int(f), int(policy), _ptr(k), k.size,
                                     _ptr(fp), _ptr(i1), _ptr(i2))
    if rc != 0:
        raise ValueError(f"invalid hash parameters m={m} f={f} policy={policy}")
    return fp, i1, i2


def fpr_expected(f: int, b: int, alpha: float, policy: int = CFO_POLICY_XOR) -> float:
    """Eq. 4 (Sec. 2.1) with the fingerprint alphabet used here: the
    fingerprint is never zero, so it takes 2^f - 1 values (2^(f-1) - 1 under
    the Offset policy, whose top tag bit is the choice bit)."""
    vals = (2 ** f - 1) if policy == CFO_POLICY_XOR else (2 ** (f - 1) - 1)
    return 1.0 - (1.0 - 1.0 / vals) ** (2 * b * alpha)


def fpr_bound(n_neg: int, f: int, b: int, alpha: float,
              policy: int = CFO_POLICY_XOR) -> float:
    """Largest false-positive COUNT accepted on n_neg negatives: the Eq. 4
    expectation E plus five standard deviations of a Poisson count, plus 1."""
    e = n_neg * fpr_expected(f, b, alpha, policy)
    return e + 5.0 * math.sqrt(e) + 1.0


class OracleFilter:
    """One sequential filter.  ``m`` buckets of ``b`` slots of ``f`` bits."""

    def __init__(self, m: int, f: int = 16, b: int = 4, max_evictions: int = 500,
                 policy: int = CFO_POLICY_XOR, eviction: int = CFO_EVICT_BFS,
                 library=None):
        # `library`: another build of the oracle source bound with bind()
        # (the tests' planted-mistake variants); default: liboracle.so.
        self._L = library if library is not None else lib()
        self.m, self.f, self.b = int(m), int(f), int(b)
        self.max_evictions, self.policy, self.eviction = max_evictions, policy, eviction
        h = self._L.cfo_create(self.m, f, b, max_evictions, policy, eviction)
        if not h:
            raise ValueError(f"invalid oracle parameters m={m} f={f} b={b} "
                             f"policy={policy} eviction={eviction}")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.cfo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- single-key --------------------------------------------------------
    def hash(self, key: int):
        fp, i1, i2 = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
        self._L.cfo_hash(self._h, int(key) & (2**64 - 1), ctypes.byref(fp),
                         ctypes.byref(i1), ctypes.byref(i2))
        return fp.value, i1.value, i2.value

    def alt(self, j: int, tag: int) -> int:
        return int(self._L.cfo_alt(self._h, j, tag))

    def insert(self, key: int):
        ev = ctypes.c_uint32()
        ok = self._L.cfo_insert(self._h, int(key) & (2**64 - 1), ctypes.byref(ev))
        return bool(ok), ev.value

    def contains(self, key: int) -> bool:
        return bool(self._L.cfo_contains(self._h, int(key) & (2**64 - 1)))

    def remove(self, key: int) -> bool:
        return bool(self._L.cfo_remove(self._h, int(key) & (2**64 - 1)))

    # -- batches -----------------------------------------------------------
    def hash_batch(self, keys):
        k = _u64(keys)
        fp = np.empty(k.size, np.uint32)
        i1 = np.empty(k.size, np.uint64)
        i2 = np.empty(k.size, np.uint64)
        self._L.cfo_hash_batch(self._h, _ptr(k), k.size, _ptr(fp), _ptr(i1), _ptr(i2))
        return fp, i1, i2

    def insert_batch(self, keys, want_evictions: bool = False):
        k = _u64(keys)
        flags = np.empty(k.size, np.uint8)
        ev = np.empty(k.size, np.uint32) if want_evictions else None
        self._L.cfo_insert_batch(self._h, _ptr(k), k.size, _ptr(flags),
                                 _ptr(ev) if ev is not None else None)
        return (flags, ev) if want_evictions else flags

    def contains_batch(self, keys) -> np.ndarray:
        k = _u64(keys)
        flags = np.empty(k.size, np.uint8)
        self._L.cfo_contains_batch(self._h, _ptr(k), k.size, _ptr(flags))
        return flags

    def remove_batch(self, keys) -> np.ndarray:
        k = _u64(keys)
        flags = np.empty(k.size, np.uint8)
        self._L.cfo_remove_batch(self._h, _ptr(k), k.size, _ptr(flags))
        return flags

    # -- state ---------------------------------------------------------------
    def clear(self):
        self._L.cfo_clear(self._h)

    def get_slot(self, j: int, s: int) -> int:
        return int(self._L.cfo_get_slot(self._h, j, s))

    def set_slot(self, j: int, s: int, tag: int):
        self._L.cfo_set_slot(self._h, j, s, tag)

    def table_bytes(self) -> int:
        return int(self._L.cfo_table_bytes(self._h))

    def snapshot(self) -> np.ndarray:
        n = int(self._L.cfo_snapshot_bytes(self._h))
        buf = np.empty(n, np.uint8)
        rc = self._L.cfo_snapshot(self._h, _ptr(buf), n)
        if rc != 0:
            raise RuntimeError(f"cfo_snapshot failed: {rc}")
        return buf

    def load(self, snap: np.ndarray):
        buf = np.ascontiguousarray(snap, dtype=np.uint8)
        rc = self._L.cfo_load(self._h, _ptr(buf), buf.size)
        if rc != 0:
            raise RuntimeError(f"cfo_load failed: {rc}")

    def table_words(self) -> np.ndarray:
        """The raw table (no header) as bytes."""
        return self.snapshot()[64:]

    def slots(self) -> np.ndarray:
        """The table as an (m, b) array of stored tags, read slot by slot
        through the oracle's own layout code (slow; for small m)."""
        out = np.empty((self.m, self.b), np.uint32)
        g = self._L.cfo_get_slot
        for j in range(self.m):
            for s in range(self.b):
                out[j, s] = g(self._h, j, s)
        return out

    def stats(self) -> dict:
        st = _Stats()
        self._L.cfo_get_stats(self._h, ctypes.byref(st))
        return {n: int(getattr(st, n)) for n, _ in _Stats._fields_}

    def victims(self):
        n = int(self._L.cfo_victims(self._h, None, None, 0))
        tags = np.empty(n, np.uint32)
        buckets = np.empty(n, np.uint64)
        if n:
            self._L.cfo_victims(self._h, _ptr(tags), _ptr(buckets), n)
        return tags, buckets
