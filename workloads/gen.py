"""ctypes front end of ``gen.cu`` (host loops and device kernels)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cu")
_LIB = os.path.join(_HERE, "libcfwl.so")
_lock = threading.Lock()
_lib = None

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


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
    """Compile ``gen.cu`` into ``libcfwl.so`` in-tree for sm_103a."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and _elf_matches_host(_LIB)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run([_nvcc(), *NVCC_ARCH, "-O3", "-lineinfo", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
            L.wl_splitmix64_host.argtypes = [vp, u64, u64, u64]
            L.wl_query_mix_host.argtypes = [vp, u64, vp, u64, u64, u64, u64]
            L.wl_low32_host.argtypes = [vp, u64, u32, u64]
            L.wl_high_host.argtypes = [vp, u64, u64, u64]
            L.wl_zipf_host.argtypes = [vp, u64, u64, u64, u64, ctypes.c_double]
            for n in ("wl_splitmix64_dev", "wl_high_dev"):
                getattr(L, n).argtypes = [vp, u64, u64, u64, vp]
                getattr(L, n).restype = ctypes.c_int
            L.wl_low32_dev.argtypes = [vp, u64, u32, u64, vp]
            L.wl_low32_dev.restype = ctypes.c_int
            L.wl_query_mix_dev.argtypes = [vp, u64, vp, u64, u64, u64, u64, vp]
            L.wl_query_mix_dev.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def keys(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs [start, start+n) of the splitmix64 stream `seed` (pairwise
    distinct within one seed)."""
    out = np.empty(int(n), np.uint64)
    lib().wl_splitmix64_host(_p(out), out.size, seed, start)
    return out


def query_mix(n: int, pos_keys: np.ndarray, pos_seed: int, neg_seed: int,
              neg_start: int) -> np.ndarray:
    """50/50 mix: even j -> pos_keys[splitmix64(pos_seed)_{j/2} mod len];
    odd j -> splitmix64(neg_seed) output neg_start + j/2."""
    pk = np.ascontiguousarray(pos_keys, dtype=np.uint64)
    out = np.empty(int(n), np.uint64)
    lib().wl_query_mix_host(_p(out), out.size, _p(pk), pk.size, pos_seed,
                            neg_seed, neg_start)
    return out


def low32_keys(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Distinct keys in [0, 2^32): a 32-bit bijection of the index."""
    out = np.empty(int(n), np.uint64)
    lib().wl_low32_host(_p(out), out.size, seed & 0xFFFFFFFF, start)
    return out


def high_keys(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Keys in [2^32, 2^64) (disjoint from every low32 key)."""
    out = np.empty(int(n), np.uint64)
    lib().wl_high_host(_p(out), out.size, seed, start)
    return out


def zipf_keys(n: int, universe: int, s: float = 1.1, rank_seed: int = 33,
              key_seed: int = 3) -> np.ndarray:
    """n Zipf(s)-duplicated keys over a universe of `universe` distinct
    splitmix64 keys (continuous power-law inverse CDF; host only)."""
    out = np.empty(int(n), np.uint64)
    lib().wl_zipf_host(_p(out), out.size, rank_seed, key_seed, universe, s)
    return out


# ---- device (raw pointers from torch tensors) -------------------------------
def _chk(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} launch failed (rc={rc})")


def keys_dev(ptr: int, n: int, seed: int, start: int = 0, stream: int = 0):
    _chk(lib().wl_splitmix64_dev(ptr, n, seed, start, stream), "wl_splitmix64_dev")


def query_mix_dev(ptr: int, n: int, keys_ptr: int, n_keys: int, pos_seed: int,
                  neg_seed: int, neg_start: int, stream: int = 0):
    _chk(lib().wl_query_mix_dev(ptr, n, keys_ptr, n_keys, pos_seed, neg_seed,
                                neg_start, stream), "wl_query_mix_dev")


def low32_keys_dev(ptr: int, n: int, seed: int, start: int = 0, stream: int = 0):
    _chk(lib().wl_low32_dev(ptr, n, seed & 0xFFFFFFFF, start, stream), "wl_low32_dev")


def high_keys_dev(ptr: int, n: int, seed: int, start: int = 0, stream: int = 0):
    _chk(lib().wl_high_dev(ptr, n, seed, start, stream), "wl_high_dev")
