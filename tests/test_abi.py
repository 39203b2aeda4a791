"""The C-ABI library loads without a GPU and exports every symbol that
include/cf.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cf_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_cf_build", os.path.join(ROOT, "paper_2603_15486_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return ctypes.CDLL(mod.build())


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("cf_create", "cf_insert", "cf_contains", "cf_remove", "cf_snapshot",
              "cf_load", "cf_stats", "cf_hash_debug", "cf_create_at"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_every_symbol():
    from paper_2603_15486_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_host_side_validation_without_gpu(lib):
    """Pure host functions answer without touching a GPU."""
    from paper_2603_15486_gb300._lib import CfConfig, load
    L = load()
    ok = CfConfig(1 << 10, 16, 4, 500, 0, 0, 0)
    assert L.cf_table_bytes(1 << 10, 16, 4) == (1 << 10) * 4 * 2
    assert L.cf_table_bytes(1000, 8, 16) == 1000 * 16
    assert L.cf_table_bytes(1 << 32, 32, 16) == (1 << 32) * 64
    for m, f, b in ((0, 16, 4), ((1 << 32) + 1, 16, 4), (8, 12, 4), (8, 16, 6)):
        assert L.cf_table_bytes(m, f, b) == 0
    assert L.cf_required_bytes(ctypes.byref(ok)) >= (1 << 10) * 8 + 256
    for bad in (CfConfig(1000, 16, 4, 500, 0, 0, 0),     # XOR needs 2^k
                CfConfig(1 << 10, 12, 4, 500, 0, 0, 0),  # f
                CfConfig(1 << 10, 16, 6, 500, 0, 0, 0),  # b
                CfConfig(1 << 33, 16, 4, 500, 0, 0, 0),  # m > 2^32
                CfConfig(1, 16, 4, 500, 1, 0, 0),        # Offset needs m >= 2
                CfConfig(1 << 10, 16, 4, 500, 2, 0, 0)): # policy
        assert L.cf_required_bytes(ctypes.byref(bad)) == 0
    offset = CfConfig(1000, 16, 4, 500, 1, 0, 0)
    assert L.cf_required_bytes(ctypes.byref(offset)) >= 1000 * 8 + 256
    assert L.cf_status_str(0) == b"ok"
    assert L.cf_version() >= 10000
    h = ctypes.c_void_p()
    assert L.cf_create_ex(ctypes.byref(CfConfig(1000, 16, 4, 0, 0, 0, 0)),
                          ctypes.byref(h)) == 1  # CF_EINVAL before any CUDA call
    assert L.cf_destroy(None) == 0
    # Setters refuse a missing filter before touching it (CF_EINVAL).
    assert L.cf_set_eviction_levels(None, 1, 0, 0, 0) == 1
    assert L.cf_set_host_reads(None, 0) == 1
    assert L.cf_set_eviction_map(None, 1, 0) == 1
    assert L.cf_version() >= 10200
