"""The bounds-checked build of the library (libcf_debug.so: every bucket
index range-checked on the device, a bad one recorded in the error word and
clamped, never trapped).

* In the normal build the touch export refuses an index beyond the table on
  the host.
* The checked build is built, and the small parity suites (plain and sliced
  paths, the full-bucket map, the eviction levels, batched launches) run
  against it in a subprocess, with every filter audited for bounds
  violations after each test; the checked build's own check is shown to
  catch a planted bad index.
"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_touch_refuses_out_of_range_in_normal_build():
    import ctypes

    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib
    L = _lib.load()
    if L.cf_debug_bounds_checked():
        pytest.skip("this process runs the checked build")
    g = cf.CuckooFilter(1 << 10, 16, 4, 500)
    occ = ctypes.c_uint64()
    assert L.cf_debug_touch_bucket(g.handle, 1 << 10, ctypes.byref(occ), None) == 1
    g.insert(torch.arange(1, 2001, dtype=torch.int64, device="cuda"))
    total = 0
    for j in (0, 1, (1 << 10) - 1):
        assert L.cf_debug_touch_bucket(g.handle, j, ctypes.byref(occ), None) == 0
        total += occ.value
    assert 0 <= total <= 12


def test_checked_build_catches_a_bad_index():
    import ctypes

    import paper_2603_15486_gb300 as cf
    from paper_2603_15486_gb300 import _lib
    L = _lib.load()
    if not L.cf_debug_bounds_checked():
        pytest.skip("runs in the checked build only (see the next test)")
    m = 1 << 10
    g = cf.CuckooFilter(m, 16, 4, 500)
    occ = ctypes.c_uint64()
    assert L.cf_debug_touch_bucket(g.handle, m + 5, ctypes.byref(occ), None) == 0
    st = g.stats()
    assert st["error_word"] & 8 and st["debug_bad_index"] == m + 6
    g.close()  # keep the audit fixture from flagging this planted case


@pytest.mark.slow
def test_parity_suites_under_the_checked_build():
    if os.environ.get("CF_BOUNDS_AUDIT") == "1":
        pytest.skip("already inside the audited run")
    sys.path.insert(0, os.path.join(ROOT, "paper_2603_15486_gb300"))
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_cf_build", os.path.join(ROOT, "paper_2603_15486_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = mod.build(debug_bounds=True)
    env = dict(os.environ, CF_LIBRARY=lib, CF_BOUNDS_AUDIT="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "gpu",
           os.path.join(ROOT, "tests", "test_gpu_parity.py"),
           os.path.join(ROOT, "tests", "test_gpu_slice.py"),
           os.path.join(ROOT, "tests", "test_gpu_evict_map.py"),
           os.path.join(ROOT, "tests", "test_gpu_levels.py"),
           os.path.join(ROOT, "tests", "test_gpu_batched.py"),
           os.path.join(ROOT, "tests", "test_gpu_debug_bounds.py"),
           "-k", "not cas_limit and not parity_suites_under"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
