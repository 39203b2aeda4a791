import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than ~20 s")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


# Bounds audit (CF_BOUNDS_AUDIT=1, used with CF_LIBRARY=<libcf_debug.so> by
# tests/test_gpu_debug_bounds.py): after every test, no filter the test made
# may have hit an out-of-range bucket index (error-word bit 3).
if os.environ.get("CF_BOUNDS_AUDIT") == "1":
    import weakref

    _made = []

    @pytest.fixture(autouse=True)
    def _bounds_audit(monkeypatch):
        from paper_2603_15486_gb300 import _lib, filter as cf_filter
        assert _lib.load().cf_debug_bounds_checked() == 1, "not the checked library"
        orig = cf_filter.CuckooFilter.__init__

        def init(self, *a, **k):
            orig(self, *a, **k)
            _made.append(weakref.ref(self))

        monkeypatch.setattr(cf_filter.CuckooFilter, "__init__", init)
        _made.clear()
        yield
        for r in _made:
            f = r()
            if f is None or not f.handle:
                continue
            st = f.stats()
            assert not (st["error_word"] & 8) and st["debug_bad_index"] == 0, st
