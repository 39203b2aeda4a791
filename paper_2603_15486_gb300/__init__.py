"""GB300 (sm_103a) cuckoo filter: batched insert / query / delete of 64-bit
keys on a partial-key cuckoo table, following "Cuckoo-GPU: Accelerating
Cuckoo Filters on Modern GPUs" (Dortmann, Vieth, Schmidt, 2026).

The kernels and the C ABI live in ``libcf.so`` (``csrc/``, ``include/cf.h``);
this package only marshals arguments.  Importing fails if the library has
not been built: there is no CPU fallback.
"""
from . import _lib

_lib.load()

from .filter import (Batch, CuckooFilter, Server, hash_debug, make_config,  # noqa: E402,F401
                     plain_run_trace, required_bytes)

__all__ = ["Batch", "CuckooFilter", "Server", "hash_debug", "make_config",
           "plain_run_trace", "required_bytes"]
