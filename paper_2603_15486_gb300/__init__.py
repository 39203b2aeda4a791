"""GB300 (sm_103a) cuckoo filter: batched insert / query / delete of 64-bit
keys on a partial-key cuckoo table, following "Cuckoo-GPU: Accelerating
Cuckoo Filters on Modern GPUs" (Dortmann, Vieth, Schmidt, 2026).

The kernels and the C ABI live in ``libcf.so`` (``csrc/``, ``include/cf.h``);
this package only marshals arguments.  Importing fails if the library has
not been built: there is no CPU fallback.
"""
from . import _lib

_lib.load()

from .filter import CuckooFilter, hash_debug, make_config, required_bytes  # noqa: E402,F401

__all__ = ["CuckooFilter", "hash_debug", "make_config", "required_bytes"]
