"""Sequential CPU cuckoo-filter oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2603_15486_gb300``)
never imports it, and the two share no code.

The arithmetic lives in ``cf_oracle.c`` (plain C, one slot at a time); this
module builds it with gcc and wraps it with ctypes and numpy.
"""
from .oracle import (  # noqa: F401
    CFO_EVICT_BFS,
    CFO_EVICT_DFS,
    CFO_POLICY_OFFSET,
    CFO_POLICY_XOR,
    OracleFilter,
    build,
    fpr_bound,
    fpr_expected,
    hash_params,
    lib,
    xxh64_u64,
)
