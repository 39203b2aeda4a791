"""Seeded synthetic workloads for the cuckoo filter (inputs only).

This package holds no filter arithmetic.  It generates keys and query mixes
with counter-based splitmix64 streams (``gen.cu``), on the host (numpy
arrays) or on the device (raw device pointers + a CUDA stream), so that the
oracle tests, the GPU tests and the benchmark all see identical bytes.

The named workloads mirror the paper's synthetic setup (Sec. 5.2: uniform
64-bit keys, 16-bit fingerprints, 95% load factor; Sec. 5.3: positives in
[0, 2^32), negatives in [2^32, 2^64)).
"""
from .gen import (  # noqa: F401
    build,
    high_keys,
    high_keys_dev,
    keys,
    keys_dev,
    lib,
    low32_keys,
    low32_keys_dev,
    query_mix,
    query_mix_dev,
    zipf_keys,
)
from .configs import (  # noqa: F401
    BY_NAME,
    LARGE,
    MEDIUM,
    REF_STEP,
    SCALE,
    SINGLE,
    Workload,
    lf_count,
    multi_filter_layout,
    serve_trace,
)
