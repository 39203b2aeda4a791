"""ctypes loader for libcf.so (the CUDA kernels + C ABI of include/cf.h).

There is no fallback: if the shared library is missing or does not load,
importing the package raises.  Build it with ``python -c "import
__graft_entry__ as g; g.build()"`` or ``python paper_2603_15486_gb300/build.py``.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# CF_LIBRARY selects another build of the same library (the bounds-checked
# libcf_debug.so that build.py --debug-bounds makes); default libcf.so.
LIB_PATH = os.environ.get("CF_LIBRARY") or os.path.join(HERE, "libcf.so")


class CfConfig(ctypes.Structure):
    _fields_ = [("num_buckets", ctypes.c_uint64), ("fp_bits", ctypes.c_uint32),
                ("slots_per_bucket", ctypes.c_uint32),
                ("max_evictions", ctypes.c_uint32), ("policy", ctypes.c_uint32),
                ("eviction", ctypes.c_uint32), ("victim_capacity", ctypes.c_uint32)]


class CfStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "occupancy", "insert_ok", "insert_fail", "remove_ok", "remove_fail",
        "evictions", "victims", "rollbacks", "rollback_lost", "contention")] + [
        ("error_word", ctypes.c_uint32), ("victim_capacity", ctypes.c_uint32),
        ("map_builds", ctypes.c_uint64), ("cas_retry", ctypes.c_uint64 * 7),
        ("debug_bad_index", ctypes.c_uint64),
        ("level_passes", ctypes.c_uint64), ("level_steps", ctypes.c_uint64),
        ("level_runout", ctypes.c_uint64)]


class CfBatchItem(ctypes.Structure):
    _fields_ = [("filter", ctypes.c_void_p), ("keys", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("out_flags", ctypes.c_void_p),
                ("op", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class CfTuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_uint32), ("keys_per_thread", ctypes.c_uint32),
                ("block", ctypes.c_uint32), ("frontier", ctypes.c_uint32),
                ("ms", ctypes.c_float)]


class CfServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_wave_items", ctypes.c_uint32), ("max_wave_keys", ctypes.c_uint64),
                ("use_graphs", ctypes.c_uint32), ("watchdog_us", ctypes.c_uint32)]


class CfRequest(ctypes.Structure):
    _fields_ = [("filter_id", ctypes.c_uint32), ("op", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("out_flags", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class CfCompletion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("tag", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("wave_size", ctypes.c_uint32),
                ("submit_s", ctypes.c_double), ("launch_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class CfServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "waves", "late_waves", "keys_completed", "used_bytes")] + [
        ("live_filters", ctypes.c_uint32), ("pending_filters", ctypes.c_uint32)]


KERNEL_KINDS = ("insert_direct", "insert_evict", "contains", "remove",
                "slice_split", "slice_probe1", "slice_probe2", "slice_merge",
                "evict_map", "copy_h2d", "copy_d2h", "evict_level")


class CfKernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * len(KERNEL_KINDS)),
                ("ms", ctypes.c_double * len(KERNEL_KINDS))]


# Every symbol include/cf.h declares, with (restype, argtypes).
_vp, _u64, _u32, _int = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
_st = ctypes.c_int
_pcfg = ctypes.POINTER(CfConfig)
SIGNATURES = {
    "cf_table_bytes": (ctypes.c_size_t, [_u64, _u32, _u32]),
    "cf_required_bytes": (ctypes.c_size_t, [_pcfg]),
    "cf_snapshot_bytes": (ctypes.c_size_t, [_vp]),
    "cf_create": (_st, [_u64, _u32, _u32, _u32, ctypes.POINTER(_vp)]),
    "cf_create_ex": (_st, [_pcfg, ctypes.POINTER(_vp)]),
    "cf_create_at": (_st, [_vp, ctypes.c_size_t, _pcfg, ctypes.POINTER(_vp)]),
    "cf_destroy": (_st, [_vp]),
    "cf_get_config": (_st, [_vp, _pcfg]),
    "cf_table_ptr": (_vp, [_vp]),
    "cf_insert": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_insert_ex": (_st, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "cf_contains": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_remove": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_clear": (_st, [_vp, _vp]),
    "cf_insert_host": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_contains_host": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_remove_host": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_insert_host_async": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_contains_host_async": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_remove_host_async": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_set_staging_chunk": (_st, [_vp, _u64]),
    "cf_set_slicing": (_st, [_vp, _int, _u64, _u64]),
    "cf_set_eviction_map": (_st, [_vp, _int, _u64]),
    "cf_set_eviction_levels": (_st, [_vp, _int, ctypes.c_uint32, _u64, _u64]),
    "cf_set_host_reads": (_st, [_vp, _int]),
    "cf_debug_set_cas_limit": (_st, [_vp, _u32]),
    "cf_debug_bounds_checked": (_int, []),
    "cf_debug_touch_bucket": (_st, [_vp, _u64, ctypes.POINTER(_u64), _vp]),
    "cf_stats": (_st, [_vp, ctypes.POINTER(CfStats), _vp]),
    "cf_victims": (_st, [_vp, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp]),
    "cf_snapshot": (_st, [_vp, _vp, ctypes.c_size_t, _int, _vp]),
    "cf_load": (_st, [_vp, _vp, ctypes.c_size_t, _int, _vp]),
    "cf_count_occupied": (_st, [_vp, ctypes.POINTER(_u64), _vp]),
    "cf_hash_debug": (_st, [_vp, _u64, _u32, _u64, _u32, _vp, _vp, _vp, _vp]),
    "cf_debug_insert_serial": (_st, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "cf_insert_noalloc": (_st, [_vp, _vp, _u64, _vp, _vp]),
    "cf_server_create": (_st, [ctypes.POINTER(CfServerConfig), ctypes.POINTER(_vp)]),
    "cf_server_destroy": (_st, [_vp]),
    "cf_server_add_filter": (_st, [_vp, _pcfg, ctypes.POINTER(_u32)]),
    "cf_server_remove_filter": (_st, [_vp, _u32]),
    "cf_server_filter_state": (_st, [_vp, _u32, ctypes.POINTER(ctypes.c_int32)]),
    "cf_server_get_filter": (_vp, [_vp, _u32]),
    "cf_server_submit": (_st, [_vp, ctypes.POINTER(CfRequest), ctypes.POINTER(_u64)]),
    "cf_server_poll": (_u32, [_vp, ctypes.POINTER(CfCompletion), _u32]),
    "cf_server_drain": (_st, [_vp, _u32]),
    "cf_server_stats": (_st, [_vp, ctypes.POINTER(CfServerStats)]),
    "cf_server_run_trace": (_st, [_vp, ctypes.POINTER(CfRequest), ctypes.POINTER(ctypes.c_double),
                                  _u32, ctypes.POINTER(CfCompletion)]),
    "cf_plain_run_trace": (_st, [ctypes.POINTER(_vp), _u32, ctypes.POINTER(CfRequest),
                                 ctypes.POINTER(ctypes.c_double), _u32,
                                 ctypes.POINTER(CfCompletion), _vp]),
    "cf_batch_create": (_st, [_u32, _u64, ctypes.POINTER(_vp)]),
    "cf_batch_destroy": (_st, [_vp]),
    "cf_batch_set": (_st, [_vp, ctypes.POINTER(CfBatchItem), _u32]),
    "cf_batch_launch": (_st, [_vp, _vp]),
    "cf_batch_graph_launch": (_st, [_vp, _vp]),
    "cf_batch_autotune": (_st, [_vp, _vp, ctypes.POINTER(CfTuning)]),
    "cf_batch_set_variant": (_st, [_vp, _u32]),
    "cf_batch_get_tuning": (_st, [_vp, ctypes.POINTER(CfTuning)]),
    "cf_batch_variant_count": (_u32, [_vp]),
    "cf_set_kernel_timing": (_st, [_vp, _int]),
    "cf_read_kernel_times": (_st, [_vp, ctypes.POINTER(CfKernelTimes), _int]),
    "cf_probe_gather": (_st, [_vp, _u64, _u64, _u32, _u32, _u64, _vp, _vp]),
    "cf_set_l2_fetch_granularity": (_st, [_u32]),
    "cf_get_l2_fetch_granularity": (_st, [ctypes.POINTER(_u32)]),
    "cf_status_str": (ctypes.c_char_p, [_st]),
    "cf_last_error": (ctypes.c_char_p, []),
    "cf_version": (_int, []),
}

_lib = None


def load():
    """Load libcf.so once; raise if it is missing (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: the CUDA library has not been built "
            "(run paper_2603_15486_gb300/build.py). There is no CPU fallback.")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class CfError(RuntimeError):
    def __init__(self, status: int, what: str):
        L = load()
        msg = L.cf_status_str(status).decode()
        detail = (L.cf_last_error() or b"").decode()
        super().__init__(f"{what}: {msg} ({status}) {detail}".strip())
        self.status = status


def check(status: int, what: str):
    if status != 0:
        raise CfError(status, what)
