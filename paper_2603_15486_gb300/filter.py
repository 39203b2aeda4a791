"""Python binding of libcf: argument marshalling only.

Every operation is one call into the C ABI (include/cf.h); every step of the
insert / query / delete path runs in the library's CUDA kernels.  PyTorch
supplies device memory (tensors) and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (KERNEL_KINDS, CfBatchItem, CfCompletion, CfConfig, CfKernelTimes,
                   CfRequest, CfServerConfig, CfServerStats, CfStats, CfTuning, check)

POLICIES = {"xor": 0, "offset": 1}
EVICTIONS = {"bfs": 0, "dfs": 1}


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream or None
    return int(stream) or None


def _dev_keys(keys: torch.Tensor) -> torch.Tensor:
    if not isinstance(keys, torch.Tensor) or not keys.is_cuda:
        raise TypeError("keys must be a CUDA tensor (use *_host for host keys)")
    if keys.dtype not in (torch.int64, torch.uint64):
        raise TypeError(f"keys must be int64/uint64, got {keys.dtype}")
    if not keys.is_contiguous():
        raise ValueError("keys must be contiguous")
    return keys


def _dev_out(out, n: int, dtype, device) -> torch.Tensor:
    if out is None:
        return torch.empty(n, dtype=dtype, device=device)
    if not out.is_cuda or out.dtype != dtype or out.numel() < n or not out.is_contiguous():
        raise ValueError(f"output must be a contiguous CUDA {dtype} tensor of >= {n}")
    return out


def make_config(num_buckets: int, fp_bits: int = 16, slots_per_bucket: int = 4,
                max_evictions: int = 500, policy: str = "xor",
                eviction: str = "bfs", victim_capacity: int = 0) -> CfConfig:
    return CfConfig(int(num_buckets), int(fp_bits), int(slots_per_bucket),
                    int(max_evictions), POLICIES[policy], EVICTIONS[eviction],
                    int(victim_capacity))


def required_bytes(**kw) -> int:
    cfg = make_config(**kw)
    return int(_lib.load().cf_required_bytes(ctypes.byref(cfg)))


class CuckooFilter:
    """A cuckoo filter on the current CUDA device.

    ``memory``: optional caller-owned CUDA uint8 tensor of at least
    ``required_bytes(...)`` bytes (cf_create_at); otherwise the library
    allocates (cf_create_ex)."""

    def __init__(self, num_buckets: int, fp_bits: int = 16, slots_per_bucket: int = 4,
                 max_evictions: int = 500, policy: str = "xor", eviction: str = "bfs",
                 victim_capacity: int = 0, memory: Optional[torch.Tensor] = None):
        self._L = _lib.load()
        self.cfg = make_config(num_buckets, fp_bits, slots_per_bucket, max_evictions,
                               policy, eviction, victim_capacity)
        self.num_buckets, self.fp_bits, self.slots_per_bucket = (
            int(num_buckets), int(fp_bits), int(slots_per_bucket))
        self.max_evictions, self.policy, self.eviction = max_evictions, policy, eviction
        h = ctypes.c_void_p()
        self._memory = memory
        if memory is None:
            check(self._L.cf_create_ex(ctypes.byref(self.cfg), ctypes.byref(h)),
                  "cf_create_ex")
        else:
            if not memory.is_cuda or memory.dtype != torch.uint8:
                raise TypeError("memory must be a CUDA uint8 tensor")
            check(self._L.cf_create_at(memory.data_ptr(), memory.numel(),
                                       ctypes.byref(self.cfg), ctypes.byref(h)),
                  "cf_create_at")
        self._h = h
        self.device = torch.cuda.current_device()

    # ---- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.cf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    @property
    def table_bytes(self) -> int:
        return self.num_buckets * self.slots_per_bucket * self.fp_bits // 8

    @property
    def capacity(self) -> int:
        return self.num_buckets * self.slots_per_bucket

    # ---- hot path ------------------------------------------------------------
    def insert(self, keys: torch.Tensor, flags: Optional[torch.Tensor] = None,
               evictions: Optional[torch.Tensor] = None, stream=None,
               want_flags: bool = True) -> Optional[torch.Tensor]:
        keys = _dev_keys(keys)
        n = keys.numel()
        fl = _dev_out(flags, n, torch.uint8, keys.device) if (want_flags or flags is not None) else None
        ev = None
        if evictions is not None:
            ev = _dev_out(evictions, n, torch.int32, keys.device)
        check(self._L.cf_insert_ex(self._h, keys.data_ptr(), n,
                                   fl.data_ptr() if fl is not None else None,
                                   ev.data_ptr() if ev is not None else None,
                                   _stream_handle(stream)), "cf_insert")
        return fl

    def contains(self, keys: torch.Tensor, out: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
        keys = _dev_keys(keys)
        out = _dev_out(out, keys.numel(), torch.uint8, keys.device)
        check(self._L.cf_contains(self._h, keys.data_ptr(), keys.numel(),
                                  out.data_ptr(), _stream_handle(stream)), "cf_contains")
        return out

    def remove(self, keys: torch.Tensor, out: Optional[torch.Tensor] = None,
               stream=None, want_flags: bool = True) -> Optional[torch.Tensor]:
        keys = _dev_keys(keys)
        fl = _dev_out(out, keys.numel(), torch.uint8, keys.device) if (want_flags or out is not None) else None
        check(self._L.cf_remove(self._h, keys.data_ptr(), keys.numel(),
                                fl.data_ptr() if fl is not None else None,
                                _stream_handle(stream)), "cf_remove")
        return fl

    def insert_serial(self, keys: torch.Tensor, evictions: bool = True, stream=None):
        keys = _dev_keys(keys)
        n = keys.numel()
        fl = torch.empty(n, dtype=torch.uint8, device=keys.device)
        ev = torch.empty(n, dtype=torch.int32, device=keys.device) if evictions else None
        check(self._L.cf_debug_insert_serial(self._h, keys.data_ptr(), n, fl.data_ptr(),
                                             ev.data_ptr() if ev is not None else None,
                                             _stream_handle(stream)), "cf_debug_insert_serial")
        return fl, ev

    # ---- host-buffer forms (end to end) ---------------------------------------
    @staticmethod
    def _host(a, dtype) -> np.ndarray:
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                raise TypeError("host buffers expected")
            return a
        return np.ascontiguousarray(a, dtype=dtype)

    def _host_call(self, fn, keys, out, what, stream, need_out=True):
        k = self._host(keys, np.uint64)
        n = k.numel() if isinstance(k, torch.Tensor) else k.size
        if out is None and need_out:
            out = np.empty(n, np.uint8)
        kp = k.data_ptr() if isinstance(k, torch.Tensor) else k.ctypes.data
        op = None if out is None else (out.data_ptr() if isinstance(out, torch.Tensor)
                                       else out.ctypes.data)
        check(fn(self._h, kp, n, op, _stream_handle(stream)), what)
        return out

    def insert_host(self, keys, out=None, stream=None):
        return self._host_call(self._L.cf_insert_host, keys, out, "cf_insert_host", stream)

    def contains_host(self, keys, out=None, stream=None):
        return self._host_call(self._L.cf_contains_host, keys, out, "cf_contains_host", stream)

    def remove_host(self, keys, out=None, stream=None):
        return self._host_call(self._L.cf_remove_host, keys, out, "cf_remove_host", stream)

    def insert_host_async(self, keys, out=None, stream=None):
        """Asynchronous insert from host buffers: `out` (and `keys`) must stay
        alive until `stream` synchronises."""
        return self._host_call(self._L.cf_insert_host_async, keys, out,
                               "cf_insert_host_async", stream)

    def contains_host_async(self, keys, out=None, stream=None):
        return self._host_call(self._L.cf_contains_host_async, keys, out,
                               "cf_contains_host_async", stream)

    def remove_host_async(self, keys, out=None, stream=None):
        return self._host_call(self._L.cf_remove_host_async, keys, out,
                               "cf_remove_host_async", stream)

    def set_staging_chunk(self, keys_per_chunk: int):
        check(self._L.cf_set_staging_chunk(self._h, int(keys_per_chunk)), "cf_set_staging_chunk")

    def set_host_reads(self, mode: str = "staged"):
        """How sliced host-buffer calls get their keys (cf_set_host_reads):
        "staged" copies or "in_place" reads of pinned keys by the scatter."""
        check(self._L.cf_set_host_reads(self._h, {"staged": 0, "in_place": 1}[mode]),
              "cf_set_host_reads")

    def set_slicing(self, mode: str = "auto", slice_bytes: int = 0, max_chunk: int = 0):
        """Slice-partitioned execution (cf_set_slicing): mode "off", "auto"
        or "always"; slice_bytes / max_chunk 0 take the library defaults."""
        code = {"off": 0, "auto": 1, "always": 2}[mode]
        check(self._L.cf_set_slicing(self._h, code, int(slice_bytes), int(max_chunk)),
              "cf_set_slicing")

    # ---- state -----------------------------------------------------------------
    def set_eviction_map(self, mode: str = "auto", min_queue: int = 0):
        """Full-bucket map of the eviction loop: "off", "auto" or "always"
        (cf_set_eviction_map)."""
        modes = {"off": 0, "auto": 1, "always": 2}
        check(self._L.cf_set_eviction_map(self._h, modes[mode], int(min_queue)),
              "cf_set_eviction_map")

    def set_eviction_levels(self, mode: str = "on", n_levels: int = 0, min_queue: int = 0,
                            stop_queue: int = 0):
        """Slice-grouped eviction levels of the sliced insert
        (cf_set_eviction_levels): "off", "on" (device-buffer inserts into
        filters with buckets of at most 8 bytes; the default) or "always"
        (every sliced insert); 0 takes the library defaults."""
        code = {"off": 0, "on": 1, "always": 2}[mode]
        check(self._L.cf_set_eviction_levels(self._h, code, int(n_levels), int(min_queue),
                                             int(stop_queue)),
              "cf_set_eviction_levels")

    def set_cas_limit(self, limit: int = 0):
        """Test knob: bound of the CAS retry loops (0 = default 4096)."""
        check(self._L.cf_debug_set_cas_limit(self._h, int(limit)), "cf_debug_set_cas_limit")

    def clear(self, stream=None):
        check(self._L.cf_clear(self._h, _stream_handle(stream)), "cf_clear")

    def stats(self, stream=None) -> dict:
        st = CfStats()
        check(self._L.cf_stats(self._h, ctypes.byref(st), _stream_handle(stream)), "cf_stats")
        out = {}
        for n, _ in CfStats._fields_:
            v = getattr(st, n)
            out[n] = [int(x) for x in v] if n == "cas_retry" else int(v)
        return out

    def victims(self, stream=None):
        cnt = ctypes.c_uint64()
        check(self._L.cf_victims(self._h, None, None, 0, ctypes.byref(cnt),
                                 _stream_handle(stream)), "cf_victims")
        n = cnt.value
        tags = np.empty(n, np.uint32)
        buckets = np.empty(n, np.uint64)
        if n:
            check(self._L.cf_victims(self._h, tags.ctypes.data, buckets.ctypes.data, n,
                                     ctypes.byref(cnt), _stream_handle(stream)), "cf_victims")
        return tags, buckets

    def snapshot_bytes(self) -> int:
        return int(self._L.cf_snapshot_bytes(self._h))

    def snapshot(self, device: bool = False, stream=None):
        """64-byte header + raw table; numpy (host) or a CUDA uint8 tensor."""
        n = self.snapshot_bytes()
        if device:
            buf = torch.empty(n, dtype=torch.uint8, device="cuda")
            check(self._L.cf_snapshot(self._h, buf.data_ptr(), n, 1,
                                      _stream_handle(stream)), "cf_snapshot")
            return buf
        buf = np.empty(n, np.uint8)
        check(self._L.cf_snapshot(self._h, buf.ctypes.data, n, 0, _stream_handle(stream)),
              "cf_snapshot")
        return buf

    def load(self, snap, stream=None):
        if isinstance(snap, torch.Tensor) and snap.is_cuda:
            check(self._L.cf_load(self._h, snap.data_ptr(), snap.numel(), 1,
                                  _stream_handle(stream)), "cf_load")
        else:
            buf = np.ascontiguousarray(snap, dtype=np.uint8)
            check(self._L.cf_load(self._h, buf.ctypes.data, buf.size, 0,
                                  _stream_handle(stream)), "cf_load")

    def count_occupied(self, stream=None) -> int:
        v = ctypes.c_uint64()
        check(self._L.cf_count_occupied(self._h, ctypes.byref(v), _stream_handle(stream)),
              "cf_count_occupied")
        return v.value

    def set_kernel_timing(self, enable: bool = True):
        check(self._L.cf_set_kernel_timing(self._h, int(bool(enable))), "cf_set_kernel_timing")

    def kernel_times(self, reset: bool = True) -> dict:
        """{kernel: (launches, total ms)} measured with CUDA events on the
        launching streams while timing was enabled."""
        t = CfKernelTimes()
        check(self._L.cf_read_kernel_times(self._h, ctypes.byref(t), int(bool(reset))),
              "cf_read_kernel_times")
        return {k: (int(t.launches[i]), float(t.ms[i])) for i, k in enumerate(KERNEL_KINDS)}

    def table_view(self) -> torch.Tensor:
        """The live device table as a uint8 tensor (no copy; do not write)."""
        ptr = self._L.cf_table_ptr(self._h)
        return _device_bytes(ptr, self.table_bytes, self)


class _Owner:
    pass


def _device_bytes(ptr: int, nbytes: int, owner) -> torch.Tensor:
    """Wrap a raw device pointer as a CUDA uint8 tensor (kept alive by owner)."""
    class _CAI:
        def __init__(self):
            self.__cuda_array_interface__ = {
                "shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                "version": 3, "strides": None}
    t = torch.as_tensor(_CAI(), device="cuda")
    t._cf_owner = owner  # noqa: SLF001
    return t


def hash_debug(keys: torch.Tensor, fp_bits: int, num_buckets: int, policy: str = "xor",
               stream=None):
    L = _lib.load()
    keys = _dev_keys(keys)
    n = keys.numel()
    fp = torch.empty(n, dtype=torch.int32, device=keys.device)
    i1 = torch.empty(n, dtype=torch.int64, device=keys.device)
    i2 = torch.empty(n, dtype=torch.int64, device=keys.device)
    check(L.cf_hash_debug(keys.data_ptr(), n, fp_bits, num_buckets, POLICIES[policy],
                          fp.data_ptr(), i1.data_ptr(), i2.data_ptr(),
                          _stream_handle(stream)), "cf_hash_debug")
    return fp, i1, i2


OPS = {"insert": 0, "contains": 1, "remove": 2}


class Batch:
    """A multi-filter launch plan (cf_batch_*): many filters' insert /
    query / delete batches in one persistent kernel (+ one eviction
    kernel), optionally as a replayed CUDA graph, with an autotuner."""

    def __init__(self, max_items: int, max_keys: int):
        self._L = _lib.load()
        h = ctypes.c_void_p()
        check(self._L.cf_batch_create(int(max_items), int(max_keys), ctypes.byref(h)),
              "cf_batch_create")
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.cf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, items):
        """items: iterable of (CuckooFilter, op, keys, flags) with op in
        {"insert", "contains", "remove"}; keys/flags CUDA tensors (flags may
        be None except for "contains")."""
        items = list(items)
        arr = (CfBatchItem * max(1, len(items)))()
        keep = []
        for i, (filt, op, keys, flags) in enumerate(items):
            keys = _dev_keys(keys)
            arr[i].filter = filt.handle
            arr[i].keys = keys.data_ptr()
            arr[i].n = keys.numel()
            arr[i].out_flags = flags.data_ptr() if flags is not None else None
            arr[i].op = OPS[op]
            keep += [filt, keys, flags]
        check(self._L.cf_batch_set(self._h, arr, len(items)), "cf_batch_set")
        self._keep = keep

    def launch(self, stream=None, graph: bool = False):
        fn = self._L.cf_batch_graph_launch if graph else self._L.cf_batch_launch
        check(fn(self._h, _stream_handle(stream)), "cf_batch_launch")

    def autotune(self, stream=None) -> dict:
        t = CfTuning()
        check(self._L.cf_batch_autotune(self._h, _stream_handle(stream), ctypes.byref(t)),
              "cf_batch_autotune")
        return {n: getattr(t, n) for n, _ in CfTuning._fields_}

    def set_variant(self, v: int):
        check(self._L.cf_batch_set_variant(self._h, int(v)), "cf_batch_set_variant")

    def tuning(self) -> dict:
        t = CfTuning()
        check(self._L.cf_batch_get_tuning(self._h, ctypes.byref(t)), "cf_batch_get_tuning")
        return {n: getattr(t, n) for n, _ in CfTuning._fields_}

    def variant_count(self) -> int:
        return int(self._L.cf_batch_variant_count(self._h))


FILTER_STATES = {0: "pending", 1: "live", 2: "closing", 3: "closed"}


def _completions_to_dict(arr, n):
    out = np.empty(n, dtype=[("request_id", "u8"), ("tag", "u8"), ("status", "i4"),
                             ("wave_size", "u4"), ("submit_s", "f8"), ("launch_s", "f8"),
                             ("done_s", "f8")])
    for i in range(n):
        c = arr[i]
        out[i] = (c.request_id, c.tag, c.status, c.wave_size, c.submit_s, c.launch_s, c.done_s)
    return out


def _requests(reqs):
    """reqs: list of (filter_id, op, keys_tensor, flags_tensor_or_None, tag)."""
    arr = (CfRequest * max(1, len(reqs)))()
    keep = []
    for i, (fid, op, keys, flags, tag) in enumerate(reqs):
        keys = _dev_keys(keys)
        arr[i] = CfRequest(int(fid), OPS[op], keys.data_ptr(), keys.numel(),
                           flags.data_ptr() if flags is not None else None, int(tag))
        keep += [keys, flags]
    return arr, keep


class Server:
    """Serving loop with continuous batching (cf_server_*): filters live on
    the device, requests are batched into waves of multi-filter launches,
    several waves in flight, filters admitted against an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 4,
                 max_wave_items: int = 256, max_wave_keys: int = 1 << 22,
                 use_graphs: bool = True, watchdog_us: int = 0):
        self._L = _lib.load()
        cfg = CfServerConfig(int(hbm_budget_bytes), int(max_inflight), int(max_wave_items),
                             int(max_wave_keys), int(bool(use_graphs)), int(watchdog_us))
        h = ctypes.c_void_p()
        check(self._L.cf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cf_server_create")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.cf_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_filter(self, num_buckets: int, fp_bits: int = 16, slots_per_bucket: int = 4,
                   max_evictions: int = 500, policy: str = "xor", eviction: str = "bfs") -> int:
        cfg = make_config(num_buckets, fp_bits, slots_per_bucket, max_evictions, policy, eviction)
        fid = ctypes.c_uint32()
        check(self._L.cf_server_add_filter(self._h, ctypes.byref(cfg), ctypes.byref(fid)),
              "cf_server_add_filter")
        return fid.value

    def remove_filter(self, fid: int):
        check(self._L.cf_server_remove_filter(self._h, int(fid)), "cf_server_remove_filter")

    def filter_state(self, fid: int) -> str:
        st = ctypes.c_int32()
        check(self._L.cf_server_filter_state(self._h, int(fid), ctypes.byref(st)),
              "cf_server_filter_state")
        return FILTER_STATES[st.value]

    def filter_handle(self, fid: int) -> Optional[int]:
        return self._L.cf_server_get_filter(self._h, int(fid))

    def submit(self, fid: int, op: str, keys: torch.Tensor, flags=None, tag: int = 0) -> int:
        keys = _dev_keys(keys)
        r = CfRequest(int(fid), OPS[op], keys.data_ptr(), keys.numel(),
                      flags.data_ptr() if flags is not None else None, int(tag))
        rid = ctypes.c_uint64()
        check(self._L.cf_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)),
              "cf_server_submit")
        self._keep[rid.value] = (keys, flags)
        return rid.value

    def poll(self, max_n: int = 4096):
        arr = (CfCompletion * max_n)()
        n = self._L.cf_server_poll(self._h, arr, max_n)
        out = _completions_to_dict(arr, n)
        for rid in out["request_id"]:
            self._keep.pop(int(rid), None)
        return out

    def drain(self, timeout_ms: int = 600000) -> int:
        """0 when everything submitted has completed, else the status
        (4 = CF_ETIMEOUT)."""
        return int(self._L.cf_server_drain(self._h, int(timeout_ms)))

    def stats(self) -> dict:
        st = CfServerStats()
        check(self._L.cf_server_stats(self._h, ctypes.byref(st)), "cf_server_stats")
        return {n: int(getattr(st, n)) for n, _ in CfServerStats._fields_}

    def run_trace(self, reqs, arrival_s):
        """Replay (filter_id, op, keys, flags, tag) requests at the given
        arrival times (seconds from the start); returns the completions by
        request index."""
        arr, keep = _requests(reqs)
        n = len(reqs)
        arrivals = (ctypes.c_double * max(1, n))(*[float(a) for a in arrival_s])
        out = (CfCompletion * max(1, n))()
        check(self._L.cf_server_run_trace(self._h, arr, arrivals, n, out), "cf_server_run_trace")
        return _completions_to_dict(out, n)


def plain_run_trace(filters, reqs, arrival_s, stream=None):
    """The baseline: each request alone, in arrival order, one synchronised
    cf_insert / cf_contains / cf_remove at a time.  filters[i] serves
    filter_id i."""
    L = _lib.load()
    arr, keep = _requests(reqs)
    n = len(reqs)
    fl = (ctypes.c_void_p * max(1, len(filters)))(*[f.handle if f is not None else None
                                                    for f in filters])
    arrivals = (ctypes.c_double * max(1, n))(*[float(a) for a in arrival_s])
    out = (CfCompletion * max(1, n))()
    check(L.cf_plain_run_trace(fl, len(filters), arr, arrivals, n, out,
                               _stream_handle(stream)), "cf_plain_run_trace")
    return _completions_to_dict(out, n)
