#!/usr/bin/env python3
"""Benchmark: insert / query / delete Mops/s of one large cuckoo filter.

Workload (one "step" = one pass of the whole hot path):
  a filter of 2^28 buckets x 4 slots x 16-bit fingerprints (2 GiB table,
  max 500 evictions), cleared, then filled with uniform splitmix64 keys
  (seed 2) through load factors 0.5 -> 0.8 -> 0.95 (1,020,054,732 inserts in
  three calls), then 2^30 queries at a 50% positive mix, then the first 2^28
  inserted keys deleted.  Keys are generated on the device before timing.

Output: ONE JSON line (rank 0).  ``value`` = total ops of all ranks / the
slowest rank's device time (CUDA events on the launching stream).  The
table (2 GiB) and key arrays (8 GB) exceed L2 (129 MB), so no flush is
needed between steps.  ``roofline`` relates the dominant phase to the
measured HBM copy bandwidth, ``cpu_baseline`` times the CPU oracle on a
scale model of the same workload, ``e2e`` repeats the measurement through
the host-buffer C-ABI calls with the H2D/D2H copies inside the timed region.

``--impl reference`` times the CPU oracle (the reference implementation of
the method) on the host cores instead, one bounded sample per step.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "insert/query/delete Mops/s at LF 0.95 vs HBM roofline; served p99 vs plain"
# Eviction levels per insert pass when --levels is 0 (the library default).
DEFAULT_LEVELS = 12

# DRAM bytes (read + write) per launch of the dominant kernel come from the
# committed ncu summary of the large workload, which records them with a
# hash of the kernel sources they were measured on; they are reported only
# while the sources still have that hash (else the roofline's traffic is
# null until the capture is taken again).
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "dram_large_2^28x4_f16_lf0.95.md")
KERNEL_SOURCES = ("cf_types.h", "cf_device.cuh", "cf_kernels.cuh", "cf_slice.cuh",
                  "cf_levels.cuh", "cf_launch.cuh", "cf_inst_f16.cu")


def kernel_sources_sha() -> str:
    """First 16 hex digits of the SHA-256 of the sources the single-filter
    kernels are compiled from."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_15486_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None if the summary has no figure for it or was taken on other kernel
    sources.  The summary holds lines of the form
    `traffic <kernel> <bytes per launch> sources <sha16>`."""
    import re
    try:
        text = open(TRAFFIC_PROFILE).read()
    except OSError:
        return None
    sha = kernel_sources_sha()
    for m in re.finditer(r"^traffic (\w+) ([0-9.e+]+) sources ([0-9a-f]{16})\s*$", text, re.M):
        if m.group(1) == kernel and m.group(3) == sha:
            return float(m.group(2))
    return None


SECTOR = 32


# ---------------------------------------------------------------------------
# Multi-rank harness (also exercised on CPU with gloo by the tests).
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_sum(t_local: float, ops_local: float, group=None):
    """Max of the elapsed time and sum of the ops over all ranks."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return t_local, ops_local
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    o = torch.tensor([ops_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(o, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(o.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)
        except Exception:
            self.proc = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[1]), float(parts[2]), parts[4:8]))
            except Exception:
                continue
        inside = [r for r in rows if self.t0 is None or (self.t0 - 0.2 <= r[0] <= self.t1 + 0.2)]
        use = inside or rows
        if not use:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in use),
                "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use)}


# ---------------------------------------------------------------------------
# The CPU oracle on a scale model: baseline timing + bucket-touch counts.
# ---------------------------------------------------------------------------
def oracle_run(W, repeat: int = 1):
    """Run the workload W on the CPU oracle (one thread).  Returns
    (seconds, ops, stats-per-phase) of the LAST repeat."""
    import oracle
    import workloads

    keys = workloads.keys(W.key_seed, W.n_insert)
    q = workloads.query_mix(W.n_queries, keys, W.query_pos_seed, W.key_seed, W.n_insert)
    dels = keys[: W.n_deletes]
    res = None
    for _ in range(repeat):
        o = oracle.OracleFilter(W.m, W.f, W.b, W.max_evictions)
        t0 = time.perf_counter()
        for lo, hi in W.insert_segments():
            o.insert_batch(keys[lo:hi])
        s_ins = o.stats()
        t1 = time.perf_counter()
        o.contains_batch(q)
        t2 = time.perf_counter()
        o.remove_batch(dels)
        t3 = time.perf_counter()
        s = o.stats()
        res = (t3 - t0, W.ops_per_step(),
               {"insert": {"ops": W.n_insert, "s": t1 - t0,
                           "bucket_reads": s_ins["ins_bucket_reads"],
                           "bucket_writes": s_ins["ins_bucket_writes"],
                           "direct_reads": s_ins["ins_direct_reads"],
                           "direct_writes": s_ins["ins_direct_writes"],
                           "evict_keys": s_ins["ins_evict_keys"]},
                "query": {"ops": W.n_queries, "s": t2 - t1,
                          "bucket_reads": s["qry_bucket_reads"], "bucket_writes": 0},
                "delete": {"ops": W.n_deletes, "s": t3 - t2,
                           "bucket_reads": s["rem_bucket_reads"],
                           "bucket_writes": s["rem_bucket_writes"]}})
        o.close()
    return res


def kernel_bytes(phases: dict, bucket_bytes: int, n_insert: int, n_query: int,
                 n_delete: int) -> dict:
    """Algorithmic bytes per step of each kernel, from the oracle's bucket
    counts (per operation) scaled to the workload's operation counts:
    32-byte sectors of the buckets it reads and writes, plus 8 B of key and
    1 B of flag per key it handles.  Insert phase 1 handles every key; phase
    2 handles the keys whose two buckets were full (it re-reads the key)."""
    spb = max(1, math.ceil(bucket_bytes / SECTOR)) * SECTOR
    ins = phases["insert"]
    per = ins["ops"]
    d_touch = (ins["direct_reads"] + ins["direct_writes"]) / per
    e_touch = (ins["bucket_reads"] + ins["bucket_writes"] - ins["direct_reads"]
               - ins["direct_writes"]) / per
    e_keys = ins["evict_keys"] / per
    q = phases["query"]
    d = phases["delete"]
    return {"insert_direct": n_insert * (d_touch * spb + 9),
            "insert_evict": n_insert * (e_touch * spb + 9 * e_keys),
            "evict_map": 0.0,  # set by the caller from the builds per step
            "contains": n_query * (q["bucket_reads"] / q["ops"] * spb + 9),
            "remove": n_delete * ((d["bucket_reads"] + d["bucket_writes"]) / d["ops"] * spb + 9)}


def merge_eviction_times(ktimes: dict, kb: dict, steps: int):
    """The eviction (Alg. 1 phase 2) of a sliced insert runs as the slice-
    grouped levels and the loop for what they leave: one entry "eviction"
    (the levels' timer records as its launches, the two kinds' time, the
    eviction's algorithmic bytes) and its split per step.  Without level
    records the times stay as they are (None for the split)."""
    ktimes = dict(ktimes)
    lv = ktimes.pop("evict_level", (0, 0.0))
    if not lv[0]:
        return ktimes, None
    _, ms_loop = ktimes.pop("insert_evict", (0, 0.0))
    ktimes["eviction"] = (lv[0], ms_loop + lv[1])
    kb["eviction"] = kb["insert_evict"]
    return ktimes, {"levels_ms_per_step": round(lv[1] / steps, 3),
                    "loop_and_rest_ms_per_step": round(ms_loop / steps, 3)}


def slice_kernel_bytes(phases: dict, W, chunk: int) -> dict:
    """Bytes the slice-partitioned passes must move per step (their streams,
    plus one sweep of the table per bucket pass: read, and written back for
    insert / delete), from the workload's operation counts and the oracle's
    fraction of keys that need their second bucket."""
    tb = W.table_bytes
    calls = {"insert": [hi - lo for lo, hi in W.insert_segments()],
             "query": [W.n_queries], "delete": [W.n_deletes]}
    ins, q, d = phases["insert"], phases["query"], phases["delete"]
    pend = {"insert": ins["direct_reads"] / ins["ops"] - 1.0,
            "query": q["bucket_reads"] / q["ops"] - 1.0,
            "delete": d["bucket_reads"] / d["ops"] - 1.0}
    out = {"slice_split": 0.0, "slice_probe1": 0.0, "slice_probe2": 0.0, "slice_merge": 0.0}
    for op, sizes in calls.items():
        n = sum(sizes)
        passes = sum(math.ceil(x / chunk) for x in sizes)
        sweep = tb * (1 if op == "query" else 2) * passes
        pf = max(0.0, pend[op])
        out["slice_split"] += n * (8 + 8 + 4)  # key read, rec1 write, dst write
        out["slice_probe1"] += n * (8 + 4 + pf * 8) + sweep  # rec1, link, rec2
        out["slice_probe2"] += n * pf * (8 + 1) + sweep         # rec2, f2
        # merge: link, f2 of pending records, f1; out: dst, f1, flag
        out["slice_merge"] += n * (4 + pf * 1 + 1 + 4 + 1 + 1)
    return out


def bytes_per_op(phases: dict, bucket_bytes: int) -> dict:
    """Algorithmic bytes per operation: the 32-byte sectors of the buckets
    the algorithm reads and writes (counted by the oracle), plus the 8-byte
    key read and the 1-byte flag write."""
    sectors_per_bucket = max(1, math.ceil(bucket_bytes / SECTOR))
    out = {}
    for name, p in phases.items():
        touches = (p["bucket_reads"] + p["bucket_writes"]) / p["ops"]
        out[name] = touches * sectors_per_bucket * SECTOR + 8 + 1
    return out


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------
def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads
    from paper_2603_15486_gb300 import CuckooFilter

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = workloads.BY_NAME[args.workload]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream

    # ---- inputs, generated on the device (untimed) ----
    keys = torch.empty(W.n_insert, dtype=torch.int64, device=dev)
    workloads.keys_dev(keys.data_ptr(), W.n_insert, W.key_seed, 0, sh)
    queries = torch.empty(W.n_queries, dtype=torch.int64, device=dev)
    workloads.query_mix_dev(queries.data_ptr(), W.n_queries, keys.data_ptr(), W.n_insert,
                            W.query_pos_seed, W.key_seed, W.n_insert, sh)
    dels = keys[: W.n_deletes]
    ins_flags = torch.empty(W.n_insert, dtype=torch.uint8, device=dev)
    q_flags = torch.empty(W.n_queries, dtype=torch.uint8, device=dev)
    d_flags = torch.empty(W.n_deletes, dtype=torch.uint8, device=dev)
    filt = CuckooFilter(W.m, W.f, W.b, W.max_evictions)
    filt.set_slicing(args.slicing, args.slice_bytes, args.slice_chunk)
    filt.set_eviction_map(args.evict_map)
    filt.set_eviction_levels(args.evict_levels, args.levels, 0, args.level_stop)
    stream.synchronize()

    segs = W.insert_segments()

    def step(ev=None):
        filt.clear(stream=stream)
        if ev is not None:
            ev[0].record(stream)
        for lo, hi in segs:
            filt.insert(keys[lo:hi], flags=ins_flags[lo:hi], stream=stream)
        if ev is not None:
            ev[1].record(stream)
        filt.contains(queries, out=q_flags, stream=stream)
        if ev is not None:
            ev[2].record(stream)
        filt.remove(dels, out=d_flags, stream=stream)
        if ev is not None:
            ev[3].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    st = filt.stats()

    filt.set_kernel_timing(True)
    filt.kernel_times(reset=True)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_start()
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_end()
    barrier()
    clocks = sampler.stop() if sampler else None

    elapsed = t_start.elapsed_time(t_end) / 1e3
    ktimes = filt.kernel_times(reset=True)
    filt.set_kernel_timing(False)
    ops_local = float(W.ops_per_step()) * args.steps
    t_max, ops_all = reduce_max_sum(elapsed, ops_local)
    ph = {"insert": [], "query": [], "delete": []}
    for e in evs:
        ph["insert"].append(e[0].elapsed_time(e[1]) / 1e3)
        ph["query"].append(e[1].elapsed_time(e[2]) / 1e3)
        ph["delete"].append(e[2].elapsed_time(e[3]) / 1e3)
    med = {k: statistics.median(v) for k, v in ph.items()}
    st_end = filt.stats()

    # ---- correctness guard of the timed run (cheap, device-side) ----
    ins_ok = int(ins_flags.sum())
    q_pos = int(q_flags[0::2].sum())
    q_neg = int(q_flags[1::2].sum())

    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(filt, keys, queries, W, args, stream)

    if rank != 0:
        return None

    value = ops_all / t_max / 1e6
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mops/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u16", "data": "synthetic",
        "config": {"workload": W.name, "buckets": W.m, "slots_per_bucket": W.b,
                   "fp_bits": W.f, "max_evictions": W.max_evictions,
                   "load_factors": list(W.alphas), "inserts": W.n_insert,
                   "queries": W.n_queries, "query_positive_fraction": 0.5,
                   "deletes": W.n_deletes, "table_bytes": W.table_bytes,
                   "keys": "splitmix64 seed 2, uniform uint64",
                   "parallelism": f"replicas x{ws}",
                   "slicing": args.slicing, "slice_chunk": args.slice_chunk or (1 << 28),
                   "evict_map": args.evict_map,
                   "evict_levels": args.evict_levels,
                   "slice_bytes": args.slice_bytes or (32 << 20),
                   "l2": "no flush: 2 GiB table and 8 GB key arrays exceed the 129 MB L2"},
        "phases": {k: {"ms": round(v * 1e3, 3),
                       "mops": round(n / v / 1e6, 1)}
                   for k, v, n in (("insert", med["insert"], W.n_insert),
                                   ("query", med["query"], W.n_queries),
                                   ("delete", med["delete"], W.n_deletes))},
        # Kernels launched in the timed steps, from the per-kernel timer (one
        # timer record covers merge + out).
        # The levels' record covers the seed and the levels.
        "gpu_launches": sum(n_l * {"slice_merge": 2,
                                   "evict_level": (args.levels or DEFAULT_LEVELS) + 1}.get(k, 1)
                            for k, (n_l, _) in ktimes.items()),
        "checks": {"insert_ok": ins_ok, "insert_fail": W.n_insert - ins_ok,
                   "query_pos_found": q_pos, "query_pos": W.n_queries // 2,
                   "false_positives": q_neg, "fpr": q_neg / (W.n_queries // 2),
                   "occupancy_after_step": st_end["occupancy"],
                   "evictions_per_step": st["evictions"],
                   "contention": st_end["contention"],
                   "eviction_levels_per_step": st_end["level_passes"],
                   "level_steps_per_step": st_end["level_steps"],
                   "level_runout_per_step": st_end["level_runout"],
                   "cas_retry_per_step": st_end["cas_retry"]},
        "clocks": clocks,
    }

    # ---- roofline of the dominant kernel + CPU baseline (rank 0, N=1 only) ----
    peaks = load_peaks()
    cpu = None
    S = workloads.BY_NAME[args.cpu_workload if (ws == 1 and not args.no_cpu)
                          else "ref_2^20x4_f16_lf0.95"]
    secs, ops, phases = oracle_run(S)
    if ws == 1 and not args.no_cpu:
        cpu = {"value": round(ops / secs / 1e6, 3), "unit": "Mops/s", "cores": 1,
               "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"{S.name}: the same load-factor path, 50/50 query mix and "
                          f"delete fraction on {S.m} buckets ({ops} ops, {secs:.1f} s, "
                          "one thread of the host)"),
               "phases_mops": {k: round(p["ops"] / p["s"] / 1e6, 3) for k, p in phases.items()}}
    kb = kernel_bytes(phases, W.f * W.b // 8, W.n_insert, W.n_queries, W.n_deletes)
    kb.update(slice_kernel_bytes(phases, W, args.slice_chunk or (1 << 28)))
    # The full-bucket map: each build reads the table and writes m/8 bytes
    # (the counters restart with every step's clear, so st_end holds one
    # step's builds).
    kb["evict_map"] = st_end["map_builds"] * (W.table_bytes + (W.m + 31) // 32 * 4)
    ktimes, evict_parts = merge_eviction_times(ktimes, kb, args.steps)
    peak = peaks.get("hbm_gbs") or 6800.0
    kern = {}
    for k, (launches, ms) in ktimes.items():
        if not launches:
            continue
        ach = kb[k] * args.steps / (ms / 1e3) / 1e9
        kern[k] = {"launches": launches, "avg_launch_ms": round(ms / launches, 4),
                   "total_ms_per_step": round(ms / args.steps, 3),
                   ("stream_bytes_per_step" if k.startswith("slice") or k == "evict_map"
                    else "algorithmic_bytes_per_step"): int(kb[k]),
                   "achieved_GBps": round(ach, 1), "frac": round(ach / peak, 4)}
        if k == "eviction" and evict_parts:
            kern[k].update(evict_parts)
    # Per operation: the method's algorithmic bytes (32 B per bucket sector
    # the oracle touches + 9 B) at the measured operation rate.
    bpo = bytes_per_op(phases, W.f * W.b // 8)
    for name, key in (("insert", "insert"), ("query", "query"), ("delete", "delete")):
        ph = out["phases"][name]
        gbps = ph["mops"] * 1e6 * bpo[key] / 1e9
        ph.update({"algorithmic_bytes_per_op": round(bpo[key], 1),
                   "achieved_GBps": round(gbps, 1), "frac": round(gbps / peak, 4)})
    dom = max(kern, key=lambda k: kern[k]["total_ms_per_step"])
    ev = "eviction" if "eviction" in kern else "insert_evict" if "insert_evict" in kern else None
    ceiling = random_gather_ceiling(stream)
    out["roofline"] = {"bound": "hbm", "kernel": dom,
                       "achieved": kern[dom]["achieved_GBps"], "peak": peak, "unit": "GB/s",
                       "frac": kern[dom]["frac"],
                       "traffic": (args.traffic if args.traffic is not None
                                   else ncu_traffic(dom)
                                   if (W.name, args.slicing) == ("large_2^28x4_f16_lf0.95", "auto")
                                   else None),
                       "traffic_source": ("--traffic" if args.traffic is not None else
                                          "profiles/dram_large_2^28x4_f16_lf0.95.md, kernel "
                                          "sources " + kernel_sources_sha()),
                       "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"
                       if peaks.get("hbm_gbs") else "fallback 6.8 TB/s",
                       "random_sector_ceiling_GBps": ceiling["GBps_32B"],
                       # The eviction is the kernel bound by random sectors;
                       # its algorithmic rate against that ceiling.
                       "eviction_frac_of_random_sector_ceiling": round(
                           kern[ev]["achieved_GBps"] / ceiling["GBps_32B"], 3)
                       if ev else None,
                       "kernels": kern,
                       "bytes_per_op_model": "32 B x (distinct buckets read + written, "
                                             "counted by the oracle on " + S.name + ") + 9 B"}
    out["random_gather"] = ceiling
    out["cpu_baseline"] = cpu
    out["e2e"] = e2e
    # The other half of the metric: served vs plain per-request calls, and
    # many filters in one batched launch vs a loop of per-filter launches
    # (bounded runs; outside the timed region of the headline).
    if ws == 1 and not args.no_extras:
        del keys, queries, ins_flags, q_flags, d_flags
        filt.close()
        torch.cuda.empty_cache()
        out["served_vs_plain"] = serve_summary(args.extras_requests)
        out["batched_vs_loop"] = batched_summary()
    return out


def random_gather_ceiling(stream, n_access: int = 1 << 28):
    """Random 8-byte loads over a 2 GiB buffer with the query kernel's load
    instruction (cf_probe_gather): the rate HBM serves independent random
    sectors, the real ceiling of every probe of the filter."""
    import torch
    from paper_2603_15486_gb300 import _lib
    L = _lib.load()
    buf = torch.zeros(1 << 31, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    sh = stream.cuda_stream
    for _ in range(2):
        L.cf_probe_gather(buf.data_ptr(), buf.numel(), n_access, 8, 8, 3, sink.data_ptr(), sh)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc = L.cf_probe_gather(buf.data_ptr(), buf.numel(), n_access, 8, 8, 5, sink.data_ptr(), sh)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    del buf
    g = n_access / ms / 1e6
    return {"gloads_per_s": round(g, 2), "GBps_32B": round(g * 32, 1), "rc": rc,
            "what": "2^28 random 8-byte loads over 2 GiB, 8 in flight per thread"}


def e2e_run(filt, keys, queries, W, args, stream):
    """The same step through the host-buffer C-ABI calls: keys start in
    pinned host memory, flags end there; copies are inside the timing."""
    import numpy as np
    import torch

    try:
        hk = torch.empty(W.n_insert, dtype=torch.int64, pin_memory=True)
        hq = torch.empty(W.n_queries, dtype=torch.int64, pin_memory=True)
        hf_i = torch.empty(W.n_insert, dtype=torch.uint8, pin_memory=True)
        hf_q = torch.empty(W.n_queries, dtype=torch.uint8, pin_memory=True)
        hf_d = torch.empty(W.n_deletes, dtype=torch.uint8, pin_memory=True)
        pinned = True
    except RuntimeError:
        hk = torch.empty(W.n_insert, dtype=torch.int64)
        hq = torch.empty(W.n_queries, dtype=torch.int64)
        hf_i = torch.empty(W.n_insert, dtype=torch.uint8)
        hf_q = torch.empty(W.n_queries, dtype=torch.uint8)
        hf_d = torch.empty(W.n_deletes, dtype=torch.uint8)
        pinned = False
    hk.copy_(keys)
    hq.copy_(queries)
    segs = W.insert_segments()
    filt.set_staging_chunk(args.e2e_chunk)
    filt.set_host_reads(args.e2e_reads)
    # The host-to-device link's copy rate, measured outside the timed
    # region (four back-to-back copies of up to 1 GiB of the pinned keys),
    # for reading E beside it.
    nb = min(hk.numel(), 1 << 27)
    dev = torch.empty(nb, dtype=torch.int64, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        dev.copy_(hk[:nb], non_blocking=True)
        e0.record(stream)
        for _ in range(4):
            dev.copy_(hk[:nb], non_blocking=True)
        e1.record(stream)
    stream.synchronize()
    link_gbps = 4 * 8 * nb / (e0.elapsed_time(e1) / 1e3) / 1e9
    del dev

    def step():
        # The asynchronous host-buffer calls, back to back; the stream's
        # synchronisation at the end of the timed region waits for the last
        # flags to land in host memory.
        filt.clear(stream=stream)
        for lo, hi in segs:
            filt.insert_host_async(hk[lo:hi], out=hf_i[lo:hi], stream=stream)
        filt.contains_host_async(hq, out=hf_q, stream=stream)
        filt.remove_host_async(hk[: W.n_deletes], out=hf_d, stream=stream)

    for _ in range(max(1, args.e2e_warmup)):
        step()
    stream.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step()
    stream.synchronize()
    el = time.perf_counter() - t0
    t_max, ops_all = reduce_max_sum(el, float(W.ops_per_step()) * args.e2e_steps)
    h2d = 8 * (W.n_insert + W.n_queries + W.n_deletes)
    d2h = W.n_insert + W.n_queries + W.n_deletes
    return {"value": round(ops_all / t_max / 1e6, 2), "unit": "Mops/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": args.e2e_steps, "pinned": pinned,
            "ms_per_step": round(el / args.e2e_steps * 1e3, 3),
            "staging_chunk": args.e2e_chunk,
            "host_reads": args.e2e_reads,
            "h2d_link_GBps": round(link_gbps, 1),
            "api": "cf_insert_host_async / cf_contains_host_async / cf_remove_host_async "
                   "(pinned host keys in, host flags out; one stream synchronisation after "
                   "the timed steps)",
            "checks": {"insert_ok": int(hf_i.sum()), "query_pos_found": int(hf_q[0::2].sum()),
                       "remove_ok": int(hf_d.sum())}}


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle.
# ---------------------------------------------------------------------------
def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import workloads
    S = workloads.BY_NAME[args.ref_workload]
    for _ in range(args.warmup):
        oracle_run(S)
    times = []
    for _ in range(args.steps):
        secs, ops, _ = oracle_run(S)
        times.append(secs)
    tot = sum(times)
    value = S.ops_per_step() * args.steps / tot / 1e6
    return {"metric": METRIC, "value": round(value, 3), "unit": "Mops/s", "impl": "reference",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16", "data": "synthetic",
            "config": {"workload": args.workload, "sample": S.name},
            "cpu_baseline": {"value": round(value, 3), "unit": "Mops/s", "cores": 1,
                             "host_cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"each step: {S.name} ({S.ops_per_step()} ops: "
                                        "fill to LF 0.95, 50/50 queries, deletes), one thread")},
            "e2e": {"value": round(value, 3), "unit": "Mops/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# Many-filters mode: plain per-filter calls vs one batched launch per phase.
# ---------------------------------------------------------------------------
def batched_compare(steps: int, warmup: int) -> dict:
    """Many filters: one graph-replayed batched launch per operation against
    a loop of per-filter calls, on the 512-filter workload (median of
    `steps` timed repetitions after `warmup`)."""
    import torch

    import workloads
    from paper_2603_15486_gb300 import Batch, CuckooFilter

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    layout = workloads.multi_filter_layout()
    total = sum(n for _, n in layout)
    filters = [CuckooFilter(m, 16, 4, 500) for m, _ in layout]
    # Keys: filter i uses splitmix64 stream 1000+i; its queries are its n_i
    # keys followed by n_i negatives (the next outputs of the same stream).
    ins = torch.empty(total, dtype=torch.int64, device=dev)
    qry = torch.empty(2 * total, dtype=torch.int64, device=dev)
    views = []
    off = qoff = 0
    for i, (m, n) in enumerate(layout):
        workloads.keys_dev(ins[off:].data_ptr(), n, 1000 + i, 0, sh)
        workloads.keys_dev(qry[qoff:].data_ptr(), 2 * n, 1000 + i, 0, sh)
        views.append((ins[off:off + n], qry[qoff:qoff + 2 * n], ins[off:off + n // 2]))
        off += n
        qoff += 2 * n
    f_ins = torch.empty(total, dtype=torch.uint8, device=dev)
    f_q = torch.empty(2 * total, dtype=torch.uint8, device=dev)
    f_d = torch.empty(sum(n // 2 for _, n in layout), dtype=torch.uint8, device=dev)
    fl = []
    off = qoff = doff = 0
    for _, n in layout:
        fl.append((f_ins[off:off + n], f_q[qoff:qoff + 2 * n], f_d[doff:doff + n // 2]))
        off += n
        qoff += 2 * n
        doff += n // 2
    stream.synchronize()
    ops = total + 2 * total + sum(n // 2 for _, n in layout)

    P_i, P_q, P_d = (Batch(len(layout), 2 * total) for _ in range(3))
    P_i.set([(f, "insert", v[0], x[0]) for f, v, x in zip(filters, views, fl)])
    P_q.set([(f, "contains", v[1], x[1]) for f, v, x in zip(filters, views, fl)])
    P_d.set([(f, "remove", v[2], x[2]) for f, v, x in zip(filters, views, fl)])

    def clear():
        for f in filters:
            f.clear(stream=stream)

    def plain():
        for f, v, x in zip(filters, views, fl):
            f.insert(v[0], flags=x[0], stream=stream)
        for f, v, x in zip(filters, views, fl):
            f.contains(v[1], out=x[1], stream=stream)
        for f, v, x in zip(filters, views, fl):
            f.remove(v[2], out=x[2], stream=stream)

    def batched(graph):
        P_i.launch(stream=stream, graph=graph)
        P_q.launch(stream=stream, graph=graph)
        P_d.launch(stream=stream, graph=graph)

    def timed(fn):
        ms = []
        for i in range(warmup + steps):
            clear()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            stream.synchronize()
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        check = {"insert_fail": int((f_ins != 1).sum()),
                 "query_pos_missing": sum(int((x[1][:n] != 1).sum()) for x, (_, n) in zip(fl, layout)),
                 "false_positives": sum(int(x[1][n:].sum()) for x, (_, n) in zip(fl, layout)),
                 "remove_fail": int((f_d != 1).sum())}
        return ops / med / 1e3, med, check

    # Tune on realistic state: inserts on empty filters, the rest after them.
    tune = {}
    clear()
    tune["insert"] = P_i.autotune(stream=stream)
    P_i.launch(stream=stream)
    tune["contains"] = P_q.autotune(stream=stream)
    tune["remove"] = P_d.autotune(stream=stream)
    stream.synchronize()

    plain_mops, plain_ms, plain_chk = timed(plain)
    b_mops, b_ms, b_chk = timed(lambda: batched(False))
    g_mops, g_ms, g_chk = timed(lambda: batched(True))
    for f in filters:
        f.close()
    return {"config": {"workload": "512 filters, 2^8-2^22 buckets x 4, f16, keys 10^2-10^6 "
                                   "log-uniform clipped to LF 0.95; insert, query (n pos + n neg), "
                                   "delete n/2", "filters": len(layout), "keys": total,
                       "table_bytes": sum(m * 8 for m, _ in layout), "ops_per_step": ops},
            "plain": {"mops": round(plain_mops, 2), "ms": round(plain_ms, 3), "checks": plain_chk},
            "batched": {"mops": round(b_mops, 2), "ms": round(b_ms, 3), "checks": b_chk},
            "graph": {"mops": round(g_mops, 2), "ms": round(g_ms, 3), "checks": g_chk},
            "speedup_vs_plain": round(g_mops / plain_mops, 2),
            "tuning": tune,
            "gpu_launches_per_step": {"plain": sum(2 + 1 + 1 for _ in layout),
                                      "batched": 2 + 1 + 1}}


def batched_arm(args):
    import torch

    torch.cuda.set_device(0)
    r = batched_compare(args.steps, args.warmup)
    return {"metric": "multi-filter insert/query/delete Mops/s (one batched launch vs a loop "
                      "of per-filter launches)",
            "mode": "batched", "value": r["graph"]["mops"], "unit": "Mops/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            **r}


def batched_summary() -> dict:
    """The default bench line's batched-vs-loop figures (3 timed
    repetitions after 1)."""
    r = batched_compare(3, 1)
    # Insert placement is nondeterministic, so the false-positive count (which
    # depends on where the tags landed) may differ between the two forms; the
    # failures and the positives missed must not.
    exact = ("insert_fail", "query_pos_missing", "remove_fail")
    return {"workload": r["config"]["workload"],
            "graph_mops": r["graph"]["mops"], "plain_loop_mops": r["plain"]["mops"],
            "speedup": r["speedup_vs_plain"],
            "launches_per_step": r["gpu_launches_per_step"],
            "checks": {"plain": r["plain"]["checks"], "graph": r["graph"]["checks"]},
            "checks_equal": all(r["graph"]["checks"][k] == r["plain"]["checks"][k]
                                for k in exact)}


# ---------------------------------------------------------------------------
# Serving mode: continuous batching vs one plain call per request.
# ---------------------------------------------------------------------------
def _lat_stats(c, n_keys):
    import numpy as np
    lat = (c["done_s"] - c["submit_s"]) * 1e3
    span = float(c["done_s"].max() - c["submit_s"].min())
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3),
            "mops": round(n_keys / span / 1e6, 1),
            "req_per_s": round(len(c) / span, 1),
            "timeouts": int((c["status"] == 4).sum()),
            "errors": int(((c["status"] != 0) & (c["status"] != 4)).sum())}


def serve_compare(n_requests: int, rate_points, admission: bool = True, seed: int = 5):
    """Served (continuous batching) against plain per-request calls on the
    serving workload: saturated throughput, then Poisson arrivals at each
    (name, fraction, of) in rate_points, the rate being fraction x the
    saturated request rate of `of` ("served" or "plain"); p50 / p99
    latency of both forms at each rate.  With admission, also the same
    requests on a server whose HBM budget holds only some of the filters."""
    import numpy as np
    import torch

    import workloads
    from workloads.serve import materialize
    from paper_2603_15486_gb300 import CuckooFilter, Server, _lib, plain_run_trace

    L = _lib.load()
    stream = torch.cuda.Stream()
    sizes, plan = workloads.serve_trace(n_requests)
    budget = 64 << 30
    srv = Server(budget, max_inflight=4, max_wave_items=512, max_wave_keys=1 << 22,
                 use_graphs=True)
    fids = [srv.add_filter(m, 16, 4, 500) for m in sizes]
    plain = [CuckooFilter(m, 16, 4, 500) for m in sizes]
    reqs, keep = materialize(sizes, plan, stream)
    n_keys = sum(p[2] for p in plan)
    sreqs = [(fids[f], op, k, fl, i) for i, (f, op, k, fl) in enumerate(reqs)]
    preqs = [(f, op, k, fl, i) for i, (f, op, k, fl) in enumerate(reqs)]
    assert srv.drain(600000) == 0
    while srv.stats()["live_filters"] < len(fids):
        time.sleep(0.01)

    def reset():
        assert srv.drain(600000) == 0
        for fid in fids:
            h = srv.filter_handle(fid)
            assert h, "server filter not live"
            L.cf_clear(h, None)
        for f in plain:
            f.clear()
        torch.cuda.synchronize()

    R = len(reqs)
    reset()
    c = srv.run_trace(sreqs, [0.0] * R)
    sat_served = _lat_stats(c, n_keys)
    reset()
    p = plain_run_trace(plain, preqs, [0.0] * R, stream=stream)
    sat_plain = _lat_stats(p, n_keys)
    caps = {"served": sat_served["req_per_s"], "plain": sat_plain["req_per_s"]}
    loads = {}
    rng = np.random.default_rng(seed)
    for name, frac, of in rate_points:
        lam = frac * caps[of]
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=R))
        arrivals -= arrivals[0]
        reset()
        c = srv.run_trace(sreqs, arrivals)
        reset()
        p = plain_run_trace(plain, preqs, arrivals, stream=stream)
        loads[name] = {"rate_req_s": round(lam, 1), "served": _lat_stats(c, n_keys),
                       "plain": _lat_stats(p, n_keys)}
    st = srv.stats()
    srv.close()
    out = {"workload": f"{R} requests over {len(sizes)} filters "
                       "(2^16-2^26 buckets x 4, f16), mix 1 insert : 8 query : "
                       "1 delete, n = 2^(20u)", "requests": R, "keys": n_keys,
           "saturated": {"served": sat_served, "plain": sat_plain,
                         "speedup": round(sat_served["mops"] / sat_plain["mops"], 2)},
           "poisson": loads,
           "server": {"waves": st["waves"],
                      "mean_wave_requests": round(st["completed"] / max(1, st["waves"]), 2)}}
    if not admission:
        return out
    # Admission under a small budget: the same requests, saturated, into
    # fresh filters on a server whose HBM budget holds only some of them;
    # each filter is removed right after its last request is submitted, so
    # the waiting filters are admitted as earlier ones close.
    small = 4 << 30
    srv2 = Server(small, max_inflight=4, max_wave_items=512, max_wave_keys=1 << 22,
                  use_graphs=True)
    fids2 = [srv2.add_filter(m, 16, 4, 500) for m in sizes]
    last = {}
    for i, (f, _op, _k, _fl) in enumerate(reqs):
        last[f] = i
    first_pending = srv2.stats()["pending_filters"]
    t0 = time.perf_counter()
    for i, (f, op, k, fl) in enumerate(reqs):
        srv2.submit(fids2[f], op, k, fl, i)
        if last[f] == i:
            srv2.remove_filter(fids2[f])
    rc2 = srv2.drain(600000)
    t_adm = time.perf_counter() - t0
    done2 = srv2.poll(R + 64)
    st2 = srv2.stats()
    srv2.close()
    out["admission"] = {"hbm_budget_bytes": small,
                        "filters_waiting_at_start": first_pending,
                        "drain_status": rc2, "completed": int(len(done2)),
                        "all_ok": bool(len(done2) == R and (done2["status"] == 0).all()),
                        "ms": round(t_adm * 1e3, 1), "mops": round(n_keys / t_adm / 1e6, 1),
                        "used_bytes_after": st2["used_bytes"]}
    return out


def serve_arm(args):
    import torch

    torch.cuda.set_device(0)
    pts = [(f"{int(f * 100)}%", f, "served") for f in (0.5, 0.8, 0.95)]
    pts += [("50%_of_plain_capacity", 0.5, "plain"), ("80%_of_plain_capacity", 0.8, "plain")]
    r = serve_compare(args.serve_requests, pts)
    return {"metric": "served p50/p99 latency and Mops/s vs plain per-request launches",
            "mode": "serve", "value": r["saturated"]["served"]["mops"], "unit": "Mops/s",
            "n_gpus": 1, "higher_is_better": True,
            "config": {"workload": r["workload"] + "; Poisson arrivals at 50/80/95% of the "
                                                  "served capacity and 50/80% of the plain one",
                       "requests": r["requests"], "keys": r["keys"],
                       "hbm_budget_bytes": 64 << 30, "max_inflight_waves": 4,
                       "max_wave_keys": 1 << 22, "graphs": True},
            **{k: r[k] for k in ("saturated", "poisson", "admission", "server")}}


def serve_summary(n_requests: int = 1000) -> dict:
    """The default bench line's served-vs-plain figures: a bounded trace,
    saturated and at Poisson rates of 50% and 80% of the plain form's
    capacity (where the plain form keeps up)."""
    r = serve_compare(n_requests, [("50%_of_plain_capacity", 0.5, "plain"),
                                   ("80%_of_plain_capacity", 0.8, "plain")],
                      admission=False)
    out = {"workload": r["workload"],
           "saturated_mops": {"served": r["saturated"]["served"]["mops"],
                              "plain": r["saturated"]["plain"]["mops"]}}
    for name, v in r["poisson"].items():
        out[name] = {"rate_req_s": v["rate_req_s"],
                     "served": {k: v["served"][k] for k in ("p50_ms", "p99_ms", "mops")},
                     "plain": {k: v["plain"][k] for k in ("p50_ms", "p99_ms", "mops")}}
    return out


# ---------------------------------------------------------------------------
# Ablations of the paper's Sec. 5.4 on the paper's geometry (f16, b = 16).
# ---------------------------------------------------------------------------
def sweep_arm(args):
    """The parameter sweep: fingerprint bits 8 / 16 / 32 x slots 4 / 8 / 16
    on 2^26 buckets, each filled from empty in steps to load factors 0.90,
    0.92, 0.94, 0.96 and 0.98 with distinct keys from [0, 2^32); after each
    step the step's insert rate, failures and eviction-depth percentiles,
    then the query rate of 2^24 stored keys and of 2^24 negatives from
    [2^32, 2^64) with their false-positive rate against Eq. 4 (the paper's
    FPR protocol, Sec. 5.3).  Then Zipf(1.1)-duplicated keys filled to LF
    0.95 on 2^22 buckets for two geometries.  Per-key eviction counts take
    the plain kernels."""
    import numpy as np
    import torch

    import workloads
    from paper_2603_15486_gb300 import CuckooFilter

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    def eq4(f, b, alpha):  # Eq. 4 with fingerprints 1 .. 2^f - 1
        return 1.0 - (1.0 - 1.0 / (2.0 ** f - 1.0)) ** (2.0 * b * alpha)

    m = 1 << 26
    lfs = (0.90, 0.92, 0.94, 0.96, 0.98)
    nq = 1 << 24
    neg = torch.empty(nq, dtype=torch.int64, device="cuda")
    workloads.high_keys_dev(neg.data_ptr(), nq, 8, 0, sh)
    qout = torch.empty(nq, dtype=torch.uint8, device="cuda")
    geoms = []
    for f in (8, 16, 32):
        for b in (4, 8, 16):
            nmax = workloads.lf_count(m, b, lfs[-1])
            keys = torch.empty(nmax, dtype=torch.int64, device="cuda")
            workloads.low32_keys_dev(keys.data_ptr(), nmax, 3, 0, sh)
            stream.synchronize()
            g = CuckooFilter(m, f, b, 500)
            lo, pts = 0, []
            for a in lfs:
                hi = workloads.lf_count(m, b, a)
                fl = torch.empty(hi - lo, dtype=torch.uint8, device="cuda")
                evc = torch.empty(hi - lo, dtype=torch.int32, device="cuda")
                t_ins = timed(lambda: g.insert(keys[lo:hi], flags=fl, evictions=evc,
                                               stream=stream))
                e = evc.cpu().numpy()
                fails = int((fl != 1).sum())
                npos = min(nq, hi)
                if not pts:  # untimed first query (first-launch setup on the host)
                    g.contains(keys[:npos], out=qout[:npos], stream=stream)
                t_qp = timed(lambda: g.contains(keys[:npos], out=qout[:npos], stream=stream))
                found = int(qout[:npos].sum())
                t_qn = timed(lambda: g.contains(neg, out=qout, stream=stream))
                fp = int(qout.sum())
                alpha = g.stats(stream=stream)["occupancy"] / (m * b)
                pts.append({"lf": a, "insert_mops": round((hi - lo) / t_ins / 1e3, 1),
                            "inserted": hi - lo, "fails": fails,
                            "evictions_p50_p90_p95_p99_max": [int(np.percentile(e, q))
                                                              for q in (50, 90, 95, 99)]
                            + [int(e.max())],
                            "query_pos_mops": round(npos / t_qp / 1e3, 1),
                            "query_pos_found": found, "query_pos": npos,
                            "query_neg_mops": round(nq / t_qn / 1e3, 1),
                            "fpr": fp / nq, "fpr_eq4": round(eq4(f, b, alpha), 8)})
                lo = hi
            g.close()
            del keys
            geoms.append({"f": f, "b": b, "table_bytes": m * b * f // 8, "points": pts})
    # Zipf(1.1)-duplicated keys (a universe of as many distinct keys as the
    # fill), filled to LF 0.95 in one call: failures and victims, no
    # assertion of zero (copies of a key beyond the 2b its two buckets hold
    # each run the eviction loop to max_evictions and fail).
    mz = 1 << 22
    zipf = []
    for f, b in ((16, 4), (16, 16)):
        n = workloads.lf_count(mz, b, 0.95)
        zk = torch.from_numpy(workloads.zipf_keys(n, n).view(np.int64)).to("cuda")
        g = CuckooFilter(mz, f, b, 500, victim_capacity=1 << 20)
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        evc = torch.empty(n, dtype=torch.int32, device="cuda")
        t = timed(lambda: g.insert(zk, flags=fl, evictions=evc, stream=stream))
        st = g.stats(stream=stream)
        e = evc.cpu().numpy()
        zipf.append({"f": f, "b": b, "buckets": mz, "keys": n,
                     "insert_mops": round(n / t / 1e3, 1), "fails": int((fl != 1).sum()),
                     "victims": st["victims"],
                     "evictions_p50_p90_p95_p99_max": [int(np.percentile(e, q))
                                                       for q in (50, 90, 95, 99)]
                     + [int(e.max())]})
        g.close()
        del zk
    return {"metric": "parameter sweep: insert / query Mops/s, eviction depth and FPR by "
                      "fingerprint bits, slots and load factor",
            "mode": "sweep", "unit": "Mops/s", "n_gpus": 1, "higher_is_better": True,
            "value": next(p["insert_mops"] for gm in geoms if gm["f"] == 16 and gm["b"] == 16
                          for p in gm["points"] if p["lf"] == 0.96),
            "config": {"workload": "sweep_2^26 (f 8/16/32 x b 4/8/16, LF 0.90-0.98)",
                       "buckets": m, "keys": "distinct low32 (seed 3); negatives high "
                       "(seed 8); Zipf(1.1) over a universe of n keys (rank seed 33)",
                       "negatives": nq, "value_is": "f16 b16 insert Mops/s of the step "
                       "to LF 0.96"},
            "geometries": geoms, "zipf": zipf}


def ablation_arm(args):
    import numpy as np
    import torch

    import workloads
    from paper_2603_15486_gb300 import CuckooFilter

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    def ev(fn, reps=3):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            pre = fn("pre")
            e0.record(stream)
            fn("run")
            e1.record(stream)
            stream.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    # Eviction policy (Fig. 5-6): 2^28 slots (2^24 buckets x 16), pre-fill
    # 3/4 of the target, time the last quarter.
    m, b = 1 << 24, 16
    slots = m * b
    keys = torch.empty(slots, dtype=torch.int64, device="cuda")
    workloads.keys_dev(keys.data_ptr(), slots, 2, 0, sh)
    stream.synchronize()
    evict = {}
    for pol in ("bfs", "dfs"):
        g = CuckooFilter(m, 16, b, 500, eviction=pol)
        g.set_slicing(args.slicing, args.slice_bytes, args.slice_chunk)
        rows = {}
        for alpha in (0.75, 0.8, 0.85, 0.9, 0.95, 0.98, 1.0):
            n = workloads.lf_count(m, b, alpha)
            q = (3 * n) // 4
            evc = torch.empty(n - q, dtype=torch.int32, device="cuda")
            fl = torch.empty(n - q, dtype=torch.uint8, device="cuda")

            def step(phase, q=q, n=n, evc=evc, fl=fl, g=g):
                if phase == "pre":
                    g.clear(stream=stream)
                    g.insert(keys[:q], want_flags=False, stream=stream)
                else:
                    g.insert(keys[q:n], flags=fl, evictions=evc, stream=stream)
            ms = ev(step)
            e = evc.cpu().numpy()
            rows[str(alpha)] = {"mops": round((n - q) / ms / 1e3, 1), "ms": round(ms, 3),
                                "evictions_p90_p95_p99_max": [int(np.percentile(e, 90)),
                                                              int(np.percentile(e, 95)),
                                                              int(np.percentile(e, 99)),
                                                              int(e.max())],
                                "fails": int((fl != 1).sum())}
        evict[pol] = rows
        g.close()
    # Bucket policy (Fig. 7): LF 0.95, L2-resident (2^22 slots) and
    # DRAM-resident (2^28 slots); insert, query+, query-, delete.
    policy = {}
    for name, mm in (("L2_2^22_slots", 1 << 18), ("DRAM_2^28_slots", 1 << 24)):
        n = workloads.lf_count(mm, b, 0.95)
        pos = keys[:n]
        neg = torch.empty(n, dtype=torch.int64, device="cuda")
        workloads.keys_dev(neg.data_ptr(), n, 2, slots, sh)
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        res = {}
        for pol in ("xor", "offset"):
            g = CuckooFilter(mm, 16, b, 500, policy=pol)
            g.set_slicing(args.slicing, args.slice_bytes, args.slice_chunk)

            def ins(phase, g=g):
                if phase == "pre":
                    g.clear(stream=stream)
                else:
                    g.insert(pos, flags=out, stream=stream)
            t_ins = ev(ins)
            fails = int((out != 1).sum())
            t_qp = ev(lambda ph, g=g: ph == "run" and g.contains(pos, out=out, stream=stream))
            found = int(out.sum())
            t_qn = ev(lambda ph, g=g: ph == "run" and g.contains(neg, out=out, stream=stream))
            fpc = int(out.sum())

            def rem(phase, g=g):
                if phase == "pre":
                    g.clear(stream=stream)
                    g.insert(pos, want_flags=False, stream=stream)
                else:
                    g.remove(pos, out=out, stream=stream)
            t_rm = ev(rem)
            res[pol] = {"insert_mops": round(n / t_ins / 1e3, 1),
                        "query_pos_mops": round(n / t_qp / 1e3, 1),
                        "query_neg_mops": round(n / t_qn / 1e3, 1),
                        "delete_mops": round(n / t_rm / 1e3, 1),
                        "insert_fails": fails, "query_pos_found": found, "n": n,
                        "fpr": round(fpc / n, 7)}
            g.close()
        policy[name] = res
    # Sorted insertion (Sec. 4.6.3): the batch sorted by primary bucket
    # before the plain insert kernels, against the unsorted plain insert and
    # the slice-partitioned insert.  The sort is the library's (torch.sort,
    # a device radix sort), as the paper's variant used CUB's; the filter's
    # own kernels hash (cf_hash_debug) and insert.
    from paper_2603_15486_gb300 import hash_debug
    sorted_ins = {}
    for name, mm in (("L2_2^22_slots", 1 << 18), ("DRAM_2^28_slots", 1 << 24)):
        n = workloads.lf_count(mm, b, 0.95)
        pos = keys[:n]
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        res = {}
        for variant in ("unsorted_plain", "sorted_plain", "sliced"):
            g = CuckooFilter(mm, 16, b, 500)
            g.set_slicing("always" if variant == "sliced" else "off")
            part = {}

            def run(phase, g=g, variant=variant, part=part):
                if phase == "pre":
                    g.clear(stream=stream)
                    return
                if variant != "sorted_plain":
                    g.insert(pos, flags=out, stream=stream)
                    return
                with torch.cuda.stream(stream):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    _, i1, _ = hash_debug(pos, 16, mm, stream=stream)
                    order = torch.sort(i1, stable=False).indices
                    ks = pos[order]
                    e0.record(stream)
                    g.insert(ks, flags=out, stream=stream)
                    e1.record(stream)
                    part["e"] = (e0, e1)
            t = ev(run)
            rec = {"ms": round(t, 3), "mops": round(n / t / 1e3, 1),
                   "insert_fails": int((out != 1).sum())}
            if variant == "sorted_plain":
                ins_ms = part["e"][0].elapsed_time(part["e"][1])
                rec["insert_only_ms"] = round(ins_ms, 3)
                rec["hash_sort_gather_ms"] = round(t - ins_ms, 3)
            res[variant] = rec
            g.close()
        sorted_ins[name] = res
    return {"metric": "ablations: BFS vs DFS eviction (Fig. 5-6 protocol), XOR vs Offset "
                      "bucket policy (Fig. 7 protocol), sorted insertion (Sec. 4.6.3)",
            "mode": "ablation", "unit": "Mops/s",
            "value": policy["DRAM_2^28_slots"]["xor"]["insert_mops"], "n_gpus": 1,
            "higher_is_better": True,
            "config": {"geometry": "f16, b = 16", "eviction_table": "2^28 slots (2^24 buckets)",
                       "eviction_protocol": "pre-fill 3/4 of the target load, time the last 1/4",
                       "policy_load_factor": 0.95, "slicing": args.slicing},
            "eviction": evict, "bucket_policy": policy, "sorted_insertion": sorted_ins}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["main", "batched", "serve", "ablation", "sweep"],
                    default="main",
                    help="main: the large-filter headline; batched / serve: the "
                         "many-filters and serving workloads (one JSON line each)")
    ap.add_argument("--serve-requests", type=int, default=4000)
    ap.add_argument("--workload", default="large_2^28x4_f16_lf0.95")
    ap.add_argument("--cpu-workload", default="scale_2^22x4_f16_lf0.95")
    ap.add_argument("--ref-workload", default="ref_2^20x4_f16_lf0.95")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the served-vs-plain and batched-vs-loop summaries")
    ap.add_argument("--extras-requests", type=int, default=1000,
                    help="requests of the served-vs-plain summary trace")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-reads", choices=["staged", "in_place"], default="staged",
                    help="how the end-to-end leg's sliced passes get their keys "
                         "(cf_set_host_reads)")
    ap.add_argument("--e2e-warmup", type=int, default=1)
    ap.add_argument("--e2e-chunk", type=int, default=1 << 27,
                    help="keys per staging chunk of the host-buffer calls (eight "
                         "chunks are staged: 2^27 keys hold 8 GiB of keys in flight, "
                         "enough to keep the host link busy through the longest "
                         "eviction pass)")
    ap.add_argument("--slicing", choices=["off", "auto", "always"], default="auto",
                    help="slice-partitioned execution of the filter calls (cf_set_slicing)")
    ap.add_argument("--evict-map", choices=["off", "auto", "always"], default="auto",
                    help="full-bucket map of the eviction loop (cf_set_eviction_map)")
    ap.add_argument("--evict-levels", choices=["off", "on", "always"], default="on",
                    help="slice-grouped eviction levels (cf_set_eviction_levels; \"on\": "
                         "device-buffer inserts, \"always\": the host-buffer ones too)")
    ap.add_argument("--levels", type=int, default=0,
                    help="eviction levels per insert pass (0: the library default, 12)")
    ap.add_argument("--level-stop", type=int, default=0,
                    help="fewest chains a level runs with (0: the library default, 2^18)")
    ap.add_argument("--slice-bytes", type=int, default=0,
                    help="table bytes per slice (0: the library default, 32 MiB)")
    ap.add_argument("--slice-chunk", type=int, default=0,
                    help="keys per sliced pass (0: the library default, 2^28)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture "
                         "(default: the committed full-size capture, if taken on the "
                         "current kernel sources)")
    args = ap.parse_args(argv)
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1")
    if args.impl == "reference":
        out = reference_arm(args)
    elif args.mode == "batched":
        out = batched_arm(args)
    elif args.mode == "serve":
        out = serve_arm(args)
    elif args.mode == "ablation":
        out = ablation_arm(args)
    elif args.mode == "sweep":
        out = sweep_arm(args)
    else:
        out = gpu_arm(args)
    if out is not None:
        print(json.dumps(out), flush=True)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            dist.destroy_process_group()
    except Exception:
        pass


if __name__ == "__main__":
    main()
