"""Host-side logic of bench.py: the multi-rank reduction (gloo, two CPU
ranks), the algorithmic byte model and the CPU reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, ops = bench.reduce_max_sum(1.0 + rank, 10.0 * (rank + 1))
    bench.barrier()
    q.put((rank, t, ops, bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_max_time_sum_ops():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, ops, env in got:
        assert t == 2.0 and ops == 30.0
        assert env == (2, rank, rank)


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_sum(3.5, 7.0) == (3.5, 7.0)


def test_bytes_per_op_model():
    sys.path.insert(0, ROOT)
    import bench
    ph = {"query": {"ops": 4, "bucket_reads": 6, "bucket_writes": 0},
          "insert": {"ops": 2, "bucket_reads": 2, "bucket_writes": 2}}
    b8 = bench.bytes_per_op(ph, 8)     # 8-byte buckets: one sector each
    assert b8["query"] == 1.5 * 32 + 9
    assert b8["insert"] == 2 * 32 + 9
    b64 = bench.bytes_per_op(ph, 64)   # 64-byte buckets: two sectors each
    assert b64["query"] == 1.5 * 64 + 9


def test_eviction_times_merge_levels_and_loop():
    sys.path.insert(0, ROOT)
    import bench
    kb = {"insert_evict": 50e9, "slice_probe1": 1.0}
    kt = {"insert_evict": (10, 30.0), "evict_level": (5, 70.0), "slice_probe1": (10, 5.0)}
    got, parts = bench.merge_eviction_times(kt, kb, 5)
    assert got == {"slice_probe1": (10, 5.0), "eviction": (5, 100.0)}
    assert kb["eviction"] == 50e9
    assert parts == {"levels_ms_per_step": 14.0, "loop_and_rest_ms_per_step": 6.0}
    # Without level records (levels off, or the plain path) nothing changes.
    kt2 = {"insert_evict": (10, 30.0), "evict_level": (0, 0.0)}
    got2, parts2 = bench.merge_eviction_times(kt2, {"insert_evict": 1.0}, 5)
    assert got2 == {"insert_evict": (10, 30.0)} and parts2 is None


def test_slice_stream_byte_model():
    """Per-pass stream bytes of the sliced path, worked by hand for a table
    of 1000 bytes and one call per operation: 100 inserts (half pending
    after their first bucket), 200 queries (a quarter pending), 50 deletes
    (none pending), passes of at most 64 keys."""
    sys.path.insert(0, ROOT)
    import bench

    class W:
        table_bytes = 1000
        n_queries, n_deletes = 200, 50

        def insert_segments(self):
            return [(0, 100)]

    ph = {"insert": {"ops": 100, "direct_reads": 150},
          "query": {"ops": 200, "bucket_reads": 250},
          "delete": {"ops": 50, "bucket_reads": 50}}
    got = bench.slice_kernel_bytes(ph, W(), 64)
    # passes: insert 2, query 4, delete 1; sweeps: read once for queries,
    # read and written back for insert and delete.
    sweep = 1000 * (2 * 2 + 1 * 4 + 2 * 1)
    assert got["slice_split"] == 350 * 20
    assert got["slice_probe1"] == 100 * (12 + 0.5 * 8) + 200 * (12 + 0.25 * 8) + 50 * 12 + sweep
    assert got["slice_probe2"] == 100 * 0.5 * 9 + 200 * 0.25 * 9 + sweep
    assert got["slice_merge"] == 100 * (11 + 0.5) + 200 * (11 + 0.25) + 50 * 11


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mops/s"
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
