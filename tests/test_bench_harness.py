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
