"""The N > 1 path of bench.py (independent replicas, one per rank): the job time is the
slowest rank's, the throughput counts every rank's solves, and the reference arm runs
on rank 0 only.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")  # rank 1 is slower
    value = bench.job_throughput(world, 4, ms / 1e3)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank_and_counts_all_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 15.0
        assert abs(value - 2 * 4 / 0.015) < 1e-9


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=0)) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_measured_line():
    """bench.py --impl reference on a tiny mesh (CPU): one JSON line with impl, value,
    the oracle's thread count, an e2e entry and a step time that is the step's own wall
    time (steps x ms_per_step fits in the run)."""
    import json
    import subprocess
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    t0 = time.time()
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--nel", "4",
                          "--steps", "2", "--warmup", "3"], capture_output=True, text=True, check=True, timeout=600)
    wall = time.time() - t0
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["steps"] * d["ms_per_step"] / 1e3 <= wall
