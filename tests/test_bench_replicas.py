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
