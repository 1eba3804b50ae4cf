"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
region's duration is the slowest rank's, every rank sees it, and the
whole-job throughput counts every rank's replica (weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        local = [3.5, 7.25][rank]  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local, world, torch.device("cpu"))
        q.put((rank, slowest, bench.job_throughput(1000, 10, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_both_replicas():
    import multiprocessing as mp
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == 7.25
        assert value == pytest.approx(1000 * 10 * 2 / 7.25 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.job_throughput(10, 4, 1, 2.0) == pytest.approx(20 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=0)) is None
    assert capsys.readouterr().out == ""
