"""Multi-process (gloo, CPU) checks of the benchmark's rank logic: the job
time is the slowest rank's, and the whole-job value counts every rank's
region (weak scaling, no data-path collective)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    worst = bench.max_over_ranks(ms, world)
    val = bench.weak_scaling_value(2_160_000, world, 100, worst)
    dist.barrier()
    q.put((rank, worst, val))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_weak_scaling(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    worst = 10.0 + 5.0 * (world - 1)
    for rank, w, v in out:
        assert w == worst
        assert v == pytest.approx(world * 2_160_000 * 100 / (worst * 1e-3))


def test_single_process_value():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.weak_scaling_value(10, 1, 4, 2.0) == pytest.approx(10 * 4 / 2e-3)


def test_launcher_environment_is_read(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (3, 4, 1)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k)
    assert bench.dist_env() == (0, 1, 0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    # under torchrun the other ranks return at once, without work or output
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=1)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
