"""The N > 1 path of bench.py on CPU: two gloo ranks, one process each (the
GPU launch uses NCCL with the same calls).  Every rank solves its own
instance (replicas, weak scaling); the job's time is the slowest rank's and
its units are summed over ranks; the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        steps = [1.5 + rank, 2.0 * (rank + 1)]  # rank 0: 3.5 ms, rank 1: 6.5 ms
        iters = [70 + 10 * rank, 70]
        total_ms, units = bench.job_totals(steps, iters, world, "cpu")
        e2e = bench.job_max_ms([10.0 - 4 * rank], world, "cpu")
        out[rank] = (total_ms, units, e2e)
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_summed_units():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    units = bench.H * bench.W * bench.L * float((70 + 70) + (80 + 70))
    for rank in range(world):
        total_ms, u, e2e = res[rank]
        assert total_ms == pytest.approx(6.5)
        assert u == pytest.approx(units)
        assert e2e == pytest.approx(10.0)


def test_single_rank_needs_no_process_group():
    total_ms, units = bench.job_totals([1.0, 2.0], [7, 9], 1, "cpu")
    assert total_ms == 3.0 and units == bench.H * bench.W * bench.L * 16


def test_ranks_solve_their_own_instances():
    from paper_2004_11227_gb300 import synth

    a, b = bench.rank_instance(0, 64), bench.rank_instance(1, 64)
    assert not np.array_equal(a.costs[0], b.costs[0])
    assert a.costs.shape == (bench.L, 64, 64)
    np.testing.assert_array_equal(a.costs, synth.config5(64, 64).costs)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args())
    assert buf.getvalue() == ""
