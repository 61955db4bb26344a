"""The multi-GPU bookkeeping of bench.py (one independent melt per rank, the
slowest rank's time, the whole-job rate) on two gloo ranks on the CPU, and
the reference arm's rank split."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 25.0 * rank            # rank 1 is the slow one
        ms = bench.reduce_max(dist, local_ms, "cpu")
        out[rank] = (bench.rank_seed(rank), ms, bench.aggregate_rate(world, 1000, 10, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] != res[1][0]                 # independent melts
    assert res[0][1] == res[1][1] == 125.0         # max over ranks
    # every rank's particles over the slowest time: 2 x 1000 x 10 / 0.125 s
    assert res[0][2] == pytest.approx(160000.0)


def test_single_process_needs_no_group():
    assert bench.reduce_max(None, 3.5, "cpu") == 3.5
    assert bench.aggregate_rate(1, 1_000_000, 100, 10.0) == pytest.approx(1e10)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        nchains, nbeads, cpu_seconds, steps, warmup = 10, 10, 0.1, 1, 3
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
