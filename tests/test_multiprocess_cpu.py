"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas, no
data-path collective) agree on the slowest rank's time, the whole-job rate
counts every rank's units, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, device="cpu")
        out[rank] = (ms, bench.whole_job_rate(1e6, ms, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, rate = out[0]
    assert ms == 15.0
    # 2 ranks x 1e6 units in 15 ms
    assert rate == pytest.approx(2e6 / 15e-3 / 1e6)


def test_single_process_without_group():
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5
    assert bench.whole_job_rate(4e6, 2.0, 1) == pytest.approx(2000.0)


def test_reference_arm_only_on_rank_zero(capsys):
    class Args:
        steps, warmup, gpus = 3, 3, 2
    bench.run_reference(Args, world=2, rank=1)
    assert capsys.readouterr().out == ""
