"""Host logic of the multi-GPU (replicas) benchmark on CPU: two gloo ranks
take the barrier, the max over ranks of their times and the whole-job
throughput; the reference arm does no work on ranks other than 0."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    bench.barrier(world)
    local = [2.0, 3.0][rank]                                    # seconds this rank took
    value, t = bench.job_throughput(world, 1000, 5, local, device="cpu")
    out[rank] = (value, t)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_job_throughput():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, t = out[r]
        assert t == 3.0                                         # max over ranks
        assert value == pytest.approx(world * 1000 * 5 / 3.0)   # all ranks' points


def test_reference_arm_is_a_no_op_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, ref_seconds = 2, 1, 0.1
    assert bench.run_reference(Args()) == 0


def test_single_rank_throughput_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    value, t = bench.job_throughput(1, 1 << 20, 20, 0.15)
    assert t == 0.15 and value == pytest.approx((1 << 20) * 20 / 0.15)
