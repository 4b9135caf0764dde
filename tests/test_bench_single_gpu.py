"""Host logic of bench.py on CPU: the library's tensor-core kernels use
cluster TMA multicast on the GPU's own weight copies, so the benchmark
refuses any launch on more than one GPU before it touches a GPU; the
reference arm (the FP64 oracle on host cores) does its work on rank 0 only."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class Args:
    gpus = 1
    steps, warmup, ref_seconds = 2, 1, 0.1


def test_one_gpu_is_accepted(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.single_gpu_only(Args()) is None


def test_more_gpus_are_refused_before_any_gpu_work(monkeypatch, capsys):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    a = Args()
    a.gpus = 2
    assert bench.run_gpu(a) == 2
    line = json.loads(capsys.readouterr().out.strip())
    assert "single GPU only" in line["error"]


def test_torchrun_ranks_are_refused(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "4")
    assert bench.single_gpu_only(Args()) is not None
    assert bench.run_gpu(Args()) == 2
    assert "WORLD_SIZE 4" in json.loads(capsys.readouterr().out.strip())["error"]


def test_reference_arm_is_a_no_op_on_other_ranks(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_parity_sample_is_seeded_distinct_and_large():
    idx = bench.parity_sample(1 << 20)
    assert idx.size == bench.PARITY_POINTS >= 65536
    assert (idx == bench.parity_sample(1 << 20)).all()
    assert (idx[1:] > idx[:-1]).all() and idx[0] >= 0 and idx[-1] < (1 << 20)
    small = bench.parity_sample(1000)
    assert (small == list(range(1000))).all()
