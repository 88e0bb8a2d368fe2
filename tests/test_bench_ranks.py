"""Host logic of the multi-rank bench (replicas: one independent copy of the
workload per rank, no collective on the data path).  Two gloo ranks on the
CPU check that the job time is the slowest rank's, that the whole-job rate
counts every rank's units, and that only rank 0 runs the reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r timed (10 + r) ms for the steps and (30 - r) ms end to end
        got = bench._max_over_ranks([10.0 + rank, 30.0 - rank], "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ws = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0] == [11.0, 30.0] and out[1] == [11.0, 30.0]


def test_single_rank_values_pass_through():
    assert bench._max_over_ranks([1.5, 2.5], "cpu") == [1.5, 2.5]


def test_job_rate_counts_every_rank():
    # 2 replicas of 1,000 points, 4 steps in 8 ms: 8,000 points in 8 ms
    assert bench._job_rate(2, 1000, 4, 8.0) == pytest.approx(1.0e6)
    assert bench._job_rate(1, 1000, 4, 8.0) == pytest.approx(0.5e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        workload, ref_elems, warmup, steps = "c1_two_atom_4cube", 1, 0, 1

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "_oracle_steps", boom)
    assert bench.run_reference(Args()) is None
