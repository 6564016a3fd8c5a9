"""The replicas path of bench.py on CPU: two gloo ranks (the GPU run uses NCCL with the same calls).

Each rank times its own replica; the whole-job rate divides the frames of all ranks by the slowest
rank's step time, and the ranks meet at barriers around the timed region."""
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


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        step_ms = [0.50, 0.75][rank]          # the second replica is the slow one
        bench.barrier_if_distributed()
        slowest = bench.max_over_ranks(step_ms)
        bench.barrier_if_distributed()
        out.put((rank, slowest, bench.job_rate(slowest, world)))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [0.75, 0.75]                    # both ranks see the slowest step
    assert all(abs(r[2] - 2 * 1000.0 / 0.75) < 1e-9 for r in res)  # 2 frames per 0.75 ms


def test_single_process_needs_no_group():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_rate(0.5, 1) == 2000.0
    bench.barrier_if_distributed()   # a no-op without a process group


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")

    class A:  # the fields run_reference reads before it returns on a non-zero rank
        steps, warmup, gpus, scale = 1, 0, 2, 1.0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
