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


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host, here on a 5% scene) prints one JSON
    line with the contract's keys; its e2e moves no bytes."""
    import json
    import subprocess
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    t0 = time.perf_counter()
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--scale", "0.05"], capture_output=True, text=True, timeout=600,
                         env=env, cwd=root)
    wall = time.perf_counter() - t0
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "frames/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    # the line reports frames it timed: the timed region fits inside the process's own run time
    assert d["steps"] * d["ms_per_step"] / 1000.0 < wall
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
