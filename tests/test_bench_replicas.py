"""The replica path of bench.py (one process per GPU, no data-path
collective) exercised on the CPU: two gloo ranks reduce their timings to the
slowest rank's, the whole-job rate counts every replica's points, and the
reference arm launched by torchrun prints one line, from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=2)
    try:
        # rank 0 is slower on the first timing, rank 1 on the second
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.0], "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / f"rank{r}.json") as f:
            assert json.load(f) == [2.0, 10.0, 3.0]


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks([0.25, 7.5], "cpu") == [0.25, 7.5]


def test_whole_job_rate_counts_every_replica():
    # 2 replicas x 16,777,216 points x 100 steps in 79.2 ms (the slowest rank)
    v = bench.whole_job_rate(16_777_216, 100, 2, 79.2)
    assert v == pytest.approx(2 * 16_777_216 * 100 / 0.0792 / 1e9, rel=1e-15)
    assert bench.whole_job_rate(16_777_216, 100, 1, 79.2) == pytest.approx(v / 2, rel=1e-15)


def test_reference_arm_is_silent_off_rank_zero(monkeypatch, capsys):
    import argparse
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, impl="reference")
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["config"] == bench.arm_config(2)
    assert line["steps"] == 1 and line["warmup"] == 3
