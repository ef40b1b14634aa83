"""The N > 1 path of bench.py (replicas, no data-path collective) on two CPU ranks over gloo:
the slowest rank's time, the whole-job value, per-rank problems, and the reference arm
printing on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.0][rank]  # rank 1 is the slower one
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        A, B = bench.rank_problem(64, 48, rank)
        digest = float(np.abs(A).sum() + np.abs(B).sum())
        digests = [None] * world
        dist.all_gather_object(digests, digest)
        out[rank] = (slowest, bench.job_value(world, 2.0 * 64 * 64 * 48, slowest), digests)
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_and_job_value():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        slowest, value, digests = out[rank]
        assert slowest == 5.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 2.0 * 64 * 64 * 48 / 5e-3 * 1e-12)
        assert digests[0] != digests[1]  # each rank multiplies its own problem


def test_one_rank_is_identity():
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.job_value(1, 2e12, 1000.0) == pytest.approx(2.0)


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm runs on rank 0; other ranks exit 0 without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--n", "256", "--steps", "1", "--warmup", "0", "--ref-seconds", "1"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--n", "256", "--steps", "1", "--warmup", "0", "--ref-seconds", "1"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
