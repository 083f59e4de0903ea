"""The multi-GPU path is replicas only: each rank runs the whole step on its
own GPU, and the job's time is the slowest replica's.  Its host logic -- the
max-over-ranks reduction, the per-step value, and the reference arm running
on rank 0 only -- is checked here with world size 2 on the gloo backend
(CPU processes, 127.0.0.1 rendezvous)."""

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = [12.5, 17.25][rank]  # the second replica is the slow one
        got = bench.max_over_ranks(ms, world, "cpu")
        out[rank] = (got, bench.replica_value(got, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of a process that may hold CUDA state
    out = mgr.dict()
    mp.spawn(_replica, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == (17.25, 17.25 / 2)


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_value(3.5, 1) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
