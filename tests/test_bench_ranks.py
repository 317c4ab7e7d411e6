"""Host logic of bench.py's multi-rank run, on CPU with gloo (world size 2).

The method needs no exchange between GPUs: N ranks run N independent
replicas of the workload (weak scaling).  What the ranks share is the timing
protocol -- a barrier on both sides of the timed region, the maximum of the
per-rank times, one whole-job value -- and the reference arm, which only
rank 0 runs.  These tests run that protocol in two gloo processes.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms_max = bench.max_over_ranks(times[rank], world, device="cpu")
        bench.barrier(world)
        q.put((rank, ms_max, bench.job_value(1.0e9, world, ms_max)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [1.25, 2.5]          # ms per step of rank 0 and rank 1
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in got:
        assert ms_max == 2.5                      # the slowest rank sets the time
        assert value == pytest.approx(2 * 1.0e9 / 2.5e-3)   # units of both ranks


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_value(5.0e9, 1, 2.0) == pytest.approx(2.5e12)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""                # only rank 0 prints the line
