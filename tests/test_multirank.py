"""The benchmark's multi-rank path on the CPU (gloo, world size 2).

bench.py under torchrun runs one independent replica per GPU (the hull does
not shard; no data-path collective): each rank times its own steps, the
slowest rank's time bounds the step (max over ranks), and the whole-job rate
counts every rank's points.  These tests run those pieces in two gloo
processes, and check that the reference arm leaves the work to rank 0.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = [3.0, 5.0][rank]                    # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        pts_per_rank = 3 * 1000
        rate = bench.whole_job_rate(pts_per_rank * world, ms)
        dist.barrier()
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 5.0                               # both ranks see the slowest rank's time
        assert rate == pytest.approx(2 * 3000 / 5e-3 / 1e6)


def test_single_process_helpers_need_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, None, "cpu") == 4.5
    assert bench.whole_job_rate(60_000_000, 0.7) == pytest.approx(60e6 / 0.7e-3 / 1e6)


def test_reference_arm_leaves_the_work_to_rank_zero():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""                      # rank 1 prints nothing and does no work
