"""The N-GPU form of the benchmark on two CPU ranks over gloo.

The global stage of one array is not partitioned across GPUs: with --gpus N
every rank solves its own replica of the workload (no collective on the data
path) and the job's rate is every rank's units over the slowest rank's time.
These tests run that host logic with world size 2 and check the reference arm's
rank gating (rank 0 alone does the work and prints).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        rate, slowest = bench.whole_job_rate(dist, world, 500.0, seconds[rank], device="cpu")
        ref = bench.reference_arm(None) if rank != 0 else "skipped"
        q.put((rank, rate, slowest, ref))
    finally:
        dist.destroy_process_group()


def _run(world, seconds):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, seconds, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            rank, rate, slowest, ref = q.get(timeout=120)
            out[rank] = (rate, slowest, ref)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    return out


def test_whole_job_rate_is_units_over_slowest_rank():
    out = _run(2, [0.010, 0.025])
    for rank in (0, 1):
        rate, slowest, _ = out[rank]
        assert slowest == pytest.approx(0.025)            # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 500.0 / 0.025)   # all ranks' units over that time


def test_reference_arm_works_on_rank_zero_only():
    out = _run(2, [0.010, 0.010])
    assert out[1][2] is None        # rank 1 returns at once, without running the oracle


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    rate, slowest = bench.whole_job_rate(None, 1, 300.0, 0.5, device="cpu")
    assert slowest == 0.5 and rate == pytest.approx(600.0)
