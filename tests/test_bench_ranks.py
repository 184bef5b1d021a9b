"""Host logic of the benchmark's multi-rank run (replicas, one RVE per rank), on the CPU:
two gloo ranks agree on the slowest rank's time, the whole-job throughput counts every
rank's voxels, and the reference arm runs on rank 0 alone."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 7.0 * rank, dist, "cpu")  # rank 1 is slower
        e2e = bench.max_over_ranks(2.5 - rank, dist, "cpu")         # rank 0 is slower
        q.put((rank, ms, e2e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 107.0, 2.5), (1, 107.0, 2.5)]


def test_job_throughput_and_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    # two ranks of 256^3 voxels, 0.5 s per step for the slowest: 2 * 2^24 / 0.5
    assert bench.job_throughput(256 ** 3, 2, 0.5) == 4 * 256 ** 3


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        assert bench.reference_arm(None, rank=1, world=2) is None
    assert out.getvalue() == ""
