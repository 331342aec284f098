"""The benchmark's multi-rank plumbing on CPU (gloo, world size 2). The path
does not shard: every rank runs its own replica, so the only exchanges are
the barrier around the timed region and the max over ranks of the elapsed
time; rank 0 alone runs the reference arm."""
import os
import socket
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    try:
        got_ws, got_rank, local = bench.dist_setup()
        assert (got_ws, got_rank, local) == (ws, rank, rank)
        assert dist.get_backend() == "gloo"
        bench.barrier(ws)
        # ranks time different durations; everyone reports the slowest
        ms_local = 100.0 + 50.0 * rank
        ms_max = bench.max_over_ranks(ws, ms_local, torch.device("cpu"))
        rate = bench.job_rate_mops(1_000_000, 5, ws, ms_max)
        # a second setup call joins the existing group instead of failing
        bench.dist_setup()
        ref = None
        if rank != 0:
            class A:
                steps, warmup = 1, 1
            ref = bench.reference_arm(A(), bench.WORKLOADS["cuckoo_2e24"], "cuckoo_2e24")
        bench.barrier(ws)
        q.put((rank, ms_max, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_rank_barrier_max_and_job_rate():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, ms_max, rate, ref in res:
        assert ms_max == 150.0  # the slower rank's time, on every rank
        # 2 ranks x 5 steps x 1e6 ops in 0.15 s
        assert rate == pytest.approx(2 * 5 * 1e6 / 0.15 / 1e6)
        if rank == 1:
            assert ref == 0  # rank 1 leaves the reference arm without work
