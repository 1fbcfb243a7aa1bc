"""The multi-rank measurement logic of bench.py, on the CPU with two gloo ranks:
each rank times its own replica of the batch, the job's step time is the
slowest rank's (all-reduce MAX), and the job's throughput counts every rank's
cells (weak scaling).  No GPU and no data-path collective are involved."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slowest
        step_max = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
        q.put((rank, step_max, bench.job_gcups(world, 1e11, step_max)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_step_and_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, step_max, gcups in got:
        assert step_max == 15.0                          # the MAX over ranks, on every rank
        assert gcups == pytest.approx(2 * 1e11 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, torch.device("cpu")) == 12.5
    assert bench.job_gcups(1, 1.024e11, 26.7) == pytest.approx(1.024e11 / 26.7e-3 / 1e9)
