"""The benchmark's multi-rank path on CPU: two gloo ranks (127.0.0.1), each timing its own
replica; the job time is the slowest rank's and the job rate counts every rank's units."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 0.25 + 0.5 * rank  # rank 1 is the slower replica
        job_s = bench.max_over_ranks(local_s, device="cpu")
        rate = bench.job_rate(1000.0, job_s, world)
        dist.barrier()
        out.put((rank, job_s, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(world))
    for rank, job_s, rate in got:
        assert job_s == pytest.approx(0.75)
        assert rate == pytest.approx(2 * 1000.0 / 0.75)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5, device="cpu") == 1.5
    assert bench.job_rate(10.0, 2.0, 1) == 5.0
