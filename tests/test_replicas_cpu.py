"""The multi-GPU path is replicas only: each rank runs the whole workload and
the bench reports the units of all ranks over the slowest rank's time.  The
aggregation is checked with two gloo ranks on the CPU, and so is the bench's
other host-side arithmetic."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 1.5 + rank  # rank 1 is the slow one
        t = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (t, bench.whole_job_rate(1000.0, t * 1e-3, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, rate = res[0]
    assert t == 2.5
    assert rate == pytest.approx(2 * 1000.0 / 2.5e-3)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0


def test_solve_over_products():
    import bench
    assert abs(bench.solve_over_products({"warm_seconds": 6.46e-3, "applies": 41}, 0.0845) - 1.8646) < 1e-3
    assert bench.solve_over_products({"warm_seconds": 1.0, "applies": 0}, 0.1) is None
    assert bench.solve_over_products({"warm_seconds": 1.0, "applies": 3}, None) is None
