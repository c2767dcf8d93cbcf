"""The multi-rank aggregation of bench.py (replicas, weak scaling) on CPU: two gloo
ranks with different timed regions; the whole-job value is the units of all ranks over
the slowest rank's time, identical on every rank."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [0.5, 2.0, 1.25, 0.75][rank]
        value, sec = bench.job_throughput(1000.0, secs, dist, None)
        dist.barrier()
        q.put((rank, value, sec))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_job_throughput_over_gloo_ranks(world):
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([0.5, 2.0, 1.25, 0.75][:world])
    for rank, value, sec in out:
        assert sec == slowest
        assert value == pytest.approx(world * 1000.0 / slowest, rel=1e-15)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench

    value, sec = bench.job_throughput(300.0, 1.5)
    assert sec == 1.5 and value == pytest.approx(200.0, rel=1e-15)
