"""The multi-rank path of bench.py on CPU: N processes run independent
replicas (the path has no data exchange: every progenitor batch is its own
problem), the timed region is the slowest rank's, and the value is the units
all ranks processed per second of it.  Two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank              # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, torch.device("cpu"))
        rate = bench.whole_job_rate(1000, 4, world, ms_max)
        q.put((rank, ms_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms_max, rate in got:
        assert ms_max == 15.0                      # both ranks see the slowest rank's time
        assert rate == pytest.approx(1000 * 4 * 2 / 15.0e-3)


def test_single_process_keeps_the_local_time():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(100, 10, 1, 2.0) == pytest.approx(5e5)
