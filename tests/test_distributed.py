"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, no GPU.

Each rank relaxes its own configuration on its own GPU (weak scaling, no data
collective); the only collective is the max-reduction of the step time.  Here
two CPU ranks report different local times and must agree on the job figures.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, value = bench.aggregate(100.0 + 50.0 * rank, 1e12, world, device="cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1e12 / 0.150)


def test_single_rank_aggregate_needs_no_process_group():
    import bench

    ms, value = bench.aggregate(200.0, 5e11, 1)
    assert ms == 200.0 and value == pytest.approx(5e11 / 0.2)
