"""The multi-rank host logic of bench.py (replicas, max-over-ranks job time,
whole-job throughput) on world_size 2 with the gloo backend on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, t = bench.aggregate(1000.0, 1.0 + rank, world)    # rank 1 is the slow one
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        value, t = out[r]
        assert t == 2.0                       # max over ranks
        assert value == pytest.approx(world * 1000.0 / 2.0)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(500.0, 0.5, 1) == (1000.0, 0.5)
