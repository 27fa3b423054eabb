"""The bench's multi-rank aggregation on two gloo ranks (CPU): each rank
traces its own batch (weak scaling, no collective on the data path); the job
value is the sum of the ranks' rays over the longest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rays, ms = 1000.0 * (rank + 1), 50.0 + 25.0 * rank
    out = bench.aggregate_ranks(rays, ms, world, torch.device("cpu"))
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r] == (3000.0, 75.0)


def test_aggregate_single_rank():
    torch = pytest.importorskip("torch")
    import bench
    assert bench.aggregate_ranks(123.0, 4.5, 1, torch.device("cpu")) == (123.0, 4.5)
