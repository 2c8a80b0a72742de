"""The multi-rank path of bench.py (independent replicas, no data-path
collective): two gloo ranks on the CPU, each with its own work and time; the
whole-job value is the sum of the units over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, tmax = bench.replica_value(units=1000.0 * (rank + 1), seconds=1.0 + rank, dist=dist, device="cpu")
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_replica_value_two_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax = out[r]
        assert tmax == 2.0
        assert value == pytest.approx(3000.0 / 2.0)


def test_replica_value_single():
    import bench
    assert bench.replica_value(500.0, 2.0) == (250.0, 2.0)
