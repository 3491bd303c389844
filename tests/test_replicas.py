"""Replica aggregation of bench.py over two gloo ranks on the CPU: the whole-job value is all
ranks' units over the slowest rank's time (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [2.0, 3.0][rank]
    units = [1000.0, 1000.0][rank]
    q.put((rank, bench.aggregate(ms_local, units, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, value = res[r]
        assert ms == pytest.approx(3.0)
        assert value == pytest.approx(2000.0 / 3e-3)


def test_single_replica():
    import bench
    assert bench.aggregate(4.0, 100.0, 1) == (4.0, pytest.approx(25000.0))
