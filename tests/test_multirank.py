"""Multi-process host logic of bench.py with world size 2 on the gloo
backend (CPU): independent replicas, the job's time is the slowest rank's
and its throughput counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    units = [100.0, 140.0][rank]
    t, u = bench.reduce_over_ranks(ms, units, dist, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    port = _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (20.0, 240.0)


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(3.0, 7.0, None, "cpu") == (3.0, 7.0)
