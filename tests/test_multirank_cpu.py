"""The whole-job timing of bench.py under torchrun on two CPU ranks (gloo): the slowest
rank's time and the sum of the ranks' crossings."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


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
    ms, cross = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1))
    out[rank] = (ms, cross)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (150.0, 3000.0)


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7.0)
