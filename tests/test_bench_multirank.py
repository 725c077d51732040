"""Replica aggregation of bench.py across ranks (gloo, world size 2, CPU):
the job time is the slowest rank's and the site updates add up."""
import os
import socket

import pytest
import torch
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
    dist.barrier()
    ms, upd = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), dist, "cpu")
    out[rank] = (ms, upd)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (15.0, 3000.0)


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_ranks(3.5, 42) == (3.5, 42)
