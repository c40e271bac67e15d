"""The bench's multi-rank aggregation (replicas: max time over ranks, units summed)
with two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    t, u = bench.whole_job(1.0 + rank, 10.0 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_aggregation_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    # slowest rank's time, all ranks' units
    assert res[0] == res[1] == (2.0, 30.0)


def test_whole_job_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(1.5, 7.0, None, None) == (1.5, 7.0)
