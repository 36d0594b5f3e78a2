"""The replicas-only multi-GPU path of the benchmark: whole-job time is the slowest
rank's, iterations are summed over ranks (world size 2, gloo, CPU)."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, iters = bench.aggregate(torch, dist, 1.5 + rank, 1000 * (rank + 1), "cpu")
    out[rank] = (secs, iters)
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (2.5, 3000.0) and out[1] == (2.5, 3000.0)


def test_aggregate_single_process():
    import torch

    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(torch, None, 2.0, 10, "cpu") == (2.0, 10.0)
