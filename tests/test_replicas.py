"""Replicas-only multi-GPU path of bench.py on CPU: two gloo ranks, each
with its own timed total; the reported wall time is the maximum over ranks
and the aggregate ms/frame divides it by the frames of all ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total, per_frame = bench.replica_reduce(100.0 + 50.0 * rank, 10)
    out[rank] = (total, per_frame)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1] == (150.0, 150.0 / 20)


def test_single_process_is_its_own_total():
    import bench
    assert bench.replica_reduce(42.0, 7) == (42.0, 6.0)
