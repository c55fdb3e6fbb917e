"""The multi-GPU form of the bench is replicas only (the single solve does not shard): each rank
solves its own copy and the reported time is the slowest rank's.  This checks that reduction
with two gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        v = bench.max_over_ranks(10.0 + 3.5 * rank, torch.device("cpu"))
        out[rank] = v
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert dict(out) == {0: 13.5, 1: 13.5}


def test_max_over_ranks_without_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(7.25, torch.device("cpu")) == 7.25
