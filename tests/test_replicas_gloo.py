"""The multi-GPU bench path is replicas only: ranks share nothing but the
final max-over-ranks timing.  Checked here with two gloo processes on the CPU
(127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        # each replica reports its own time; the job time is the slowest one
        results[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_processes():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(_worker, args=(world, port, results), nprocs=world, join=True,
                           start_method="spawn")
        assert dict(results) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_process_is_identity():
    import torch
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
