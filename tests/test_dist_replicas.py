"""Host-side logic of the multi-GPU form (independent replicas, one per rank):
the timed total is the maximum over ranks, so the whole-job value is set by the
slowest replica.  Runs as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    out[rank] = bench.max_over_ranks(local)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_without_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
