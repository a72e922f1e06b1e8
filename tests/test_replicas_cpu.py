"""The multi-GPU path is replicas only: every rank solves its own densities
and the bench reports all ranks' solves over the slowest rank's time.  This
checks that aggregation with two gloo ranks on the CPU (no GPU involved)."""
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

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    elapsed = 10.0 + 5.0 * rank          # rank 1 is the slow replica
    out[rank] = bench.allreduce_max(elapsed, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_process_is_identity():
    import bench
    assert bench.allreduce_max(3.5, None, "cpu") == 3.5
