"""Timing of the multi-GPU bench (one z slab per rank): the time is the
slowest rank's and the job value counts every rank's nodes.  Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")     # rank 1 is the slow one
    out[rank] = (t, bench.job_mlups(world, 1000, 10, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 2.0
        assert abs(v - world * 1000 * 10 / 2.0 / 1e6) < 1e-15


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_mlups(1, 2_000_000, 5, 2.0) == 5.0
