"""The benchmark's multi-rank logic on CPU: world_size 2 over gloo (127.0.0.1).

Replicas are independent (no data-path collective); the only communication is
the barrier and the max-over-ranks reduction of the timed region, from which
the whole-job rate is formed."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = 1.0 + rank          # rank 1 is the slower replica
    dist.barrier()
    tmax = bench.max_over_ranks(local_seconds, dist)
    rate = bench.whole_job_rate(100.0, world, tmax)
    out[rank] = (tmax, rate)
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (2.0, 100.0 * world / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
