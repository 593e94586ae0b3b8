"""The N>1 benchmark path on CPU: replicas time themselves, the whole-job
time is the slowest rank's (all_reduce MAX over gloo), and the rate counts
every rank's queries.  world_size 2, launched as two processes."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 1000.0 if rank == 0 else 2500.0          # rank 1 is the slow one
    qps, max_ms = bench.whole_job_qps(local_ms, nq_per_rank=10_000, steps=5, world=world)
    out[rank] = (qps, max_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        qps, max_ms = out[r]
        assert max_ms == 2500.0
        assert qps == pytest.approx(2 * 10_000 * 5 / 2.5)


def test_single_rank_needs_no_collective():
    import bench
    qps, max_ms = bench.whole_job_qps(500.0, 10_000, 4, 1)
    assert max_ms == 500.0 and qps == pytest.approx(80_000.0)
