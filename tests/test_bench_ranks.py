"""The replica bench's multi-rank arithmetic on CPU: two gloo ranks, each with
its own step time; every rank must see the slowest rank's time, and the job
rate is all ranks' units over that time (weak scaling, no data-path
collective)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.rank_max(ms_by_rank[rank])
        out[rank] = (ms, bench.job_throughput(world, 1_048_576, ms))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ms_by_rank", [(0.08, 0.11), (0.5, 0.2)])
def test_two_gloo_ranks_take_the_slowest(ms_by_rank):
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, ms_by_rank, out), nprocs=world,
                           join=True, start_method="spawn")
        res = dict(out)
    slow = max(ms_by_rank)
    for r in range(world):
        ms, rate = res[r]
        assert ms == pytest.approx(slow, rel=0, abs=1e-12)
        assert rate == pytest.approx(world * 1_048_576 / (slow * 1e-3), rel=1e-12)


def test_single_process_is_identity():
    import bench
    assert not (dist.is_available() and dist.is_initialized())
    assert bench.rank_max(0.123) == 0.123
    assert bench.job_throughput(1, 1000, 2.0) == pytest.approx(5e5)
