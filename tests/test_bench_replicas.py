"""The benchmark's replica path on two gloo ranks (CPU): every rank gets the slowest rank's time, and
the job rate counts the units of all ranks over that time (weak scaling, no data-path collective)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")
    out[rank] = (t, bench.job_rate(world, 3, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_rate():
    world, port = 2, 29517
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, v = out[r]
        assert t == 150.0
        assert abs(v - world * 3 * 10 / 0.150) < 1e-9


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 1, 300, 1000.0) == 300.0
