"""The multi-rank logic of bench.py (replicas, one process per GPU, max over ranks)
on CPU with two gloo ranks: every rank sees the slowest rank's time and the
whole-job value counts the queries of all ranks."""
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
    ms = 10.0 * (rank + 1)                 # rank 1 is the slowest
    got = bench.reduce_max(ms, world)
    dist.barrier()
    out[rank] = (got, bench.whole_job_qps(10_000, world, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == pytest.approx(2 * 10_000 / 0.020)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.whole_job_qps(100, 1, 10.0) == pytest.approx(10_000.0)
