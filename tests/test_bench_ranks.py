"""The multi-rank bookkeeping of bench.py (replicas: one independent cavity per rank) on two CPU
ranks over gloo: every rank sees the slowest rank's time, and the whole-job rate counts every
rank's work."""
import os

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, world)  # rank 1 is the slow one
    rate = bench.whole_job_rate(1000.0, t, world)
    with open(f"{out}.{rank}", "w") as fh:
        fh.write(f"{t} {rate}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    port = 31500 + (os.getpid() % 2000)
    out = str(tmp_path / "r")
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, rate = map(float, open(f"{out}.{r}").read().split())
        assert t == 2.5 and rate == 2 * 1000.0 / 2.5


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
