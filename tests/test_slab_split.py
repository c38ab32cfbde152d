"""The cavity step shards into y-slabs: two CPU ranks (torch.distributed, gloo), each advancing
its own rows of the oracle field and exchanging one halo row of populations per step with its
neighbour, reproduce the unsplit oracle bitwise.

This is the decomposition a multi-GPU run would use (each wall, lid and NEE reference node only
reads rows y-1..y+1, or the inner row of its wall); here it is exercised on the host only.
"""
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _slab_worker(rank, world, port, nx, ny, steps, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = O.Params.from_re(nx, ny, 80.0, 0.1)
    bounds = np.linspace(0, ny, world + 1).astype(int)
    y0, y1 = bounds[rank], bounds[rank + 1]
    f = O.init(p)  # every rank holds a full-size array but only trusts rows y0-1 .. y1
    for _ in range(steps):
        g = f.copy()
        for y in range(y0, y1):
            for x in range(nx):
                g[y, x] = O.step_node(p, f, x, y)
        # halo exchange: send my first and last owned rows, receive the neighbours' edge rows
        reqs = []
        if rank > 0:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(g[y0])), rank - 1))
        if rank < world - 1:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(g[y1 - 1])), rank + 1))
        if rank > 0:
            buf = torch.empty((nx, 9), dtype=torch.float64)
            dist.recv(buf, rank - 1)
            g[y0 - 1] = buf.numpy()
        if rank < world - 1:
            buf = torch.empty((nx, 9), dtype=torch.float64)
            dist.recv(buf, rank + 1)
            g[y1] = buf.numpy()
        for r in reqs:
            r.wait()
        f = g
    np.save(out_path + f".{rank}.npy", f[y0:y1])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slab_split_matches_unsplit(tmp_path):
    import torch.multiprocessing as mp

    nx, ny, steps, world = 14, 17, 6, 2
    port = 29500 + (os.getpid() % 2000)
    out = str(tmp_path / "slab")
    mp.spawn(_slab_worker, args=(world, port, nx, ny, steps, out), nprocs=world, join=True)
    parts = [np.load(out + f".{r}.npy") for r in range(world)]
    p = O.Params.from_re(nx, ny, 80.0, 0.1)
    ref = O.run(p, O.init(p), steps)
    assert np.array_equal(np.concatenate(parts), ref)
