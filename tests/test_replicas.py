"""The replica path across ranks (CPU, gloo, world size 2): shards are
disjoint and their union is the single-rank release; the report reduces to
total work over the slowest rank's time."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp_

from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import replicas as R


def _rank(rank, world, port, out):
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = I.random_box_field(2, 3, 6, seed=5)
    Lx, Ly, Lz = f.extent
    rel = I.Release(50, (0.0, 0.0, 0.0), (Lx, Ly, Lz), seed=77)
    mine = R.shard_release(rel, rank)
    st = O.release_box(f, mine.n, mine.lo, mine.hi, mine.seed, mine.id_offset)
    r = O.track(f, st)
    steps = float(r["steps"].astype(np.int64).sum())
    ms = 10.0 * (rank + 1)
    tot, slow, rate = R.job_rate(steps, ms, world)
    import torch
    gx = torch.tensor(r["gx"])
    allx = [torch.zeros_like(gx) for _ in range(world)]
    dist.all_gather(allx, gx)
    if rank == 0:
        out.put((tot, slow, rate, [a.numpy() for a in allx]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas():
    import oracle as O
    ctx = mp_.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tot, slow, rate, allx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    f = I.random_box_field(2, 3, 6, seed=5)
    Lx, Ly, Lz = f.extent
    both = O.track(f, O.release_box(f, 100, (0.0, 0.0, 0.0), (Lx, Ly, Lz), seed=77))
    assert np.array_equal(np.concatenate(allx), both["gx"])
    assert tot == float(both["steps"].astype(np.int64).sum())
    assert slow == 20.0 and rate == pytest.approx(tot / 0.02)
