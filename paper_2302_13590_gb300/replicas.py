"""Replicas across GPUs: every rank tracks its own particles against its own
copy of the field (particles are independent, Introduction and Methods,
"MODPATH"), so nothing is exchanged on the data path.  Only the report is
reduced: total cell-steps (sum) over the slowest rank's time (max)."""
from __future__ import annotations

import dataclasses


def shard_release(release, rank: int):
    """The rank's own particles: the same box and seed with the Philox
    counters shifted by rank * n, so shards are disjoint (weak scaling)."""
    return dataclasses.replace(release, id_offset=release.id_offset + rank * release.n)


def job_rate(cell_steps: float, ms: float, world: int, device=None) -> tuple:
    """(total cell-steps, slowest rank's ms, cell-steps/s of the whole job)."""
    if world <= 1:
        return cell_steps, ms, cell_steps / (ms / 1e3)
    import torch
    import torch.distributed as dist
    s = torch.tensor([cell_steps], dtype=torch.float64, device=device)
    m = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(s.item()), float(m.item()), float(s.item()) / (float(m.item()) / 1e3)
