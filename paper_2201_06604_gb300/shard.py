"""Replicas across ranks: one process per GPU, each generating its own
contiguous range of the creator's streams, with no collective on the data
path (streams are independent; Sec. 2.1 creates them one after another).

Rank r of `world` owns streams [r n, (r + 1) n) of the sequence that starts at
`seed`; its first stream is the creator state after r n streams.  Timing is
the maximum over ranks and a whole-job rate counts every rank's units.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import mrg


def rank_seed(seed, rank: int, streams_per_rank: int, generator: str = "mrg32k3a") -> tuple:
    """Creator state at the first stream of `rank` (host only)."""
    return mrg.creator_advance(seed, rank * streams_per_rank, generator)


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest
    rank's time."""
    return units_per_rank * world / (max_ms / 1e3)
