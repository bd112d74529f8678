"""Weak-scaling split of the integral work over ranks.

Shell quartets are independent units, so N ranks (one process per GPU)
take every N-th quartet of each class's list and need no collective on the
data path; the only cross-rank step is the maximum of the ranks' step
times.
"""
from __future__ import annotations


def shard(lst, rank: int, world: int):
    """Every world-th element of lst, starting at rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return lst[rank::world]


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the value
    itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
