"""Cell partitioning for running one action across several processes.

The action is a sum over cells, so it shards by cells: rank r computes the
partial action of its contiguous cell range into a full-length vector, and the
partial vectors are summed (the only exchange: DoFs on partition interfaces
receive contributions from several ranks).  Batched independent problems shard
by problem with no exchange at all.
"""

from __future__ import annotations


def cell_range(n_cells: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced cell range [c0, c1) of ``rank`` among ``world`` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_cells, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def interface_sum(partial, group=None):
    """Sum the ranks' partial action vectors in place (torch.distributed all-reduce)."""
    import torch.distributed as dist
    dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial


def problems_of_rank(n_problems: int, rank: int, world: int) -> list[int]:
    """Independent problems assigned to ``rank`` (round robin; no exchange needed)."""
    return list(range(rank, n_problems, world))
