"""Distribution of the slices of one parareal iteration over ranks.

The slices of a sweep are independent units (Alg. 3, parFor over n), so a
multi-GPU run needs no collective on the data path: each rank propagates a
contiguous slice range with pr_fine_all_slices(n_begin, n_end), or its own
copy of a workload (weak scaling).  Timing takes the maximum over ranks.
"""
from __future__ import annotations


def slice_range(n_slices: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous range [n_begin, n_end) of rank `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_slices, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Maximum of a per-rank float (time in ms) over the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def gather_ranges(n_slices: int, group=None) -> list[tuple[int, int]]:
    """All ranks' slice ranges, gathered (each rank contributes its own)."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    mine = slice_range(n_slices, world, rank)
    out: list = [None] * world
    dist.all_gather_object(out, mine, group=group)
    return [tuple(r) for r in out]
