"""Slice sharding across ranks (one process per GPU).

Slices are independent least-squares problems that share the operator A
(Sec. II-B), so the data-parallel path splits a volume's slices across ranks
and every rank builds its own copy of A and solves its slices alone: no data
exchange on the path.  The only collective is the host-side max of the
per-rank times used for reporting.  The paper's distributed design (Sec.
III-B: partitioned A with hierarchical reduction between nodes) is not this:
on one node each GPU holds all of A, which fits in HBM for every workload
here.
"""
from __future__ import annotations


def slice_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first slice, count) of `rank` when `total` slices are split into
    `world` contiguous ranges whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError(f"bad split: total={total}, world={world}, rank={rank}")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def weak_range(per_rank: int, rank: int) -> tuple[int, int]:
    """(first slice, count) of `rank` when every rank takes `per_rank`
    consecutive slices of a volume of world * per_rank slices."""
    if per_rank < 0 or rank < 0:
        raise ValueError(f"bad split: per_rank={per_rank}, rank={rank}")
    return rank * per_rank, per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (the value
    itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
