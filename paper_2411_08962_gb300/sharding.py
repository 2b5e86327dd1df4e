"""Configuration sharding across ranks (one process per GPU).

The correlators of different gauge configurations (and sources) are
independent, so N ranks split the configurations and exchange nothing on the
data path: weak scaling, each rank its own configurations, one collective at
the end to take the slowest rank's time.
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> range:
    """The contiguous block of item indices of `rank` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def config_seed(base: int, index: int) -> int:
    """Seed of configuration `index` of a workload (global index, rank-independent)."""
    return base + 7919 * index


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
