"""Column sharding of block products across ranks (one process per GPU).

The block products G X and G^T Y are independent per column (Sec. 2.5: block
products are loops over columns), so ranks split or replicate column blocks with no
exchange on the data path; the only collective is the host-side timing reduction.
"""
from __future__ import annotations

from typing import Tuple


def shard_columns(total: int, world: int, rank: int) -> Tuple[int, int]:
    """(first column, column count) of `rank` when `total` columns are split evenly over
    `world` ranks; the first `total % world` ranks take one extra column."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, total >= 0")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed milliseconds) over the default group;
    the value itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
