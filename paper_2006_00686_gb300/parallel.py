"""Work split across ranks (one process per GPU).

Rays are independent (the paper computes them one by one), so the transform shards
without any exchange:
* batches: each rank projects its own images (weak scaling) -- the benchmark's mode;
* views: each rank owns a contiguous block of views of one scan; the forward needs no
  collective (each rank writes its block of the sinogram), the adjoint of the whole scan is
  the sum of the ranks' partial adjoints -- one all-reduce of the image.
"""
from __future__ import annotations

import numpy as np


def view_shards(n_views: int, world: int) -> list:
    """Contiguous, balanced blocks of view indices, one per rank (empty blocks allowed)."""
    bounds = np.linspace(0, n_views, world + 1).round().astype(np.int64)
    return [np.arange(bounds[r], bounds[r + 1], dtype=np.int64) for r in range(world)]


def rank_seeds(rank: int, batch: int, base: int) -> list:
    """Seeds of the images rank `rank` owns in a weak-scaling run (disjoint across ranks)."""
    return [base + batch * rank + b for b in range(batch)]


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (a no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_partial_adjoints(partial, group=None):
    """Sum the ranks' partial adjoint images in place (one all-reduce)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial
