"""Work split across ranks (one process per GPU).

Rays are independent (the paper computes them one by one), so the transform shards
without any exchange:
* batches: each rank projects its own images (weak scaling) -- the benchmark's mode;
* views: each rank owns a contiguous block of views of one scan; the forward needs no
  collective (each rank writes its block of the sinogram), the adjoint of the whole scan is
  the sum of the ranks' partial adjoints -- one all-reduce of the image (ShardedProjector).
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


def _group_rank_world(group=None):
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


class ShardedProjector:
    """One scan split by views over the ranks of a process group, one GPU per rank.

    Rank r owns the contiguous block ``views`` of the scan's views (``view_shards``) and a
    projector of that sub-scan: its rays are the global rays ``ray0 .. ray0 + n_rays - 1`` of
    the scan ([view][row][col] order), because a view block is a contiguous range of ray
    ids.  ``forward`` projects the full image onto the rank's block of the sinogram with no
    collective; ``adjoint`` back-projects the rank's block into a partial image and sums the
    partial images of all ranks with one all-reduce (NCCL between GPUs), so every rank ends
    with the adjoint of the whole scan.  A rank without views contributes a zero image.

    make_local(geometry) builds the rank's operator (default: the CUDA Projector); it needs
    forward(img) -> sinogram block and adjoint(block) -> image."""

    def __init__(self, geom, group=None, make_local=None, rank=None, world=None):
        self.geom = geom
        self.group = group
        self.rank, self.world = _group_rank_world(group)
        if rank is not None and world is not None:  # planning one rank's share without a group
            self.rank, self.world = int(rank), int(world)
        self.views = view_shards(geom.n_views, self.world)[self.rank]
        per_view = geom.n_rows * geom.n_cols
        self.ray0 = int(self.views[0]) * per_view if len(self.views) else 0
        self.n_rays = len(self.views) * per_view
        self.local_geom = geom.subset_views(self.views) if len(self.views) else None
        if make_local is None:
            from .xray import Projector
            make_local = Projector
        self.local = make_local(self.local_geom) if self.local_geom is not None else None

    def ray_ids(self):
        """Global ray ids of this rank's sinogram block, in its order."""
        return np.arange(self.ray0, self.ray0 + self.n_rays, dtype=np.int64)

    def forward(self, img, out=None, **kw):
        """This rank's block of the sinogram (views ``self.views``); None without views."""
        if self.local is None:
            return None
        return self.local.forward(img, out=out, **kw) if out is not None else self.local.forward(img, **kw)

    def adjoint(self, block, like=None, **kw):
        """The adjoint of the whole scan on every rank: this rank's partial image (zero without
        views, shaped and placed like ``like``, e.g. the projected image) summed over the ranks
        with one all-reduce."""
        if self.local is None:
            import torch
            z = torch.zeros_like(like)
        else:
            z = self.local.adjoint(block, **kw)
        return sum_partial_adjoints(z, self.group)

    def close(self):
        if self.local is not None and hasattr(self.local, "close"):
            self.local.close()
