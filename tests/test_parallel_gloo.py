"""Multi-rank logic on CPU with gloo, world_size 2 (each process is one rank).

The view-sharded transform: each rank projects its own block of views and back-projects it
into a partial image; the sinogram blocks concatenate to the full forward and the all-reduced
partial images equal the full adjoint.  The per-rank compute is the oracle here (no GPU in
this process); the partition and reduction are the code under test."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs, parallel

WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _geom():
    v = np.arange(12, dtype=np.float64)
    return inputs.Geometry("fan2d", 24, 20, angles=2 * math.pi * v / 12, n_cols=33, du=1.3, sod=100.0, sdd=150.0)


def _worker(rank, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        g = _geom()
        f = inputs.phantom(g, 5, 3).double().numpy().reshape(-1)
        views = parallel.view_shards(g.n_views, WORLD)[rank]
        gs = g.subset_views(views)
        y_local = O.forward(gs, f, threads=1)
        # the adjoint of this rank's views, then one all-reduce of the image
        z = torch.from_numpy(O.adjoint(gs, y_local, threads=1))
        parallel.sum_partial_adjoints(z)
        # the largest value over ranks
        m = parallel.max_over_ranks(float(rank + 1))
        out[rank] = (views, y_local, z.numpy(), m)
    finally:
        dist.destroy_process_group()


def test_view_sharded_forward_and_adjoint_gloo():
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(port, out), nprocs=WORLD, start_method="spawn", join=True)
    g = _geom()
    f = inputs.phantom(g, 5, 3).double().numpy().reshape(-1)
    y_full = O.forward(g, f, threads=1).reshape(g.n_views, g.n_cols)
    z_full = O.adjoint(g, y_full.reshape(-1), threads=1)
    views = np.concatenate([out[r][0] for r in range(WORLD)])
    np.testing.assert_array_equal(views, np.arange(g.n_views))  # a partition of the views
    y_cat = np.concatenate([out[r][1].reshape(-1, g.n_cols) for r in range(WORLD)])
    np.testing.assert_allclose(y_cat, y_full, rtol=1e-14, atol=1e-14)
    for r in range(WORLD):
        np.testing.assert_allclose(out[r][2], z_full, rtol=1e-12, atol=1e-12)
        assert out[r][3] == float(WORLD)


class _OracleLocal:
    """A rank's operator computed by the oracle (no GPU in these processes)."""

    def __init__(self, g):
        self.g = g

    def forward(self, img):
        return torch.from_numpy(O.forward(self.g, img.double().numpy().reshape(-1), threads=1))

    def adjoint(self, block):
        z = O.adjoint(self.g, block.double().numpy().reshape(-1), threads=1)
        return torch.from_numpy(z.reshape(self.g.image_shape()))


def _helix():
    v = np.arange(7, dtype=np.float64)
    return inputs.Geometry("helix", 12, 10, 8, angles=2 * math.pi * v / 5, src_z=np.linspace(-2, 2, 7), n_cols=9,
                           n_rows=5, sod=40.0, sdd=60.0)


def _sharded_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = _helix()
        f = inputs.phantom(g, 4, 8).double()
        S = parallel.ShardedProjector(g, make_local=_OracleLocal)
        y = S.forward(f)
        rng = np.random.default_rng(5)
        s_full = rng.random(g.n_rays)
        block = torch.from_numpy(s_full[S.ray0:S.ray0 + S.n_rays])
        z = S.adjoint(block, like=f)
        out[rank] = (S.ray_ids(), None if y is None else y.numpy(), z.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_projector_gloo(world):
    # the library's ShardedProjector over gloo ranks; with 3 ranks and 7 views the blocks are
    # uneven, with 8 ranks one would hold no views (see test_sharded_projector_plan)
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_sharded_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    g = _helix()
    f = inputs.phantom(g, 4, 8).double().numpy().reshape(-1)
    ids = np.concatenate([out[r][0] for r in range(world)])
    np.testing.assert_array_equal(ids, np.arange(g.n_rays))
    y_cat = np.concatenate([out[r][1] for r in range(world) if out[r][1] is not None])
    np.testing.assert_allclose(y_cat, O.forward(g, f, threads=1), rtol=1e-13, atol=1e-13)
    z_full = O.adjoint(g, np.random.default_rng(5).random(g.n_rays), threads=1)
    for r in range(world):
        np.testing.assert_allclose(out[r][2].reshape(-1), z_full, rtol=1e-12, atol=1e-12)


def test_sharded_projector_plan():
    # without a process group: every rank's share of a helical scan; the blocks reassemble the
    # scan's ray ids exactly, each block's rays are the scan's rays (source heights included),
    # and a rank without views holds no operator
    g = _helix()
    for world in (1, 2, 3, 8):
        shares = [parallel.ShardedProjector(g, make_local=lambda gg: gg, rank=r, world=world) for r in range(world)]
        np.testing.assert_array_equal(np.concatenate([s.ray_ids() for s in shares]), np.arange(g.n_rays))
        for s in shares:
            if s.n_rays == 0:
                assert s.local is None and s.forward(None) is None
                continue
            for k in (0, s.n_rays // 2, s.n_rays - 1):
                np.testing.assert_array_equal(O.ray_params(s.local, k), O.ray_params(g, s.ray0 + k))


def test_shards_and_seeds():
    for n, w in ((720, 8), (5, 8), (181, 3)):
        sh = parallel.view_shards(n, w)
        assert len(sh) == w and np.array_equal(np.concatenate(sh), np.arange(n))
        assert max(map(len, sh)) - min(map(len, sh)) <= 1
    seeds = [parallel.rank_seeds(r, 16, 200) for r in range(4)]
    flat = sum(seeds, [])
    assert len(set(flat)) == len(flat) and seeds[0][0] == 200
    assert parallel.max_over_ranks(3.5) == 3.5  # no process group: identity
