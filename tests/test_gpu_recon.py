"""Reconstruction extensions on the CUDA operators: ordered-subset SIRT against the same
iteration run with the oracle's operators, and Tikhonov-regularised least squares (CGLS)
against the normal-equation solution of the oracle's explicit system matrix."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs, recon
from tests import gpu_helpers as H


def test_subset_views_partition():
    for n, s in ((720, 8), (90, 7), (5, 5), (3, 4)):
        sub = recon.subset_views(n, s)
        flat = np.sort(np.concatenate(sub))
        assert np.array_equal(flat, np.arange(n))
        assert all(np.all(np.diff(x) == s) for x in sub if len(x) > 1)


def _oracle_os_sirt(g, b, n_subsets, sweeps):
    subs = recon.subset_views(g.n_views, n_subsets)
    sino = b.reshape(g.n_views, -1)
    parts = []
    for idx in subs:
        gs = g.subset_views(idx)
        row = O.forward(gs, np.ones(gs.n_units))
        col = O.adjoint(gs, np.ones(gs.n_rays))
        R = np.where(row > 0, 1.0 / np.where(row > 0, row, 1.0), 0.0)
        C = np.where(col > 0, 1.0 / np.where(col > 0, col, 1.0), 0.0)
        parts.append((gs, sino[idx].reshape(-1), R, C))
    x = np.zeros(g.n_units)
    for _ in range(sweeps):
        for gs, bs, R, C in parts:
            x = x + C * O.adjoint(gs, R * (bs - O.forward(gs, x)))
    return x


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["fan2d", "cone"])
def test_os_sirt_matches_oracle(name):
    g = H.fan2d_small(64, 60) if name == "fan2d" else H.cone_small(24, 24)
    f = inputs.phantom(g, 8, 12).double().numpy().reshape(-1)
    b = O.forward(g, f).astype(np.float32)
    s = recon.OSSIRT(g, torch.from_numpy(b.reshape(g.sino_shape())).cuda(), 4)
    x = s.run(3).cpu().numpy().reshape(-1)
    x_ref = _oracle_os_sirt(g, b.astype(np.float64), 4, 3)
    err = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    assert err <= 1e-3, err
    # ordered subsets reach a lower data residual than plain SIRT after the same sweeps
    from paper_2006_00686_gb300.xray import Projector
    P = Projector(g)
    bt = torch.from_numpy(b.reshape(g.sino_shape())).cuda()
    plain = recon.SIRT(P, bt)
    xs, _ = plain.run(3)
    r_os = float((P.forward(s.x) - bt).double().norm())
    r_plain = float((P.forward(xs) - bt).double().norm())
    assert r_os < r_plain
    s.close()
    P.close()


@pytest.mark.gpu
def test_cgls_tikhonov_matches_normal_equations():
    from paper_2006_00686_gb300.xray import Projector
    g = inputs.par2d_64()
    f = inputs.phantom(g, 10, 1).double().numpy().reshape(-1)
    b = O.forward(g, f)
    # explicit system matrix from the oracle's sparse rows
    A = np.zeros((g.n_rays, g.n_units))
    for r in range(g.n_rays):
        idx, ln = O.ray_units(g, r)
        A[r, idx] = ln
    lam = 100.0
    x_star = np.linalg.solve(A.T @ A + lam * np.eye(g.n_units), A.T @ b)
    P = Projector(g)
    x, norms = recon.cgls(P, torch.from_numpy(b.astype(np.float32).reshape(g.sino_shape())).cuda(), 60, lam)
    err = np.abs(x.cpu().numpy().reshape(-1) - x_star).max() / np.abs(x_star).max()
    assert err <= 2e-3, err
    assert norms[-1] <= 1e-3 * norms[0]
    P.close()
