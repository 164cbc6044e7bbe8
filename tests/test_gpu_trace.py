"""The column-trace walk of cone and helical scans (XR_ORDER_TRACE) against the oracle.

Random flat and equiangular cones and helices with off-centre anisotropic voxels, detectors
taller than the volume (rows that enter or leave through the top and bottom faces), more
rows than one 32-row block and a ragged last block; forward per ray, adjoint image, dot test, the
automatic choice, and scans too steep for the walk (more than one z plane per xy cell),
which keep the crossing-order walk."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
pi = math.pi


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _geom(kind, seed, n_rows=150, n_views=10):
    rng = np.random.default_rng(seed)
    nx, ny, nz = int(rng.integers(20, 41)), int(rng.integers(20, 41)), int(rng.integers(12, 33))
    kw = dict(dx=rng.uniform(0.7, 1.2), dy=rng.uniform(0.7, 1.2), dz=rng.uniform(0.8, 1.3),
              cx=rng.uniform(-2, 2), cy=rng.uniform(-2, 2), cz=rng.uniform(-2, 2),
              angles=np.concatenate([[0.0, pi / 2], rng.uniform(0, 2 * pi, n_views - 2)]),
              n_cols=int(rng.integers(30, 60)), n_rows=n_rows, sod=80.0, sdd=130.0)
    half_h = 0.5 * nz * kw["dz"] * 1.6  # the detector sees past the top and bottom faces
    if kind in ("cone", "helix"):
        kw.update(du=rng.uniform(1.2, 2.0), dv=2 * half_h * 130.0 / 80.0 / n_rows)
    else:
        kw.update(du=rng.uniform(0.012, 0.02), dv=2 * math.atan(half_h / 80.0) / n_rows)
    if kind.startswith("helix"):
        kw["src_z"] = np.linspace(-4.0, 4.0, n_views)
    return Geometry(kind, nx, ny, nz, **kw)


def _check_all(X, P, g, seed, what):
    f = inputs.phantom(g, 8, seed)
    f64 = f.numpy().astype(np.float64).reshape(-1)
    y = P.forward(f.cuda()).cpu().numpy().reshape(-1)
    H.check_rays(g, y, O.forward(g, f64), O.forward(g, np.abs(f64)), float(np.abs(f64).max()), what)
    rng = np.random.default_rng(seed)
    s = rng.random(g.n_rays).astype(np.float32)
    z = P.adjoint(torch.from_numpy(s.reshape(g.sino_shape())).cuda(), method=X.XR_ADJ_SCATTER)
    z = z.cpu().numpy().reshape(-1)
    H.check_adjoint(z, O.adjoint(g, s.astype(np.float64)), what)
    lhs = float(np.dot(y.astype(np.float64), s.astype(np.float64)))
    rhs = float(np.dot(f64, z.astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (what, lhs, rhs)


@pytest.mark.parametrize("kind", ["cone", "cone_arc", "helix", "helix_arc"])
@pytest.mark.parametrize("seed", [1, 2])
def test_trace_walk_matches_the_oracle(X, kind, seed):
    g = _geom(kind, 40 + seed + 10 * inputs.KINDS[kind])
    P = X.Projector(g)
    P.set_tuning(order=X.XR_ORDER_TRACE)
    _check_all(X, P, g, seed, f"{kind} trace")
    P.close()


@pytest.mark.parametrize("n_rows", [1, 31, 32, 33, 64, 65, 128, 129, 300])
def test_trace_walk_row_bands(X, n_rows):
    # one lane per row: a single row, partial and whole 32-row blocks, a ragged last block
    g = _geom("cone", 7, n_rows=n_rows, n_views=6)
    P = X.Projector(g)
    P.set_tuning(order=X.XR_ORDER_TRACE)
    _check_all(X, P, g, 3, f"cone rows={n_rows}")
    P.close()


def test_trace_walk_equals_the_crossing_order_walk(X):
    # the two walks of the same rays agree to the per-ray tolerance
    g = _geom("cone", 11, n_rows=96, n_views=12)
    f = inputs.phantom(g, 8, 5).cuda()
    P = X.Projector(g)
    P.set_tuning(order=X.XR_ORDER_TRACE)
    y1 = P.forward(f).cpu().numpy().reshape(-1).astype(np.float64)
    P.set_tuning(order=X.XR_ORDER_ROWBLOCK)
    y2 = P.forward(f).cpu().numpy().reshape(-1).astype(np.float64)
    f64 = f.cpu().numpy().astype(np.float64).reshape(-1)
    H.check_rays(g, y1, y2, O.forward(g, np.abs(f64)), float(np.abs(f64).max()), "trace vs rowblock")
    P.close()


def test_automatic_order_takes_the_trace_walk_and_steep_scans_fall_back(X):
    g = _geom("cone", 12, n_rows=40, n_views=6)
    P = X.Projector(g)
    f = inputs.phantom(g, 8, 9).cuda()
    y_auto = P.forward(f)
    P.set_tuning(order=X.XR_ORDER_TRACE)
    assert torch.equal(y_auto, P.forward(f))
    P.close()
    # a detector so tall that a row crosses several z planes inside one xy cell: the trace
    # walk does not apply and the crossing-order walk runs (same results as the oracle)
    steep = Geometry("cone", 24, 22, 20, dx=2.0, dy=2.0, dz=0.5, angles=np.linspace(0, 6, 5), n_cols=31,
                     n_rows=41, du=1.5, dv=6.0, sod=60.0, sdd=100.0)
    P = X.Projector(steep)
    P.set_tuning(order=X.XR_ORDER_TRACE)
    _check_all(X, P, steep, 4, "steep cone")
    P.close()


def test_full_size_cone_keeps_no_ray_table(X):
    # the 512^3 cone with a 1024 x 768 detector and 720 views: 566 M rays; the handle holds
    # per-view, per-column and per-sample tables only (a 32-byte record per ray would be 18 GB)
    g = inputs.cone_512()
    P = X.Projector(g)
    assert P.trace_walk
    assert P.table_bytes < 64 << 20, P.table_bytes
    P.close()
