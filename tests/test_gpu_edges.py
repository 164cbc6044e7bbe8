"""Degenerate sizes through every path: single-unit and one-wide images, a single view and a
single detector sample, batches that do not fill a chunk, rays that all miss -- forward and
both adjoints against the oracle, on the caller's-layout kernels and on the fast paths."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _cases():
    v5 = np.linspace(0.1, 2 * pi, 5, endpoint=False)
    par3 = np.stack([v5, 0.3 * np.cos(v5)], axis=1)
    # one tilt axis (phi_1 = 0): the scans run as 2D column problems; phi_2 = 0 is an
    # axis-parallel view; no column plane lies on a slice boundary
    tilt5 = np.stack([np.zeros(5), np.linspace(-1.0, 1.0, 5)], axis=1)
    return {
        "tilt_1x1x1_one_column": Geometry("par3d", 1, 1, 1, angles=tilt5, n_cols=1, n_rows=3, du=0.5, dv=0.5,
                                          u0=0.3),
        "tilt_1x6x5_one_row": Geometry("par3d", 1, 6, 5, angles=tilt5, n_cols=6, n_rows=1, dv=0.7),
        "tilt_7x4x1_one_view": Geometry("par3d", 7, 4, 1, angles=[[0.0, 0.4]], n_cols=4, n_rows=5, dv=0.9),
        "tilt_5x20x6_18_columns": Geometry("par3d", 5, 20, 6, angles=tilt5, n_cols=18, n_rows=7, du=1.1, dv=1.2),
        "par2d_1x1": Geometry("par2d", 1, 1, angles=v5, n_cols=5, du=0.4),
        "par2d_1x9": Geometry("par2d", 1, 9, angles=v5, n_cols=9, du=0.7),
        "fan2d_13x1": Geometry("fan2d", 13, 1, angles=v5, n_cols=17, du=1.1, sod=40.0, sdd=60.0),
        "fan2d_one_view_one_bin": Geometry("fan2d", 16, 12, angles=[0.7], n_cols=1, du=1.0, sod=40.0, sdd=60.0),
        "par3d_1x1x1": Geometry("par3d", 1, 1, 1, angles=par3, n_cols=3, n_rows=3, du=0.5, dv=0.5),
        "par3d_1x7x5": Geometry("par3d", 1, 7, 5, angles=par3, n_cols=9, n_rows=7, du=0.8, dv=0.8),
        "cone_9x1x6": Geometry("cone", 9, 1, 6, angles=v5, n_cols=11, n_rows=9, du=1.3, dv=1.0, sod=30.0, sdd=50.0),
        "cone_one_sample": Geometry("cone", 8, 8, 8, angles=[1.1], n_cols=1, n_rows=1, du=1.0, dv=1.0, sod=30.0,
                                    sdd=50.0),
        "helix_all_miss": Geometry("helix", 8, 8, 4, angles=v5, src_z=np.full(5, 400.0), n_cols=6, n_rows=4,
                                   du=1.0, dv=1.0, sod=30.0, sdd=50.0),
        "rays3d_single": Geometry("rays3d", 5, 4, 3, angles=[[0.2, -0.1, 0.7, 0.4]]),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("path", ["fast", "ray"])
@pytest.mark.parametrize("batch", [1, 5])
def test_degenerate_sizes(name, path, batch):
    from paper_2006_00686_gb300.xray import Projector, XR_PATH_INTERLEAVED, XR_PATH_RAY
    g = CASES[name]
    P = Projector(g)
    assert P.column_batch == name.startswith("tilt_")
    P.set_tuning(path=XR_PATH_INTERLEAVED if path == "fast" else XR_PATH_RAY)
    rng = np.random.default_rng(len(name) + batch)
    f = rng.random((batch,) + g.image_shape()).astype(np.float32)
    y = P.forward(torch.from_numpy(f).cuda()).cpu().numpy().reshape(batch, -1)
    f64 = f.astype(np.float64).reshape(batch, -1)
    y_ref = O.forward(g, f64).reshape(batch, -1)
    scale = O.forward(g, np.abs(f64)).reshape(batch, -1)
    for b in range(batch):
        H.check_rays(g, y[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}]")
    if name == "helix_all_miss":
        assert not y.any()
    yin = rng.random((batch,) + g.sino_shape()).astype(np.float32)
    z_ref = O.adjoint(g, yin.astype(np.float64).reshape(batch, -1)).reshape(batch, -1)
    methods = [1] if g.kind.startswith("rays") else [1, 2]
    for m in methods:
        z = P.adjoint(torch.from_numpy(yin).cuda(), method=m).cpu().numpy().reshape(batch, -1)
        for b in range(batch):
            if np.abs(z_ref[b]).max() == 0:
                assert not z[b].any()
            else:
                H.check_adjoint(z[b], z_ref[b], f"{name}[{b}] method {m}")
    P.close()
