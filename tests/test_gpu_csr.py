"""Compressed sparse rows of the projection matrix (xr_system_rows_count / _fill) against the
oracle's rows: every ray's units longer than the grazing threshold match exactly, lengths to
delta (Algorithm 1/2 "Output", eq. conditions_2D_1 / conditions_3D_1, the ambiguity rule of
Section 4.1); the rows equal the library's own sparse-row export entry for entry; the row
pointers are the running sums of the row lengths, also for a ray range in the middle."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
pi = math.pi
ANGLES = np.array([0.0, pi / 2, 0.41, 1.7, 2.9, 4.6])


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _geoms():
    return {
        "fan2d": Geometry("fan2d", 27, 21, dx=0.9, dy=1.1, cx=0.4, cy=-0.6, angles=ANGLES, n_cols=37, du=1.2,
                          sod=60.0, sdd=90.0),
        "cone": Geometry("cone", 19, 17, 13, dx=0.9, dy=1.1, dz=0.8, cx=0.5, cy=-0.4, cz=0.2, angles=ANGLES,
                         n_cols=23, n_rows=15, du=1.3, dv=1.2, sod=50.0, sdd=80.0),
        "par3d": Geometry("par3d", 15, 13, 11, angles=np.stack([ANGLES, 0.3 * np.sin(ANGLES)], axis=1), n_cols=19,
                          n_rows=15, du=0.9, dv=0.8),
    }


@pytest.mark.parametrize("name", ["fan2d", "cone", "par3d"])
def test_csr_rows_match_the_oracle_and_the_sparse_row_export(X, name):
    g = _geoms()[name]
    P = X.Projector(g)
    ptr, col, val = P.system_rows()
    ptr, col, val = ptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    assert ptr.shape == (g.n_rays + 1,) and ptr[0] == 0 and np.all(np.diff(ptr) >= 0)
    assert ptr[-1] == len(col) == len(val)
    rows = [(col[ptr[r]:ptr[r + 1]], val[ptr[r]:ptr[r + 1]]) for r in range(g.n_rays)]
    ref = [O.ray_units(g, r) for r in range(g.n_rays)]
    graze = H.check_unit_sets(g, rows, ref)
    assert graze <= max(4, int(ptr[-1]) // 500)
    # the same walk as the sparse-row export: equal entry for entry
    sample = H.sample_rays(g, 200, seed=3)
    for r, (i_e, l_e) in zip(sample, P.ray_units(sample)):
        np.testing.assert_array_equal(rows[r][0], i_e)
        np.testing.assert_array_equal(rows[r][1], l_e)
    P.close()


def test_csr_of_a_ray_range(X):
    g0 = _geoms()["cone"]
    g = Geometry("cone", g0.nx, g0.ny, g0.nz, dx=g0.dx, dy=g0.dy, dz=g0.dz, cx=g0.cx, cy=g0.cy, cz=g0.cz,
                 angles=np.linspace(0.0, 2 * pi, 41)[:40], n_cols=g0.n_cols, n_rows=g0.n_rows, du=g0.du, dv=g0.dv,
                 sod=g0.sod, sdd=g0.sdd)
    assert g.n_rays > 3 * 4096
    P = X.Projector(g)
    ptr_all, col_all, val_all = (t.cpu().numpy() for t in P.system_rows())
    r0, n = 1234, 777
    ptr, col, val = (t.cpu().numpy() for t in P.system_rows(r0, n))
    assert np.array_equal(ptr, ptr_all[r0:r0 + n + 1] - ptr_all[r0])
    assert np.array_equal(col, col_all[ptr_all[r0]:ptr_all[r0 + n]])
    assert np.array_equal(val, val_all[ptr_all[r0]:ptr_all[r0 + n]])
    # a large range: the one-CTA scan runs many rounds of 4096 row lengths
    ptr = P.system_rows(0, g.n_rays)[0].cpu().numpy()
    assert np.array_equal(ptr, ptr_all)
    # out-of-range requests are refused
    buf = torch.empty(8, dtype=torch.int64, device="cuda")
    assert X.lib().xr_system_rows_count(P.handle, g.n_rays - 2, 3, X._ptr(buf), None) == 2
    assert X.lib().xr_system_rows_count(P.handle, -1, 3, X._ptr(buf), None) == 2
    P.close()
