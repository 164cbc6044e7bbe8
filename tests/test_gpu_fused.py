"""Forward and adjoint in one launch (xr_project_backproject): the sinogram against the oracle's
forward, the image against the oracle's adjoint of that sinogram -- for problems of up to 256
rays per SM two threads share a ray (one per half of the grid along its driving axis), above
that one thread walks it; and the binding's checks of output buffers."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _rays(kind):
    # random ray lists (Section 4.3), each ray given by its own parameters
    from paper_2006_00686_gb300.inputs import Geometry
    rng = np.random.default_rng(11)
    if kind == "rays2d":
        half = 0.5 * math.hypot(30 * 0.9, 26 * 1.1)
        ang = np.stack([rng.uniform(-half, half, 3000), rng.uniform(0, 2 * math.pi, 3000)], axis=1)
        return Geometry("rays2d", 30, 26, dx=0.9, dy=1.1, cx=0.5, cy=-0.3, angles=ang)
    half = 0.5 * math.sqrt((18 * 0.9) ** 2 + (14 * 1.1) ** 2 + 12 ** 2)
    ang = np.stack([rng.uniform(-half, half, 3000), rng.uniform(-half, half, 3000),
                    rng.uniform(0, 2 * math.pi, 3000), rng.uniform(-math.pi / 2, math.pi / 2, 3000)], axis=1)
    return Geometry("rays3d", 18, 14, 12, dx=0.9, dy=1.1, dz=1.0, cx=0.5, cy=-0.3, cz=0.2, angles=ang)


GEOMS = {
    "par2d_64": inputs.par2d_64,
    "fan2d_96": lambda: H.fan2d_small(96, 60),
    "fan2d_128": lambda: H.fan2d_small(128, 180),  # above 256 rays per SM: one thread per ray
    "par3d_24": lambda: H.par3d_small(24),
    "cone_32": lambda: H.cone_small(32, 12),
    "helix_32": lambda: H.helix_small(32, 16, 12, 2),
    "rays2d": lambda: _rays("rays2d"),
    "rays3d": lambda: _rays("rays3d"),
}


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("batch", [1, 3])
def test_forward_adjoint_in_one_launch(X, name, batch):
    g = GEOMS[name]()
    f = torch.stack([inputs.phantom(g, 6, 20 + b) for b in range(batch)])
    f = f[0] if batch == 1 else f
    P = X.Projector(g)
    y, z = P.forward_adjoint(f.cuda())
    f64 = f.numpy().astype(np.float64).reshape(batch, -1)
    yh = y.cpu().numpy().reshape(batch, -1)
    zh = z.cpu().numpy().reshape(batch, -1)
    y_ref = O.forward(g, f64).reshape(batch, -1)
    scale = O.forward(g, np.abs(f64)).reshape(batch, -1)
    z_ref = np.asarray(O.adjoint(g, yh.astype(np.float64))).reshape(batch, -1)
    for b in range(batch):
        H.check_rays(g, yh[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}] fused forward")
        H.check_adjoint(zh[b], z_ref[b], f"{name}[{b}] fused adjoint")
    # the separate calls give the same sinogram (up to their walks' order of summation) and, up
    # to the order of additions, the image
    y2 = P.forward(f.cuda())
    z2 = P.adjoint(y2)
    assert float((y2 - y).abs().max()) <= 1e-5 * float(y.abs().max())
    assert float((z2 - z).abs().max()) <= 1e-4 * float(z.abs().max())
    P.close()


def test_output_buffers_are_checked(X):
    g = inputs.par2d_64()
    P = X.Projector(g)
    x = torch.ones(g.image_shape(), device="cuda")
    with pytest.raises(X.XRayError):
        P.forward(x, out=torch.empty(g.n_rays - 1, device="cuda"))
    with pytest.raises(X.XRayError):
        P.adjoint(torch.ones(g.sino_shape(), device="cuda"), out=torch.empty(10, device="cuda"))
    with pytest.raises(X.XRayError):
        P.forward_adjoint(x, img_out=torch.empty(g.n_units + 4, device="cuda"))
    with pytest.raises(X.XRayError):
        P.forward_adjoint(torch.ones((0,) + g.image_shape(), device="cuda"))  # an empty batch
    # overlapping buffers are refused by the library (XR_ERR_ARG)
    buf = torch.empty(g.n_units + g.n_rays, device="cuda")
    with pytest.raises(X.XRayError):
        P.forward_adjoint(x, sino_out=buf[:g.n_rays], img_out=x)
    P.close()
