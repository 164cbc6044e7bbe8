"""The attenuated transform on the GPU (eq. generalizedRadontransform with the exponential
attenuation weight) against the oracle's: forward and adjoint on reduced scans and a ray
list, no attenuation equals the plain transform, the dot test and autograd."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _rays2d():
    rng = np.random.default_rng(2)
    half = 0.5 * math.hypot(40 * 0.9, 36 * 1.1)
    ang = np.stack([rng.uniform(-half, half, 4000), rng.uniform(0, 2 * math.pi, 4000)], axis=1)
    return Geometry("rays2d", 40, 36, dx=0.9, dy=1.1, cx=0.4, cy=-0.2, angles=ang)


SCANS = {
    "fan2d_96": lambda: H.fan2d_small(96, 60),
    "par3d_32": lambda: H.par3d_small(),
    "cone_48": lambda: H.cone_small(48, 30),
    "rays2d": _rays2d,
}


def _mu(g, seed):
    # an attenuation map: a uniform disc/ball of 0.02 per unit length plus a denser phantom
    return (0.02 + 0.05 * inputs.phantom(g, 4, seed)).float()


@pytest.mark.parametrize("name", list(SCANS))
def test_attenuated_matches_oracle(name):
    from paper_2006_00686_gb300.xray import Projector
    g = SCANS[name]()
    P = Projector(g)
    mu = _mu(g, 7)
    f = torch.stack([inputs.phantom(g, 8, 20 + b) for b in range(3)])
    y = P.forward_attenuated(f.cuda(), mu.cuda()).cpu().numpy().reshape(3, -1)
    m64 = mu.double().numpy().reshape(-1)
    f64 = f.double().numpy().reshape(3, -1)
    y_ref = O.forward_attenuated(g, m64, f64)
    scale = O.forward(g, np.abs(f64))
    for b in range(3):
        H.check_rays(g, y[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}]")
    yin = np.random.default_rng(3).random(g.n_rays).astype(np.float32)
    z = P.adjoint_attenuated(torch.from_numpy(yin.reshape(g.sino_shape())).cuda(), mu.cuda()).cpu().numpy()
    H.check_adjoint(z.reshape(-1), O.adjoint_attenuated(g, m64, yin.astype(np.float64)), name)
    P.close()


def test_no_attenuation_is_the_plain_transform():
    from paper_2006_00686_gb300.xray import Projector
    g = H.fan2d_small(96, 60)
    P = Projector(g)
    f = inputs.phantom(g, 8, 4).cuda()
    y0 = P.forward_attenuated(f, torch.zeros(g.image_shape(), device="cuda"))
    y = P.forward(f)
    assert float((y0 - y).abs().max()) <= 1e-5 * float(y.abs().max())


@pytest.mark.parametrize("name", ["fan2d_96", "cone_48"])
def test_attenuated_dot_product_and_autograd(name):
    from paper_2006_00686_gb300.xray import Projector, project_attenuated
    g = SCANS[name]()
    P = Projector(g)
    mu = _mu(g, 9).cuda()
    rng = np.random.default_rng(6)
    x = torch.from_numpy(rng.random(g.image_shape(), dtype=np.float32)).cuda()
    yv = torch.from_numpy(rng.random(g.sino_shape(), dtype=np.float32)).cuda()
    lhs = float((P.forward_attenuated(x, mu).double() * yv.double()).sum())
    rhs = float((x.double() * P.adjoint_attenuated(yv, mu).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    xr = x.clone().requires_grad_(True)
    (project_attenuated(xr, mu, P) * yv).sum().backward()
    ref = P.adjoint_attenuated(yv, mu)
    assert float((xr.grad - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
    P.close()


@pytest.mark.parametrize("batch", [4, 5, 16, 20])
@pytest.mark.parametrize("name", ["fan2d_96", "rays2d"])
def test_attenuated_batched_planes(name, batch):
    # 2D batches on the interleaved layouts against the oracle and against the caller's-layout
    # kernels (the same weights: equal up to the order of the reductions)
    from paper_2006_00686_gb300.xray import Projector, XR_PATH_RAY
    g = SCANS[name]()
    P = Projector(g)
    P.reserve(batch)
    mu = _mu(g, 8).cuda()
    f = torch.stack([inputs.phantom(g, 6, 60 + b) for b in range(batch)])
    y = P.forward_attenuated(f.cuda(), mu)
    m64 = mu.double().cpu().numpy().reshape(-1)
    f64 = f.double().numpy().reshape(batch, -1)
    y_ref = O.forward_attenuated(g, m64, f64)
    scale = O.forward(g, np.abs(f64))
    yh = y.cpu().numpy().reshape(batch, -1)
    for b in range(batch):
        H.check_rays(g, yh[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"{name}[{b}]")
    z = P.adjoint_attenuated(y, mu).cpu().numpy().reshape(batch, -1)
    z_ref = O.adjoint_attenuated(g, m64, yh.astype(np.float64))
    for b in range(batch):
        H.check_adjoint(z[b], z_ref[b], f"{name}[{b}] adjoint")
    Pr = Projector(g)
    Pr.set_tuning(path=XR_PATH_RAY)
    yr = Pr.forward_attenuated(f.cuda(), mu)
    assert float((yr - y).abs().max()) <= 1e-5 * float(y.abs().max())
    P.close()
    Pr.close()
