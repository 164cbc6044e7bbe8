"""GPU: autograd (backward = adjoint kernel), finite differences, SIRT, the persistent
batched plan over uneven problems and CUDA-graph replay."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _proj(g):
    from paper_2006_00686_gb300.xray import Projector
    return Projector(g)


def test_backward_is_the_adjoint_kernel():
    from paper_2006_00686_gb300.xray import project
    g = H.par3d_small()
    P = _proj(g)
    x = inputs.phantom(g, 8, 1).cuda().requires_grad_(True)
    w = torch.rand(g.sino_shape(), device="cuda")
    (project(x, P) * w).sum().backward()
    # the 3D adjoint accumulates with atomics: equal up to the order of the float additions
    ref = P.adjoint(w)
    assert float((x.grad - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
    z_ref = O.adjoint(g, w.double().cpu().numpy().reshape(-1))
    H.check_adjoint(x.grad.cpu().numpy(), z_ref, "autograd backward")


def _fd_check(g, P, seed, eps=1.0):
    """L(x) = 0.5 ||Ax - b||^2 is quadratic: the central difference with any eps equals
    <A^T(Ax - b), v> up to rounding."""
    from paper_2006_00686_gb300.xray import project
    rng = np.random.default_rng(seed)
    x0 = inputs.phantom(g, 10, seed).cuda()
    b = P.forward(inputs.phantom(g, 10, seed + 1).cuda())
    v = torch.from_numpy(rng.standard_normal(g.image_shape()).astype(np.float32)).cuda()

    def loss(x):
        r = (P.forward(x) - b).double()
        return 0.5 * float((r * r).sum())

    x = x0.clone().requires_grad_(True)
    L = 0.5 * ((project(x, P) - b) ** 2).sum()
    L.backward()
    fd = (loss(x0 + eps * v) - loss(x0 - eps * v)) / (2 * eps)
    an = float((x.grad.double() * v.double()).sum())
    assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)
    return x0, b, x.grad


def test_gradient_finite_difference_and_oracle_reduced():
    g = H.par3d_small()
    P = _proj(g)
    x0, b, grad = _fd_check(g, P, 3)
    # oracle gradient A^T (A x - b) in float64 from the same float32 inputs
    r = O.forward(g, x0.double().cpu().numpy().reshape(-1)) - b.double().cpu().numpy().reshape(-1)
    H.check_adjoint(grad.cpu().numpy(), O.adjoint(g, r), "gradient vs oracle")


def test_gradient_finite_difference_full_par3d():
    g = inputs.par3d_256_tilt()
    P = _proj(g)
    _fd_check(g, P, 7)
    P.close()


def _oracle_sirt(g, b, n_iter):
    row = O.forward(g, np.ones(g.n_units))
    col = O.adjoint(g, np.ones(g.n_rays))
    R = np.where(row > 0, 1.0 / np.where(row > 0, row, 1.0), 0.0)
    C = np.where(col > 0, 1.0 / np.where(col > 0, col, 1.0), 0.0)
    x = np.zeros(g.n_units)
    for _ in range(n_iter):
        x = x + C * O.adjoint(g, R * (b - O.forward(g, x)))
    return x


def test_sirt_reduced_matches_oracle_sirt():
    from paper_2006_00686_gb300.recon import SIRT
    g = H.par3d_small()
    P = _proj(g)
    f = inputs.phantom(g, 10, 3)
    b = P.forward(f.cuda())
    s = SIRT(P, b)
    x, res = s.run(20, track=True)
    assert all(r1 <= r0 * (1 + 1e-6) for r0, r1 in zip(res, res[1:]))
    x_ref = _oracle_sirt(g, b.double().cpu().numpy().reshape(-1), 20)
    err = np.abs(x.cpu().numpy().reshape(-1) - x_ref).max() / np.abs(x_ref).max()
    assert err <= 1e-3, err


def test_sirt_full_par3d_graph_replay():
    from paper_2006_00686_gb300.recon import SIRT
    g = inputs.par3d_256_tilt()
    P = _proj(g)
    f = inputs.phantom(g, 30, 3, device="cuda")
    b = P.forward(f)
    s = SIRT(P, b)
    r0 = s.residual_norm()
    x, _ = s.run(20, graph=True)
    r20 = s.residual_norm()
    assert r20 < 0.5 * r0
    # eager iterations reproduce the replayed ones
    s2 = SIRT(P, b)
    x2, res = s2.run(20, track=True)
    assert all(b1 <= a1 * (1 + 1e-6) for a1, b1 in zip(res, res[1:]))
    assert torch.allclose(x, x2, rtol=1e-4, atol=1e-4 * float(x2.abs().max()))
    P.close()


def test_lsq_gradient_descent_decreases():
    from paper_2006_00686_gb300.recon import lsq_gradient_descent
    g = inputs.par2d_64()
    P = _proj(g)
    b = P.forward(inputs.phantom(g, 10, 1).cuda())
    # step below 1/||A||^2 (||A||^2 <= max row sum * max column sum)
    L = float(P.forward(torch.ones(g.image_shape(), device="cuda")).max()) * \
        float(P.adjoint(torch.ones(g.sino_shape(), device="cuda")).max())
    _, losses = lsq_gradient_descent(P, b, 15, 1.0 / L)
    assert all(l1 <= l0 for l0, l1 in zip(losses, losses[1:])) and losses[-1] < 0.5 * losses[0]


# ---------------------------------------------------------------------------------------
# Persistent batched plan over uneven problems; CUDA graphs
# ---------------------------------------------------------------------------------------

def _uneven(sides, views=90):
    out = []
    for s in sides:
        bins = int(math.ceil(1.5 * s / 8.0) * 8)
        v = np.arange(views, dtype=np.float64)
        out.append(inputs.Geometry("fan2d", s, s, angles=2 * math.pi * v / views, n_cols=bins, du=1.2,
                                   sod=1000.0, sdd=1500.0))
    return out


def test_batch_plan_matches_plain_launches():
    from paper_2006_00686_gb300.xray import BatchPlan
    geoms = _uneven([64, 200, 96, 160, 128, 33])
    Ps = [_proj(g) for g in geoms]
    xs = [inputs.phantom(g, 6, 40 + q).cuda() for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    zs = [torch.empty(g.image_shape(), device="cuda") for g in geoms]
    plan = BatchPlan(Ps, xs, ys, tile=128)
    plan.project()
    for P, x, y in zip(Ps, xs, ys):
        # the plan walks 2D problems slab by slab in warp lockstep, the single-image launch in
        # crossing order: the same lengths, summed in another order when the driving index
        # falls along the ray
        ref = P.forward(x)
        assert float((y - ref).abs().max()) <= 1e-5 * float(ref.abs().max())
    plan_adj = BatchPlan(Ps, zs, ys, tile=128)
    plan_adj.backproject()
    for P, z, y in zip(Ps, zs, ys):
        ref = P.adjoint(y, method=1)
        assert float((z - ref).abs().max()) <= 1e-5 * float(ref.abs().max())


def test_batch_plan_ray_setup_rebuilds_the_same_tables():
    # one launch for every problem's detector samples and one for every problem's rays: a
    # mixed plan (fans keep a ray table, the cone keeps none and only its detector table is
    # rebuilt) projects and back-projects bit for bit as before, also captured in a graph
    from paper_2006_00686_gb300.xray import BatchPlan
    geoms = _uneven([48, 90]) + [H.cone_small(24, 10)]
    Ps = [_proj(g) for g in geoms]
    xs = [inputs.phantom(g, 5, 70 + q).cuda() for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    zs = [torch.empty(g.image_shape(), device="cuda") for g in geoms]
    fwd, adj = BatchPlan(Ps, xs, ys), BatchPlan(Ps, zs, ys)
    fwd.project()
    y0 = [y.clone() for y in ys]
    adj.backproject()
    z0 = [z.clone() for z in zs]
    fwd.ray_setup()
    fwd.project()
    adj.backproject()
    torch.cuda.synchronize()
    for a, b in zip(ys, y0):
        assert torch.equal(a, b)
    for a, b in zip(zs, z0):
        assert float((a - b).abs().max()) <= 1e-6 * float(b.abs().max())  # atomics: order only
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fwd.ray_setup()
        fwd.project()
    for y in ys:
        y.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(ys, y0):
        assert torch.equal(a, b)
    for P in Ps:
        P.close()


def test_batch_plan_graph_replay():
    from paper_2006_00686_gb300.xray import BatchPlan
    geoms = _uneven([80, 144, 112])
    Ps = [_proj(g) for g in geoms]
    xs = [inputs.phantom(g, 6, 50 + q).cuda() for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    zs = [torch.empty(g.image_shape(), device="cuda") for g in geoms]
    fwd, adj = BatchPlan(Ps, xs, ys), BatchPlan(Ps, zs, ys)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fwd.project()
        adj.backproject()
    torch.cuda.current_stream().wait_stream(s)
    ref_y = [y.clone() for y in ys]
    ref_z = [z.clone() for z in zs]
    for t in ys + zs:
        t.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fwd.project()
        adj.backproject()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(ys, ref_y):
        assert torch.equal(a, b)
    for a, b in zip(zs, ref_z):
        assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max())


def test_projector_graph_replay_batch16():
    g = H.fan2d_small(128, 90)
    P = _proj(g)
    x = torch.stack([inputs.phantom(g, 6, 60 + b) for b in range(16)]).cuda()
    y = torch.empty(g.sino_shape(16), device="cuda")
    z = torch.empty(g.image_shape(16), device="cuda")
    P.forward(x, out=y)
    P.adjoint(y, out=z)
    ry, rz = y.clone(), z.clone()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        P.forward(x, out=y)
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(graph):
        P.ray_setup()
        P.forward(x, out=y)
        P.adjoint(y, out=z)
    y.zero_()
    z.zero_()
    graph.replay()
    torch.cuda.synchronize()
    # paths that reduce with atomics are equal up to the order of the float additions
    assert float((y - ry).abs().max()) <= 1e-6 * float(ry.abs().max())
    assert float((z - rz).abs().max()) <= 1e-6 * float(rz.abs().max())


def test_fans_uneven_64_full_size():
    from paper_2006_00686_gb300.xray import BatchPlan
    geoms = inputs.fans_uneven()
    assert len(geoms) == 64
    Ps = [_proj(g) for g in geoms]
    xs = [inputs.phantom(g, 10, 500 + q, device="cuda") for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    BatchPlan(Ps, xs, ys).project()
    for q in (0, 17, 63):
        # the single-image launch sums each ray in crossing order, the plan slab by slab: rays of
        # up to ~1500 terms differ by the rounding of the two orders (the oracle bound is below)
        ref = Ps[q].forward(xs[q])
        assert float((ys[q] - ref).abs().max()) <= 1e-4 * float(ref.abs().max())
        g = geoms[q]
        rays = H.sample_rays(g, 300, seed=q)
        f64 = xs[q].double().cpu().numpy().reshape(-1)
        y_ref = O.forward(g, f64, rays=rays)
        scale = O.forward(g, np.abs(f64), rays=rays)
        H.check_rays(g, ys[q].cpu().numpy().reshape(-1)[rays], y_ref, scale, float(np.abs(f64).max()),
                     f"uneven fan {q}")
    for P in Ps:
        P.close()
