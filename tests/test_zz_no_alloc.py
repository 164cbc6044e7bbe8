"""The batched forward projection that allocates nothing (xr_project_batched_noalloc).

It exists for callers that cannot call cudaMalloc where they project -- code running
during a global-mode stream capture, hosts whose allocator owns the whole device pool,
loops that cannot afford an allocation's synchronisation -- and keeps its work list in a
fixed array that the library reserves on the device.  Its output must equal that of the
allocating entry point (xr_batch_project) on the same problems, on two calls in a row
(the second call must not see anything left over from the first).  This file is collected
last on purpose."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2006_00686_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


def _fans(sides, views=60):
    out = []
    for s in sides:
        bins = int(math.ceil(1.5 * s / 8.0) * 8)
        v = np.arange(views, dtype=np.float64)
        out.append(inputs.Geometry("fan2d", s, s, angles=2 * math.pi * v / views, n_cols=bins, du=1.2,
                                   sod=1000.0, sdd=1500.0))
    return out


def _problems(X, Ps, xs, ys):
    arr = (X._Problem * len(Ps))()
    for q, (P, x, y) in enumerate(zip(Ps, xs, ys)):
        arr[q] = X._Problem(P.handle.value, x.data_ptr(), y.data_ptr())
    return arr


def _check_against_allocating_entry_point(X, sides, seed):
    geoms = _fans(sides)
    Ps = [X.Projector(g) for g in geoms]
    xs = [inputs.phantom(g, 6, seed + q).cuda() for q, g in enumerate(geoms)]
    ref = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    X.BatchPlan(Ps, xs, ref).project()
    out = [torch.full(g.sino_shape(), float("nan"), device="cuda") for g in geoms]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = X.lib().xr_project_batched_noalloc(_problems(X, Ps, xs, out), len(Ps), 128, stream)
    assert st == 0, X.lib().xr_status_string(st).decode()
    torch.cuda.synchronize()
    for y, r in zip(out, ref):
        scale = float(r.abs().max())
        assert float((y - r).abs().max()) <= 1e-5 * scale  # the tolerance the parity tests use
    return Ps


def test_noalloc_matches_batch_plan_on_two_calls_in_a_row(X):
    # two different work lists back to back: the shared scratch is rewritten each call
    _check_against_allocating_entry_point(X, [64, 150, 33, 96], seed=700)
    _check_against_allocating_entry_point(X, [120, 48, 200], seed=800)


def test_noalloc_rejects_more_problems_than_its_scratch_holds(X):
    g = _fans([16])[0]
    P = X.Projector(g)
    x = torch.zeros(g.image_shape(), device="cuda")
    y = torch.zeros(g.sino_shape(), device="cuda")
    n = 257  # one more than XR_NOALLOC_MAX_PROBLEMS
    arr = _problems(X, [P] * n, [x] * n, [y] * n)
    assert X.lib().xr_project_batched_noalloc(arr, n, 0, None) == 11  # XR_ERR_CAPACITY
