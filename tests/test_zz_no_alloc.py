"""The batched forward projection that allocates nothing (xr_project_batched_noalloc).

It exists for callers that cannot call cudaMalloc where they project -- code running
during a global-mode stream capture, hosts whose allocator owns the whole device pool,
loops that cannot afford an allocation's synchronisation -- and keeps its work list in a
fixed array that the library reserves on the device.  It walks every ray in crossing order
on the caller's layout, as xr_project does for one problem of these sizes, so its output must
equal that of the allocating entry point bit for bit, on two calls in a row (the second call
must not see anything left over from the first).  A batch plan of the same 2D problems walks
slabs on pair planes instead: the same lengths summed in another order, equal within the
parity tolerance.  This file is collected last on purpose."""
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


def _references(X, Ps, xs, geoms):
    """Each problem's xr_project (bitwise reference), checked against one batch plan."""
    ref = [P.forward(x) for P, x in zip(Ps, xs)]
    plan = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    X.BatchPlan(Ps, xs, plan).project()
    for r, q in zip(ref, plan):
        assert float((r - q).abs().max()) <= 1e-5 * float(r.abs().max())
    return ref


def _check_against_allocating_entry_point(X, sides, seed):
    geoms = _fans(sides)
    Ps = [X.Projector(g) for g in geoms]
    xs = [inputs.phantom(g, 6, seed + q).cuda() for q, g in enumerate(geoms)]
    ref = _references(X, Ps, xs, geoms)
    out = [torch.full(g.sino_shape(), float("nan"), device="cuda") for g in geoms]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = X.lib().xr_project_batched_noalloc(_problems(X, Ps, xs, out), len(Ps), 128, stream)
    assert st == 0, X.lib().xr_status_string(st).decode()
    torch.cuda.synchronize()
    for y, r in zip(out, ref):
        # the same walk over the same voxels in the same order: equal bit for bit
        assert torch.equal(y, r)
    return Ps


def test_noalloc_matches_batch_plan_on_two_calls_in_a_row(X):
    # two different work lists back to back: the shared scratch is rewritten each call
    _check_against_allocating_entry_point(X, [64, 150, 33, 96], seed=700)
    _check_against_allocating_entry_point(X, [120, 48, 200], seed=800)


def test_noalloc_runs_inside_a_global_mode_capture_without_allocating(X):
    # a caller that may not allocate: after one warm call (which looks up the scratch
    # address), further calls leave free device memory where it was, and a call made while
    # the stream is captured with capture_error_mode="global" -- where a cudaMalloc would
    # fail the capture -- records and replays the same result
    geoms = _fans([80, 56, 112])
    Ps = [X.Projector(g) for g in geoms]
    xs = [inputs.phantom(g, 6, 900 + q).cuda() for q, g in enumerate(geoms)]
    ref = _references(X, Ps, xs, geoms)
    out = [torch.zeros(g.sino_shape(), device="cuda") for g in geoms]
    arr = _problems(X, Ps, xs, out)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert X.lib().xr_project_batched_noalloc(arr, len(Ps), 0, stream) == 0  # warm call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert X.lib().xr_project_batched_noalloc(arr, len(Ps), 0, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for y in out:
        y.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        cap = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert X.lib().xr_project_batched_noalloc(arr, len(Ps), 0, cap) == 0
    graph.replay()
    torch.cuda.synchronize()
    for y, r in zip(out, ref):
        assert torch.equal(y, r)


def test_backproject_batched_on_two_calls_in_a_row_matches_the_oracle(X):
    # the adjoint twin shares the array: two different problem sets back to back, each
    # checked against the oracle's adjoint (the parity tolerance) and the library's scatter
    from oracle import oracle as O
    from tests import gpu_helpers as H
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for sides, seed in (([48, 90, 30], 40), ([72, 36], 60)):
        geoms = _fans(sides, views=24)
        Ps = [X.Projector(g) for g in geoms]
        rng = np.random.default_rng(seed)
        ys = [torch.from_numpy(rng.random(g.sino_shape(), dtype=np.float32)).cuda() for g in geoms]
        zs = [torch.full(g.image_shape(), float("nan"), device="cuda") for g in geoms]
        assert X.lib().xr_backproject_batched(_problems(X, Ps, zs, ys), len(Ps), stream) == 0
        torch.cuda.synchronize()
        for P, g, y, z in zip(Ps, geoms, ys, zs):
            z_ref = O.adjoint(g, y.cpu().numpy().astype(np.float64).reshape(-1))
            H.check_adjoint(z.cpu().numpy(), z_ref.reshape(g.image_shape()), "xr_backproject_batched")
            ref = P.adjoint(y, method=1)
            assert float((z - ref).abs().max()) <= 1e-5 * float(ref.abs().max())
        for P in Ps:
            P.close()


def test_noalloc_rejects_more_problems_than_its_scratch_holds(X):
    g = _fans([16])[0]
    P = X.Projector(g)
    x = torch.zeros(g.image_shape(), device="cuda")
    y = torch.zeros(g.sino_shape(), device="cuda")
    n = 257  # one more than XR_NOALLOC_MAX_PROBLEMS
    arr = _problems(X, [P] * n, [x] * n, [y] * n)
    assert X.lib().xr_project_batched_noalloc(arr, n, 0, None) == 11  # XR_ERR_CAPACITY
