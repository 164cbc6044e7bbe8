"""The remaining C entry points on the GPU: xr_tune (timing + text cache), the one-call batched
forward and adjoint, and the device error word."""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2006_00686_gb300 import inputs
from paper_2006_00686_gb300.inputs import Geometry
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2006_00686_gb300 import xray
    return xray


@pytest.mark.parametrize("scan", ["fan_x8", "cone"])
def test_xr_tune_and_its_cache(X, tmp_path, scan):
    g = H.fan2d_small(64, 40) if scan == "fan_x8" else H.cone_small(24, 12)
    batch = 8 if scan == "fan_x8" else 1
    P = X.Projector(g)
    P.reserve(batch)
    cache = tmp_path / "tune.txt"
    t1 = P.tune(str(cache))
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and len(lines[0].split()) == 7
    # a second handle of the same scan reads the choice from the cache
    P2 = X.Projector(g)
    P2.reserve(batch)
    assert P2.tune(str(cache)) == t1
    assert len(cache.read_text().splitlines()) == 1
    # the tuned handle still matches the oracle
    f = torch.stack([inputs.phantom(g, 6, 80 + b) for b in range(batch)])
    y = P.forward(f.cuda() if batch > 1 else f[0].cuda()).cpu().numpy().reshape(batch, -1)
    f64 = f.double().numpy().reshape(batch, -1)
    y_ref = O.forward(g, f64).reshape(batch, -1)
    scale = O.forward(g, np.abs(f64)).reshape(batch, -1)
    for b in range(batch):
        H.check_rays(g, y[b], y_ref[b], scale[b], float(np.abs(f64[b]).max()), f"tuned {scan}[{b}]")
    P.close()
    P2.close()


def test_one_call_batched_forward_and_adjoint(X):
    sides = [40, 72, 24]
    geoms = []
    for s in sides:
        v = np.arange(36, dtype=np.float64)
        geoms.append(Geometry("fan2d", s, s, angles=2 * math.pi * v / 36, n_cols=int(1.5 * s) // 8 * 8 + 8,
                              du=1.2, sod=300.0, sdd=450.0))
    Ps = [X.Projector(g) for g in geoms]
    xs = [inputs.phantom(g, 5, 90 + q).cuda() for q, g in enumerate(geoms)]
    ys = [torch.empty(g.sino_shape(), device="cuda") for g in geoms]
    zs = [torch.empty(g.image_shape(), device="cuda") for g in geoms]
    arr = (X._Problem * 3)()
    for q in range(3):
        arr[q] = X._Problem(Ps[q].handle.value, xs[q].data_ptr(), ys[q].data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert X.lib().xr_project_batched(arr, 3, stream) == 0
    for q in range(3):
        arr[q] = X._Problem(Ps[q].handle.value, zs[q].data_ptr(), ys[q].data_ptr())
    assert X.lib().xr_backproject_batched(arr, 3, stream) == 0
    torch.cuda.synchronize()
    for q, g in enumerate(geoms):
        ref_y = Ps[q].forward(xs[q])  # the single-image walk: same lengths, summed in crossing order
        assert float((ys[q] - ref_y).abs().max()) <= 1e-5 * float(ref_y.abs().max())
        ref = Ps[q].adjoint(ys[q], method=1)
        assert float((zs[q] - ref).abs().max()) <= 1e-5 * float(ref.abs().max())
    assert X.lib().xr_backproject_batched(arr, 0, stream) == 2  # XR_ERR_SIZE
    for P in Ps:
        P.close()


def test_device_error_word_stays_clear(X):
    g = H.cone_small(32, 12)
    P = X.Projector(g)
    x = inputs.phantom(g, 5, 3).cuda()
    y = P.forward(x)
    P.adjoint(y)
    assert P.device_error() == 0
    P.close()


def test_measurement_probes_report_plausible_peaks(X):
    # FP32 FMA: positive and not above the count of FP32 lanes at the maximum SM clock
    # (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz = 80.5 TFLOP/s; 10 % for clock reporting)
    props = torch.cuda.get_device_properties(0)
    lanes_peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    fma = X.fma_throughput(iters=2000, trials=2)
    assert 0.05 * lanes_peak < fma < 1.1 * lanes_peak
    # L2-only reads of a buffer that fits L2: above the HBM copy rate is expected, far above
    # 100 TB/s would mean the probe did not read
    bw = X.read_bandwidth(16 << 20, 4, 2)
    assert 100.0 < bw < 100_000.0
