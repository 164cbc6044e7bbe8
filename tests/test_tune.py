"""Autotuner: candidate lists and the JSON cache on CPU; on the GPU the chosen tuning
still matches the oracle and a second call reads the cache instead of timing."""
import json
import math

import numpy as np
import pytest
import torch

from paper_2006_00686_gb300 import inputs, tune
from paper_2006_00686_gb300 import xray as X


def _fan(n=40, views=24):
    v = np.arange(views, dtype=np.float64)
    return inputs.Geometry("fan2d", n, n, angles=2 * math.pi * v / views, n_cols=57, du=1.1, sod=90.0, sdd=140.0)


def test_candidates_cover_paths():
    g = _fan()
    c16 = tune.projector_candidates(g, 16)
    paths = {c["path"] for c in c16}
    assert paths == {X.XR_PATH_INTERLEAVED, X.XR_PATH_TILED, X.XR_PATH_RAY}
    assert {c["adjoint"] for c in c16} == {X.XR_ADJ_GATHER, X.XR_ADJ_SCATTER}
    assert {c["batch_chunk"] for c in c16 if c["path"] == X.XR_PATH_INTERLEAVED} == {4, 8, 16}
    # a batch below four images: the single-image copy path or the caller's layout
    assert {c["path"] for c in tune.projector_candidates(g, 1)} == {X.XR_PATH_INTERLEAVED, X.XR_PATH_RAY}
    # no candidate walks more images per thread than the batch holds (rounded to four)
    assert {c["batch_chunk"] for c in tune.projector_candidates(g, 5)
            if c["path"] == X.XR_PATH_INTERLEAVED} == {4, 8}
    g3 = inputs.Geometry("cone", 8, 8, 8, angles=np.arange(4) * 0.5, n_cols=9, n_rows=9, sod=40.0, sdd=60.0)
    c3 = tune.projector_candidates(g3, 8)
    assert {c["adjoint"] for c in c3} == {X.XR_ADJ_GATHER, X.XR_ADJ_SCATTER}
    # cone and helical scans also try the column-trace walk (scatter adjoint)
    assert {c["order"] for c in c3} == {X.XR_ORDER_VIEW, X.XR_ORDER_ROW, X.XR_ORDER_COLUMN, X.XR_ORDER_ROWBLOCK,
                                        X.XR_ORDER_TRACE}
    assert all(c["adjoint"] == X.XR_ADJ_SCATTER for c in c3 if c["order"] == X.XR_ORDER_TRACE)
    gp = inputs.Geometry("par3d", 8, 8, 8, angles=np.stack([np.arange(4) * 0.5, np.arange(4) * 0.2], axis=1),
                         n_cols=9, n_rows=9)
    assert X.XR_ORDER_TRACE not in {c["order"] for c in tune.projector_candidates(gp, 1)}
    assert all(c["path"] != X.XR_PATH_TILED for c in tune.projector_candidates(g3, 8))


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert tune._load(p) == {}
    tune._store(p, {"k": {"block": 128}})
    assert tune._load(p) == {"k": {"block": 128}}
    with open(p, "w") as fh:
        fh.write("{not json")
    assert tune._load(p) == {}  # a damaged cache is ignored, not fatal


@pytest.mark.gpu
def test_tuned_projector_matches_oracle(tmp_path):
    from oracle import oracle as O
    g = _fan()
    P = X.Projector(g)
    cache = str(tmp_path / "tune.json")
    best = tune.tune_projector(P, 8, cache_path=cache, reps=2, budget_s=0.5)
    assert P.tuning()["path"] == best["path"] and P.tuning()["adjoint"] == best["adjoint"]
    x = inputs.phantom_batch(g, 8, 4, 11, device="cuda")
    y = P.forward(x)
    ref = np.stack([O.forward(g, x[b].double().cpu().numpy().reshape(-1)) for b in range(8)])
    scale = np.abs(ref).max()
    np.testing.assert_allclose(y.double().cpu().numpy().reshape(8, -1), ref, rtol=0, atol=1e-4 * scale)
    # the second call reads the cache: same choice, nothing timed
    with open(cache) as fh:
        stored = json.load(fh)
    assert len(stored) == 1
    P2 = X.Projector(g)
    again = tune.tune_projector(P2, 8, cache_path=cache)
    assert again == best and P2.tuning()["path"] == best["path"]
    P.close()
    P2.close()
