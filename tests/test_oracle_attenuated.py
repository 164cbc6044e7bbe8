"""Pins of the oracle's attenuated transform (eq. generalizedRadontransform with the
exponential attenuation weight): no attenuation gives the plain transform, a uniform
attenuation over the image gives a closed form in the chord length, and a dense quadrature of
the defining integral along the ray built from the scan layout agrees.  CPU only."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import oracle as O
from paper_2006_00686_gb300.inputs import Geometry
from tests.test_oracle_brute import _rand_geom, _ray_list

pi = math.pi
KINDS = ["par2d", "fan2d", "fan2d_arc", "par3d", "cone", "cone_arc", "helix", "helix_arc"]


@pytest.mark.parametrize("kind", KINDS)
def test_zero_attenuation_is_the_plain_transform(kind):
    g = _rand_geom(kind, np.random.default_rng(3))
    f = np.random.default_rng(4).random(g.n_units)
    # the same terms, summed along the ray instead of by unit index
    np.testing.assert_allclose(O.forward_attenuated(g, np.zeros(g.n_units), f), O.forward(g, f), rtol=1e-14,
                               atol=1e-14)


@pytest.mark.parametrize("kind", KINDS + ["rays2d", "rays3d"])
def test_uniform_attenuation_closed_form(kind):
    # f = 1 and mu = c on the whole image: g = int_0^L exp(-c (L - t)) dt = (1 - exp(-c L)) / c
    rng = np.random.default_rng(5)
    g = _ray_list(kind, rng) if kind.startswith("rays") else _rand_geom(kind, rng)
    c = 0.37
    got = O.forward_attenuated(g, np.full(g.n_units, c), np.ones(g.n_units))
    for r in range(g.n_rays):
        p, d = B.ray_of(g, r)
        L = B.box_chord(g, p, d)
        assert got[r] == pytest.approx(-math.expm1(-c * L) / c, rel=1e-12, abs=1e-12)


def _quadrature(g, f, mu, p, d, h=2e-4):
    """int f(p + t d) exp(-int_t^inf mu(p + s d) ds) dt by the midpoint rule over the chord."""
    lo = np.array([g.cx - g.nx * g.dx / 2, g.cy - g.ny * g.dy / 2, g.cz - g.nz * g.dz / 2])
    hi = lo + np.array([g.nx * g.dx, g.ny * g.dy, g.nz * g.dz])
    three = g.nz > 1 or g.kind in ("par3d", "cone", "cone_arc", "helix", "helix_arc", "rays3d")
    t0, t1 = -np.inf, np.inf
    for a in range(3 if three else 2):
        if d[a] != 0.0:
            ta, tb = (lo[a] - p[a]) / d[a], (hi[a] - p[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
        elif not (lo[a] <= p[a] <= hi[a]):
            return 0.0
    if not t0 < t1:
        return 0.0
    n = int(math.ceil((t1 - t0) / h))
    t = t0 + (np.arange(n) + 0.5) * (t1 - t0) / n
    x = p[None, :] + t[:, None] * d[None, :]
    i = np.clip(np.floor((x[:, 0] - lo[0]) / g.dx).astype(int), 0, g.nx - 1)
    j = np.clip(np.floor((hi[1] - x[:, 1]) / g.dy).astype(int), 0, g.ny - 1)
    k = np.clip(np.floor((hi[2] - x[:, 2]) / g.dz).astype(int), 0, g.nz - 1) if three else np.zeros(n, int)
    I = (k * g.ny + j) * g.nx + i
    dt = (t1 - t0) / n
    m = mu[I] * dt
    after = np.cumsum(m[::-1])[::-1] - 0.5 * m  # attenuation from each sample to the far end
    return float(np.sum(f[I] * np.exp(-after)) * dt)


@pytest.mark.parametrize("kind", ["par2d", "fan2d", "cone", "helix", "rays2d", "rays3d"])
def test_attenuated_vs_dense_quadrature(kind):
    rng = np.random.default_rng(11)
    g = _ray_list(kind, rng, n=12) if kind.startswith("rays") else _rand_geom(kind, rng)
    f = rng.random(g.n_units)
    mu = 0.5 * rng.random(g.n_units)
    got = O.forward_attenuated(g, mu, f)
    for r in range(min(g.n_rays, 40)):
        p, d = B.ray_of(g, r)
        want = _quadrature(g, f, mu, p, d)
        assert got[r] == pytest.approx(want, rel=2e-3, abs=2e-3)


@pytest.mark.parametrize("kind", ["fan2d", "cone"])
def test_attenuated_adjoint_dot_test(kind):
    rng = np.random.default_rng(13)
    g = _rand_geom(kind, rng)
    mu = 0.3 * rng.random(g.n_units)
    x = rng.random(g.n_units)
    y = rng.random(g.n_rays)
    lhs = float(O.forward_attenuated(g, mu, x) @ y)
    rhs = float(x @ O.adjoint_attenuated(g, mu, y))
    assert lhs == pytest.approx(rhs, rel=1e-12)
