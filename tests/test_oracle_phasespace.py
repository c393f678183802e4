"""Pins of the oracle's phase-space generators (thesis Sec. "Phase space
generation from particle collisions"): conservation, on-shell masses and
phase-space volumes known in closed form or by quadrature of the Dalitz area."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


def mass2(p):
    return p[..., 0] ** 2 - p[..., 1] ** 2 - p[..., 2] ** 2 - p[..., 3] ** 2


def dalitz_volume(rs, m1, m2, m3):
    """Three-body phase-space volume: int dm12^2 dm23^2 / (128 pi^3 s)."""
    s = rs * rs

    def width(m12sq):
        m12 = math.sqrt(m12sq)
        e2 = (m12sq - m1 * m1 + m2 * m2) / (2 * m12)
        e3 = (s - m12sq - m3 * m3) / (2 * m12)
        p2 = math.sqrt(max(e2 * e2 - m2 * m2, 0.0))
        p3 = math.sqrt(max(e3 * e3 - m3 * m3, 0.0))
        return 4 * p2 * p3  # m23^2_max - m23^2_min

    a, b = (m1 + m2) ** 2, (rs - m3) ** 2
    area, _ = integrate.quad(width, a, b, epsabs=0, epsrel=1e-12, limit=200)
    return area / (128 * math.pi ** 3 * s)


def test_two_body_kinematics_and_volume():
    rs, m = 500.0, 173.0
    for c, phi in [(-0.9, 0.1), (0.0, 3.0), (0.7, 5.5)]:
        p, w = O.two_body(rs, m, m, c, phi)
        np.testing.assert_allclose(p.sum(axis=0), [rs, 0, 0, 0], atol=1e-12 * rs)
        np.testing.assert_allclose(mass2(p), m * m, rtol=1e-12)
        beta = math.sqrt(1 - 4 * m * m / rs ** 2)
        assert abs(w - beta / (8 * math.pi)) < 1e-15
    _, w0 = O.two_body(91.0, 0.0, 0.0, 0.3, 1.0)
    assert abs(w0 - 1 / (8 * math.pi)) < 1e-16


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_rambo_massless_conservation_and_flat_weight(n):
    rs = 1000.0
    rng = np.random.default_rng(n)
    for _ in range(20):
        p, w, rc = O.rambo(np.zeros(n), rs, rng.uniform(size=4 * n))
        assert rc == 0
        np.testing.assert_allclose(p.sum(axis=0), [rs, 0, 0, 0], atol=1e-12 * rs)
        np.testing.assert_allclose(mass2(p), 0.0, atol=1e-9 * rs * rs)
        sij = sum(2 * (p[i, 0] * p[j, 0] - p[i, 1:] @ p[j, 1:]) for i in range(n) for j in range(i + 1, n))
        assert abs(sij - rs * rs) < 1e-10 * rs * rs
        if n == 2:
            assert abs(w - 1 / (8 * math.pi)) < 1e-16
        if n == 3:  # massless Dalitz area s^2/2
            assert abs(w - rs ** 2 / (256 * math.pi ** 3)) < 1e-12 * w


def test_rambo_massive_two_body_is_exact_volume():
    rs, m = 600.0, 173.0
    beta = math.sqrt(1 - 4 * m * m / rs ** 2)
    rng = np.random.default_rng(5)
    for _ in range(20):
        p, w, rc = O.rambo([m, m], rs, rng.uniform(size=8))
        assert rc == 0
        np.testing.assert_allclose(p.sum(axis=0), [rs, 0, 0, 0], atol=1e-12 * rs)
        np.testing.assert_allclose(mass2(p), m * m, rtol=1e-11)
        assert abs(w - beta / (8 * math.pi)) < 1e-13 * w


def test_massive_three_body_volume_three_ways():
    rs, m = 1000.0, 173.0
    masses = [m, m, 0.0]
    exact = dalitz_volume(rs, *masses)
    rng = np.random.default_rng(7)
    n = 40000
    wr = np.empty(n)
    wh = np.empty(n)
    for i in range(n):
        p, wr[i], rc = O.rambo(masses, rs, rng.uniform(size=12))
        assert rc == 0
        if i < 200:
            np.testing.assert_allclose(p.sum(axis=0), [rs, 0, 0, 0], atol=1e-12 * rs)
            np.testing.assert_allclose(mass2(p), [m * m, m * m, 0.0], atol=1e-9 * rs * rs)
        ph, wh[i], rc = O.hierarchical(masses, rs, rng.uniform(size=5))
        assert rc == 0
        if i < 200:
            np.testing.assert_allclose(ph.sum(axis=0), [rs, 0, 0, 0], atol=1e-12 * rs)
            np.testing.assert_allclose(mass2(ph), [m * m, m * m, 0.0], atol=1e-9 * rs * rs)
    for w in (wr, wh):
        err = w.std() / math.sqrt(n)
        assert abs(w.mean() - exact) < 4 * err, (w.mean(), exact, err)


@pytest.mark.parametrize("n", [2, 3])
def test_hierarchical_massless_volume(n):
    rs = 1000.0
    rng = np.random.default_rng(11)
    exact = 1 / (8 * math.pi) if n == 2 else rs ** 2 / (256 * math.pi ** 3)
    ws = np.array([O.hierarchical(np.zeros(n), rs, rng.uniform(size=3 * n - 4))[1] for _ in range(20000)])
    if n == 2:
        np.testing.assert_allclose(ws, exact, rtol=1e-14)
    else:
        assert abs(ws.mean() - exact) < 4 * ws.std() / math.sqrt(ws.size)
