"""Pins of the closed-form p p -> t tbar quadrature (oracle/hadronic.py).

* The partonic totals are the integrals of the oracle's helicity |M|^2 over
  the angles (tests/test_oracle_me.py checks the same functions that way).
* The convolution geometry (the (L, y) variables, the knot breakpoints, the
  threshold substitution) is pinned on grids whose interpolant is known in
  closed form: x f linear in ln x times a factor linear in ln Q^2, which the
  Hermite interpolation reproduces exactly, so sigma is a plain double
  integral that scipy evaluates without any of that machinery.
* The per-cell cubic recovered from four evaluations reproduces the oracle's
  interpolation elsewhere in the cell (which is what makes it exact).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from oracle import hadronic as H
from paper_2302_03343_b300 import workloads as W

AS, MT, RS = 0.118, 173.0, 13000.0


def linear_grid(coef, cq=0.05):
    """x f = (A + B ln x) (1 + cq ln(Q^2 / Q0^2)) per flavour (coef[pid] = (A, B))."""
    g = W.synthetic_pdf_grid(0)
    lx = np.log(g.x)
    lq = np.log(g.q ** 2 / g.q[0] ** 2)
    xf = np.empty_like(g.xf)
    for k, pid in enumerate(g.pids):
        A, B = coef[int(pid)]
        xf[:, :, k] = (A + B * lx)[:, None] * (1.0 + cq * lq)[None, :]
    return W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=xf, params=g.params), 1.0 + cq * math.log(MT ** 2 / g.q[0] ** 2)


def direct(coef, K):
    """sigma by scipy: int dL int_L^0 da xf_a(a) xf_b(L - a) sigma_ab(e^L s)."""
    s = RS * RS
    L0 = math.log(4 * MT * MT / s)

    def lum(L, a, b):
        (Aa, Ba), (Ab, Bb) = coef[a], coef[b]
        val, _ = integrate.quad(lambda t: (Aa + Ba * t) * (Ab + Bb * (L - t)), L, 0.0, epsabs=0, epsrel=1e-13)
        return K * K * val

    def f(L):
        g = lum(L, 21, 21) * H.sigma_hat_gg(AS, MT, math.exp(L) * s)
        q = sum(lum(L, qf, -qf) + lum(L, -qf, qf) for qf in range(1, 6)) * H.sigma_hat_qqbar(AS, MT, math.exp(L) * s)
        return g + q

    # the threshold behaves like sqrt(L - L0): integrate in u = sqrt(L - L0)
    val, _ = integrate.quad(lambda u: f(L0 + u * u) * 2 * u, 0.0, math.sqrt(-L0), epsabs=0, epsrel=1e-12,
                            limit=200)
    return val


@pytest.mark.parametrize("coef", [
    {p: (1.5, 0.0) for p in W.PIDS},                                              # constant
    {p: (2.0 + 0.1 * abs(p) / 21, 0.08 + 0.01 * (p % 3)) for p in W.PIDS},       # linear in ln x, per flavour
])
def test_quadrature_against_direct_integration(coef):
    g, K = linear_grid(coef)
    pdf = O.Pdf(g)
    r = H.pp_ttbar_sigma(pdf, g, AS, MT, MT, RS)
    ref = direct(coef, K)
    assert abs(r["sigma_pb"] - ref) < 1e-9 * ref
    assert abs(r["gg_pb"] + r["qqbar_pb"] - r["sigma_pb"]) < 1e-12 * r["sigma_pb"]


def test_cell_cubics_reproduce_the_interpolation(oracle_pdf, pdf_grid):
    t, _ = H._uniform_log_knots(pdf_grid.x)
    rng = np.random.default_rng(0)
    for pid in (21, 2, -1):
        c = H.CellCubics(oracle_pdf, pid, t, MT * MT)
        tt = rng.uniform(t[0], t[-1], 200)
        v = np.array([oracle_pdf.xfxq2(pid, math.exp(x), MT * MT) for x in tt])
        assert np.max(np.abs(c(tt) - v) / np.abs(v)) < 1e-12


def test_partonic_totals_vanish_below_threshold():
    s = (2 * MT) ** 2 * (1 - 1e-12)
    assert H.sigma_hat_gg(AS, MT, s) == 0.0 and H.sigma_hat_qqbar(AS, MT, s) == 0.0
    # just above threshold both grow like beta: sigma(s) / beta -> constant
    r = []
    for eps in (1e-6, 1e-8):
        s = (2 * MT) ** 2 / (1 - eps)
        beta = math.sqrt(eps)
        r.append((H.sigma_hat_gg(AS, MT, s) / beta, H.sigma_hat_qqbar(AS, MT, s) / beta))
    assert abs(r[0][0] / r[1][0] - 1) < 1e-5 and abs(r[0][1] / r[1][1] - 1) < 1e-5
