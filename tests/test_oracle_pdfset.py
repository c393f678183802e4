"""Pins of the oracle's PDF-set interpolation, extrapolation and alpha_s
(oracle/src/pdfset.cpp; thesis Sec. "LHAPDF: the Les Houches Accord PDF").

Each check compares with something the oracle does not compute the same way:
stored nodes, polynomials the interpolant must reproduce exactly, power laws
the continuation rules must reproduce exactly, the two limits of the low-Q
continuation printed in the thesis, and one-loop running alpha_s.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import workloads as W


def custom_set(xs, qs, fn, pids=(21,), nmem=1):
    """A PdfSet whose values are fn(member, s, x, q) on the given sub-grid knots."""
    blocks = []
    for m in range(nmem):
        vals = []
        for s, (x, q) in enumerate(zip(xs, qs)):
            v = np.empty((len(x), len(q), len(pids)))
            for i, xi in enumerate(x):
                for j, qj in enumerate(q):
                    v[i, j, :] = fn(m, s, xi, qj)
            vals.append(v.reshape(-1))
        blocks.append(np.concatenate(vals))
    return W.PdfSet(x=list(xs), q=list(qs), pids=np.array(pids, dtype=np.int32), xf=np.array(blocks),
                    params=np.zeros((nmem, len(pids), 4)))


def logspace(lo, hi, n):
    return np.array([lo * (hi / lo) ** (k / (n - 1)) for k in range(n)])


@pytest.fixture(scope="module")
def pset():
    return W.synthetic_pdf_set(nmem=3, seed=0)


def test_nodes_of_every_subgrid_and_member(pset):
    P = O.PdfSet(pset)
    for m in range(3):
        for s in range(2):
            g = pset.member_subgrid(m, s)
            for i in range(0, len(pset.x[s]), 7):
                # the threshold knot is the upper sub-grid's
                for j in range(len(pset.q[s]) - (1 if s == 0 else 0)):
                    for fl, pid in enumerate(pset.pids):
                        got = P.xfxq2(m, int(pid), pset.x[s][i], pset.q[s][j] ** 2)
                        assert got == g[i, j, fl], (m, s, i, j, pid)
    # at the threshold the b density jumps from 0 (below) to the upper grid's value
    top = pset.member_subgrid(0, 1)[40, 0, list(pset.pids).index(5)]
    assert P.xfxq2(0, 5, pset.x[1][40], W.MB_THRESHOLD ** 2) == top > 0
    assert P.xfxq2(0, 5, pset.x[0][40], (W.MB_THRESHOLD * 0.999) ** 2) < 0.01 * top


def test_quadratics_reproduced_in_interior_cells():
    x = logspace(1e-6, 1.0, 30)
    qs = [logspace(2.0, 8.0, 7), logspace(8.0, 1000.0, 12)]
    c = (0.3, -0.7, 0.2, 0.05, -0.03, 0.011)

    def f(m, s, xi, qj):
        u, v = math.log(xi), math.log(qj * qj)
        return c[0] + c[1] * u + c[2] * v + c[3] * u * u + c[4] * u * v + c[5] * v * v
    P = O.PdfSet(custom_set([x, x], qs, f))
    rng = np.random.default_rng(1)
    for _ in range(200):
        s = int(rng.integers(2))
        ix = int(rng.integers(1, len(x) - 2))
        iq = int(rng.integers(1, len(qs[s]) - 2))
        u = math.log(x[ix]) + rng.random() * (math.log(x[ix + 1]) - math.log(x[ix]))
        v = math.log(qs[s][iq] ** 2) + rng.random() * (math.log(qs[s][iq + 1] ** 2) - math.log(qs[s][iq] ** 2))
        xi, q2 = math.exp(u), math.exp(v)
        exact = f(0, s, xi, math.sqrt(q2))
        assert abs(P.xfxq2(0, 21, xi, q2) - exact) <= 1e-11 * max(1.0, abs(exact))


def test_bilinear_where_a_subgrid_has_three_q_knots():
    x = logspace(1e-5, 1.0, 20)
    qs = [logspace(2.0, 3.0, 3), logspace(3.0, 100.0, 10)]

    def f(m, s, xi, qj):
        u, v = math.log(xi), math.log(qj * qj)
        return 2.0 + 0.4 * u - 0.3 * v + 0.07 * u * v
    P = O.PdfSet(custom_set([x, x], qs, f))
    rng = np.random.default_rng(2)
    for _ in range(100):
        u = math.log(1e-5) + rng.random() * (0.0 - math.log(1e-5))
        v = math.log(4.0) + rng.random() * (math.log(9.0) - math.log(4.0))
        xi, q2 = math.exp(u), math.exp(v)
        assert abs(P.xfxq2(0, 21, xi, q2) - f(0, 0, xi, math.sqrt(q2))) <= 1e-12 * 10


def test_low_x_and_high_q_continuation_of_power_laws():
    x = logspace(1e-5, 1.0, 25)
    qs = [logspace(2.0, 1000.0, 15)]
    A, a, p = 3.0, 0.35, 0.12

    def f(m, s, xi, qj):  # a power law in x and Q^2, far above 1e-3
        return A * xi ** (-a) * (qj * qj) ** p
    P = O.PdfSet(custom_set([x], qs, f))
    # on Q knots (where the Q direction is exact) below x_min, on x knots above Q_max
    for xi in (1e-6, 1e-8, 3e-10):
        for qj in (qs[0][1], qs[0][9]):
            assert abs(P.xfxq2(0, 21, xi, qj * qj) / f(0, 0, xi, qj) - 1.0) < 1e-12
    for q2 in (2e6, 1e9):
        for xi in (x[3], x[20], 1e-7):  # 1e-7: both outside, the x rule feeds the Q rule
            assert abs(P.xfxq2(0, 21, xi, q2) / f(0, 0, xi, math.sqrt(q2)) - 1.0) < 1e-12


def test_low_x_continuation_is_linear_in_log_x_below_threshold():
    x = logspace(1e-5, 1.0, 25)
    qs = [logspace(2.0, 1000.0, 15)]

    def f(m, s, xi, qj):  # below 1e-3 at the lowest knots: linear in ln x
        return 1e-5 * (30.0 + math.log(xi))
    P = O.PdfSet(custom_set([x], qs, f))
    for xi in (1e-6, 1e-9):
        assert abs(P.xfxq2(0, 21, xi, 100.0) - f(0, 0, xi, 10.0)) < 1e-17


def test_low_q_continuation_limits(pset):
    """The two limits the thesis prints: x f -> x f(Q2min) (Q2/Q2min)^gamma as
    Q2 -> Q2min (continuity, log-derivative gamma from the two lowest knots)
    and x f -> x f(Q2min) Q2/Q2min as Q2 -> 0."""
    P = O.PdfSet(pset)
    q2min, q2b = pset.q[0][0] ** 2, pset.q[0][1] ** 2
    for pid in (21, 2, -1):
        for xi in (1e-4, 0.05, 0.4):
            f0 = P.xfxq2(0, pid, xi, q2min)
            f1 = P.xfxq2(0, pid, xi, q2b)
            gamma = math.log(f1 / f0) / math.log(q2b / q2min)
            assert abs(P.xfxq2(0, pid, xi, q2min * (1 - 1e-12)) / f0 - 1.0) < 1e-10
            h = 1e-6
            d = (math.log(P.xfxq2(0, pid, xi, q2min * math.exp(-h))) - math.log(f0)) / (-h)
            assert abs(d - gamma) < 1e-5 * max(1.0, abs(gamma))
            for r in (1e-6, 1e-8):
                assert abs(P.xfxq2(0, pid, xi, q2min * r) / (f0 * r) - 1.0) < 1e-4


def test_outside_x_max_and_bad_input_are_nan(pset):
    P = O.PdfSet(pset)
    assert math.isnan(P.xfxq2(0, 21, 1.5, 100.0))
    assert math.isnan(P.xfxq2(0, 21, -1e-3, 100.0))
    assert math.isnan(P.xfxq2(0, 21, 1e-3, 0.0))
    assert math.isnan(P.xfxq2(0, 7, 1e-3, 100.0))
    assert math.isnan(P.xfxq2(5, 21, 1e-3, 100.0))


def test_members_are_their_own_grids(pset):
    P = O.PdfSet(pset)
    for m in range(3):
        single = W.PdfSet(x=pset.x, q=pset.q, pids=pset.pids, xf=pset.xf[m:m + 1], params=pset.params[m:m + 1])
        Pm = O.PdfSet(single)
        for xi, q2 in ((3e-4, 50.0), (0.2, 1e4), (2e-8, 3.0), (0.01, 1e9)):
            assert P.xfxq2(m, 21, xi, q2) == Pm.xfxq2(0, 21, xi, q2)
    assert P.xfxq2(1, 21, 0.01, 100.0) != P.xfxq2(2, 21, 0.01, 100.0)


def test_alphas_against_one_loop_running():
    q, a = W.synthetic_alphas_knots()
    A = O.AlphaS(q, a)
    for qi, ai in zip(q, a):
        if qi not in (W.MC_THRESHOLD, W.MB_THRESHOLD):
            assert A(qi * qi) == ai
    # at a threshold knot: the upper segment's value
    assert A(W.MB_THRESHOLD ** 2) == a[list(q).index(W.MB_THRESHOLD) + 1]
    # inside the segments: the one-loop formula the knots were drawn from
    b0 = lambda nf: (33.0 - 2.0 * nf) / (12.0 * math.pi)  # noqa: E731
    lam5 = W.MZ ** 2 * math.exp(-1.0 / (b0(5) * W.ALPHAS_MZ))
    for Q in (7.0, 20.0, W.MZ, 500.0, 5000.0):
        exact = 1.0 / (b0(5) * math.log(Q * Q / lam5))
        assert abs(A(Q * Q) / exact - 1.0) < 2e-5, Q
    assert abs(A(W.MZ ** 2) - W.ALPHAS_MZ) < 1e-5
    # above the grid: constant; below: ln alpha_s linear in ln Q^2
    assert A(1e12) == a[-1] == A(q[-1] ** 2)
    slope = math.log(a[1] / a[0]) / math.log(q[1] ** 2 / q[0] ** 2)
    for q2 in (0.5, 0.01):
        assert abs(math.log(A(q2)) - (math.log(a[0]) + slope * math.log(q2 / q[0] ** 2))) < 1e-12


def test_alphas_power_law_continuation_below_the_grid():
    q = logspace(1.0, 100.0, 10)
    a = 0.3 * (q * q) ** -0.2
    A = O.AlphaS(q, a)
    for q2 in (0.1, 0.001):
        assert abs(A(q2) / (0.3 * q2 ** -0.2) - 1.0) < 1e-12
