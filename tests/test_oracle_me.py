"""Pins of the oracle's squared matrix elements (thesis Sec. "The MadFlow
event generator": helicity amplitudes, colour decomposition, fig. pp_ttx).

Closed forms (textbook) are checked against explicit numerical Dirac traces
and against the textbook total partonic cross sections; gg -> ttg (no closed
form) is pinned by two independent formulations, gauge invariance, the soft
gluon limit of its colour-ordered amplitudes, C and Lorentz invariance, and
its two-gluon analogue reproducing the gg -> tt closed form.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from oracle import hadronic as H

AS, MT = 0.118, 173.0
EW = dict(alpha=1 / 128, mz=91.1876, gz=2.4952, sw2=0.2312)
GEV2PB = 0.3893794e9


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def two_to_two(rs, m, c, phi):
    p, _ = O.two_body(rs, m, m, c, phi)
    e = rs / 2
    return np.array([[e, 0, 0, e], [e, 0, 0, -e], p[0], p[1]])


def ggttg_point(rs, u):
    p, w, rc = O.rambo([MT, MT, 0.0], rs, u)
    assert rc == 0
    e = rs / 2
    return np.array([[e, 0, 0, e], [e, 0, 0, -e], p[0], p[1], p[2]])


# ---------------------------------------------------------------- e+e- -> mu+mu-
def test_eemumu_closed_form_vs_trace():
    for rs in (30.0, 91.0, 91.1876, 500.0):
        for c in (-0.95, -0.2, 0.4, 0.99):
            p, _ = O.two_body(rs, 0, 0, c, 0.7)
            e = rs / 2
            P = np.array([[e, 0, 0, e], [e, 0, 0, -e], p[0], p[1]])
            a = O.me2_eemumu(EW["alpha"], EW["mz"], EW["gz"], EW["sw2"], rs * rs, c)
            b = O.me2_eemumu_trace(EW["alpha"], EW["mz"], EW["gz"], EW["sw2"], P)
            assert abs(a - b) < 1e-12 * abs(a)


def test_eemumu_total_and_qed_limit():
    def sigma(rs, mz):
        s = rs * rs
        f = lambda c: O.me2_eemumu(EW["alpha"], mz, EW["gz"], EW["sw2"], s, c)
        val, _ = integrate.quad(f, -1, 1, epsrel=1e-13)
        return val * 2 * math.pi / (64 * math.pi ** 2 * s) * GEV2PB

    # with the Z decoupled the total is the QED 4 pi alpha^2 / (3 s)
    rs = 10.0
    qed = 4 * math.pi * EW["alpha"] ** 2 / (3 * rs * rs) * GEV2PB
    assert abs(sigma(rs, 1e9) - qed) < 1e-10 * qed
    # the A1 (forward-backward) term integrates to zero: sigma = 4 pi alpha^2 A0 / (3 s)
    s = 91.0 ** 2
    a0 = O.me2_eemumu(EW["alpha"], EW["mz"], EW["gz"], EW["sw2"], s, 0.0) / (4 * math.pi * EW["alpha"]) ** 2
    expect = 4 * math.pi * EW["alpha"] ** 2 * a0 / (3 * s) * GEV2PB
    assert abs(sigma(91.0, EW["mz"]) - expect) < 1e-10 * expect


# ---------------------------------------------------------------- t tbar
@pytest.mark.parametrize("rs", [360.0, 500.0, 1000.0, 4000.0])
def test_ttbar_closed_forms_vs_numerical(rs):
    s = rs * rs
    for c in (-0.9, 0.0, 0.35, 0.97):
        P = two_to_two(rs, MT, c, 1.1)
        d = P[0] - P[2]
        t = mdot(d, d)
        qq = O.me2_qqbar_ttbar(AS, MT, s, t)
        assert abs(qq - O.me2_qqbar_ttbar_trace(AS, MT, P)) < 1e-12 * qq
        gg = O.me2_gg_ttbar(AS, MT, s, t)
        assert abs(gg - O.me2_gg_ttbar_colour_ordered(AS, MT, P)) < 1e-12 * gg


@pytest.mark.parametrize("rs", [400.0, 500.0, 1000.0])
def test_ttbar_partonic_totals(rs):
    s = rs * rs
    rho = 4 * MT * MT / s
    beta = math.sqrt(1 - rho)

    def sig(me):
        def f(c):
            t = MT * MT - s / 2 * (1 - beta * c)
            return me(AS, MT, s, t)
        val, _ = integrate.quad(f, -1, 1, epsrel=1e-13)
        return val * 2 * math.pi * beta / (64 * math.pi ** 2 * s) * GEV2PB

    # the textbook totals used by the closed-form hadronic cross section
    qq_exact = H.sigma_hat_qqbar(AS, MT, s, GEV2PB)
    gg_exact = H.sigma_hat_gg(AS, MT, s, GEV2PB)
    assert abs(sig(O.me2_qqbar_ttbar) - qq_exact) < 1e-10 * qq_exact
    assert abs(sig(O.me2_gg_ttbar) - gg_exact) < 1e-10 * gg_exact


# ---------------------------------------------------------------- g g -> t tbar g
POINTS = [(1000.0, [0.3, 0.6, 0.2, 0.5, 0.7, 0.1, 0.4, 0.8, 0.55, 0.35, 0.65, 0.25]),
          (2500.0, [0.9, 0.15, 0.33, 0.77, 0.05, 0.62, 0.48, 0.21, 0.4, 0.9, 0.3, 0.6]),
          (13000.0, [0.5, 0.5, 0.1, 0.2, 0.8, 0.3, 0.7, 0.6, 0.2, 0.45, 0.9, 0.8])]


@pytest.mark.parametrize("rs,u", POINTS)
def test_ggttg_two_formulations_agree(rs, u):
    P = ggttg_point(rs, np.array(u))
    a = O.me2_gg_ttbarg(AS, MT, P)
    b = O.me2_gg_ttbarg_brute(AS, MT, P)
    assert abs(a - b) < 1e-12 * abs(a)


def test_ggttg_symmetries():
    rng = np.random.default_rng(3)
    for _ in range(5):
        P = ggttg_point(1500.0, rng.uniform(size=12))
        ref = O.me2_gg_ttbarg(AS, MT, P)
        # Bose symmetry of the incoming gluons
        assert abs(O.me2_gg_ttbarg(AS, MT, P[[1, 0, 2, 3, 4]]) - ref) < 1e-12 * ref
        # charge conjugation: top <-> anti-top momenta
        assert abs(O.me2_gg_ttbarg(AS, MT, P[[0, 1, 3, 2, 4]]) - ref) < 1e-11 * ref
        # rotation and boost invariance
        th = rng.uniform(0, math.pi)
        R = np.array([[1, 0, 0, 0], [0, math.cos(th), 0, math.sin(th)], [0, 0, 1, 0],
                      [0, -math.sin(th), 0, math.cos(th)]])
        assert abs(O.me2_gg_ttbarg(AS, MT, P @ R.T) - ref) < 1e-11 * ref
        y = 0.7
        B = np.array([[math.cosh(y), 0, 0, math.sinh(y)], [0, 1, 0, 0], [0, 0, 1, 0],
                      [math.sinh(y), 0, 0, math.cosh(y)]])
        assert abs(O.me2_gg_ttbarg(AS, MT, P @ B.T) - ref) < 1e-10 * ref


# Dirac representation, used only to build external spinors for the
# amplitude-level pins: u = (pslash + m) xi and v = (pslash - m) eta solve the
# Dirac equation for any xi, eta.
_G0 = np.diag([1, 1, -1, -1]).astype(complex)
_SIG = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]
_GK = [np.block([[np.zeros((2, 2)), s], [-s, np.zeros((2, 2))]]) for s in _SIG]


def slash(p):
    return _G0 * p[0] - sum(_GK[k] * p[k + 1] for k in range(3))


def spinors(p1, p2, m, seed=0):
    rng = np.random.default_rng(seed)
    xi = rng.normal(size=4) + 1j * rng.normal(size=4)
    eta = rng.normal(size=4) + 1j * rng.normal(size=4)
    u = (slash(p1) + m * np.eye(4)) @ xi
    v = (slash(p2) - m * np.eye(4)) @ eta
    return u.conj() @ _G0, v


def pol(k, which):
    n = np.array(k[1:]) / np.linalg.norm(k[1:])
    a = np.cross(n, [0, 0, 1.0])
    a = a / np.linalg.norm(a) if np.linalg.norm(a) > 1e-6 else np.array([1.0, 0, 0])
    b = np.cross(n, a)
    e = a if which == 0 else b
    return np.array([0, *e], dtype=complex)


def test_ggttg_partial_amplitudes_gauge_invariant():
    rng = np.random.default_rng(5)
    for _ in range(4):
        P = ggttg_point(2000.0, rng.uniform(size=12))
        q = np.array([P[0], P[1], -P[4], P[2]])
        ubar, v = spinors(P[2], P[3], MT)
        eps = [pol(P[0], 0), pol(P[1], 1), pol(P[4], 0)]
        ref = np.max(np.abs(O.ggttg_partial_amplitudes(AS, MT, q, eps, ubar, v)))
        for i in range(3):
            e2 = list(eps)
            e2[i] = q[i].astype(complex)
            amps = O.ggttg_partial_amplitudes(AS, MT, q, e2, ubar, v)
            assert np.max(np.abs(amps)) < 1e-10 * ref * np.abs(q[i][0]), (i, amps, ref)
        # the two-gluon amplitudes too
        q2 = np.array([P[0], P[1], P[2]])
        P4 = two_to_two(2000.0, MT, 0.3, 0.4)
        q2 = np.array([P4[0], P4[1], P4[2]])
        ub2, v2 = spinors(P4[2], P4[3], MT)
        e = [pol(P4[0], 0), pol(P4[1], 0)]
        ref2 = np.max(np.abs(O.ggttg_partial_amplitudes(AS, MT, q2, e, ub2, v2)))
        a2 = O.ggttg_partial_amplitudes(AS, MT, q2, [q2[0].astype(complex), e[1]], ub2, v2)
        assert np.max(np.abs(a2)) < 1e-10 * ref2 * q2[0][0]


def _soft_point(lam):
    rs = 800.0
    P4 = two_to_two(rs, MT, 0.4, 0.9)
    n = np.array([0.3, -0.5, 0.81])
    n /= np.linalg.norm(n)
    k = lam * rs / 2 * np.array([1.0, *n])
    Q = P4[0] + P4[1] - k
    M = math.sqrt(mdot(Q, Q))
    # decay Q -> t tbar along the 4-point top direction, then boost to the lab
    d = P4[2][1:] / np.linalg.norm(P4[2][1:])
    pa = math.sqrt(M * M / 4 - MT * MT)
    rest = [np.array([M / 2, *(pa * d)]), np.array([M / 2, *(-pa * d)])]
    out = []
    for r in rest:
        e = (Q[0] * r[0] + Q[1:] @ r[1:]) / M
        f = (r[0] + e) / (Q[0] + M)
        out.append(np.array([e, *(r[1:] + f * Q[1:])]))
    return P4, np.array([P4[0], P4[1], out[0], out[1], k])


def test_ggttg_soft_gluon_limit_of_colour_ordered_amplitudes():
    g = math.sqrt(4 * math.pi * AS)
    orders3 = list(itertools.permutations(range(3)))
    orders2 = list(itertools.permutations(range(2)))
    devs = []
    for lam in (1e-4, 1e-5):
        P4, P5 = _soft_point(lam)
        ubar4, v4 = spinors(P4[2], P4[3], MT, seed=1)
        ubar5, v5 = spinors(P5[2], P5[3], MT, seed=1)
        eps = [pol(P4[0], 0), pol(P4[1], 1), pol(P5[4], 1)]
        qs = -P5[4]
        a2 = O.ggttg_partial_amplitudes(AS, MT, np.array([P4[0], P4[1], P4[2]]), eps[:2], ubar4, v4)
        a3 = O.ggttg_partial_amplitudes(AS, MT, np.array([P5[0], P5[1], qs, P5[2]]), eps, ubar5, v5)
        mom = {0: P4[0], 1: P4[1], "t": P4[2], "tb": P4[3]}
        worst = 0.0
        for si, s in enumerate(orders3):
            pos = s.index(2)
            left = "t" if pos == 0 else s[pos - 1]
            right = "tb" if pos == 2 else s[pos + 1]
            eik = g * (mdot(eps[2], mom[left]) / mdot(qs, mom[left]) - mdot(eps[2], mom[right]) / mdot(qs, mom[right]))
            red = tuple(x for x in s if x != 2)
            expect = eik * a2[orders2.index(red)]
            worst = max(worst, abs(a3[si] / expect - 1))
        devs.append(worst)
    assert devs[1] < 1e-3, devs
    assert devs[1] < devs[0] / 3, devs  # deviation falls with the gluon energy


def _helicity_spinors(p, m, lam):
    """Massive helicity spinors u(p, lam), v(p, lam) in the Dirac representation."""
    pa = np.linalg.norm(p[1:])
    n = p[1:] / pa
    th, ph = math.acos(max(-1.0, min(1.0, n[2]))), math.atan2(n[1], n[0])
    def chi(l):
        return (np.array([math.cos(th / 2), np.exp(1j * ph) * math.sin(th / 2)]) if l > 0
                else np.array([-np.exp(-1j * ph) * math.sin(th / 2), math.cos(th / 2)]))
    e = p[0]
    u = np.concatenate([math.sqrt(e + m) * chi(lam), lam * pa / math.sqrt(e + m) * chi(lam)])
    v = np.concatenate([-lam * pa / math.sqrt(e + m) * chi(-lam), math.sqrt(e + m) * chi(-lam)])
    return u, v


def test_ggttg_spin_flip_symmetry():
    # With real momenta and real polarisation vectors, flipping both fermion
    # helicities conjugates every colour-ordered amplitude up to one common
    # phase, so the colour-summed square is unchanged (used by the CUDA path
    # to evaluate half of the fermion spin sum).
    rng = np.random.default_rng(9)
    for _ in range(3):
        P = ggttg_point(1800.0, rng.uniform(size=12))
        q = np.array([P[0], P[1], -P[4], P[2]])
        for h in itertools.product(range(2), repeat=3):
            eps = [pol(P[0], h[0]), pol(P[1], h[1]), pol(P[4], h[2])]
            for s, sb in ((1, 1), (1, -1)):
                u1, _ = _helicity_spinors(P[2], MT, s)
                _, v1 = _helicity_spinors(P[3], MT, sb)
                u2, _ = _helicity_spinors(P[2], MT, -s)
                _, v2 = _helicity_spinors(P[3], MT, -sb)
                a = O.ggttg_partial_amplitudes(AS, MT, q, eps, u1.conj() @ _G0, v1)
                b = O.ggttg_partial_amplitudes(AS, MT, q, eps, u2.conj() @ _G0, v2)
                ratio = b / np.conj(a)
                assert np.max(np.abs(ratio - ratio[0])) < 1e-10 * np.abs(ratio[0])
                assert abs(abs(ratio[0]) - 1.0) < 1e-10


# ---------------------------------------------------------------- q qbar -> t tbar g, q g -> t tbar q
def test_qqbar_ttbarg_gauge_invariance_and_symmetries():
    """The five diagrams of q qbar -> t tbar g: replacing the gluon
    polarisation by its momentum gives zero (the relative factors of the
    diagrams, including the three-gluon one with its complex colour factor,
    are fixed by this); charge conjugation (q <-> qbar with t <-> tbar);
    rotation and boost invariance; the crossed q g -> t tbar q is gauge
    invariant in its incoming gluon and positive."""
    rng = np.random.default_rng(21)
    for rs in (420.0, 900.0, 4000.0):
        for _ in range(4):
            P = ggttg_point(rs, rng.uniform(size=12))
            ref = O.me2_qqbar_ttbarg(AS, MT, P)
            assert ref > 0
            eg = P[4][0]
            assert abs(O.me2_qqbar_ttbarg_eps(AS, MT, P, P[4].astype(complex))) < 1e-12 * ref * eg ** 2
            assert abs(O.me2_qqbar_ttbarg(AS, MT, P[[1, 0, 3, 2, 4]]) / ref - 1) < 1e-12
            th = rng.uniform(0, math.pi)
            R = np.array([[1, 0, 0, 0], [0, math.cos(th), 0, math.sin(th)], [0, 0, 1, 0],
                          [0, -math.sin(th), 0, math.cos(th)]])
            assert abs(O.me2_qqbar_ttbarg(AS, MT, P @ R.T) / ref - 1) < 1e-11
            y = -0.9
            B = np.array([[math.cosh(y), 0, 0, math.sinh(y)], [0, 1, 0, 0], [0, 0, 1, 0],
                          [math.sinh(y), 0, 0, math.cosh(y)]])
            assert abs(O.me2_qqbar_ttbarg(AS, MT, P @ B.T) / ref - 1) < 1e-10
            # q(p0) g(p1) -> t t~ q(p4): positive, and gauge invariant in the
            # incoming gluon (the crossed momenta of q qbar -> t t~ g)
            qg = O.me2_qg_ttbarq(AS, MT, P)
            assert qg > 0
            crossed = np.array([P[0], -P[4], P[2], P[3], -P[1]])
            gauge = O.me2_qqbar_ttbarg_eps(AS, MT, crossed, (-P[1]).astype(complex))
            assert abs(gauge) < 1e-12 * qg * P[1][0] ** 2


def test_qqbar_ttbarg_soft_gluon_scaling():
    """A soft gluon radiates like dE/E: |M|^2 grows as 1/E_g^2 when the gluon
    momentum is scaled down (the tops keep the rest of the energy)."""
    rng = np.random.default_rng(22)
    rs = 800.0
    P = ggttg_point(rs, rng.uniform(size=12))
    k = P[4] / P[4][0]  # unit-energy gluon direction
    vals = []
    for lam in (1e-2, 1e-3, 1e-4):
        eg = lam * rs / 4
        # the tops share sqrt(s) - E_g back to back against the gluon in their pair frame:
        # generate them as a two-body decay of Q = P - k eg
        q = np.array([rs, 0, 0, 0]) - k * eg
        mq = math.sqrt(mdot(q, q))
        pt_rest, _ = O.two_body(mq, MT, MT, 0.3, 1.1)
        bq = q[1:] / q[0]
        g = 1 / math.sqrt(1 - bq @ bq)

        def boost(v):
            bp = bq @ v[1:]
            e = g * (v[0] + bp)
            return np.array([e, *(v[1:] + ((g - 1) * bp / (bq @ bq) + g * v[0]) * bq)])
        pts = [boost(pt_rest[0]), boost(pt_rest[1])]
        Pl = np.array([P[0], P[1], pts[0], pts[1], k * eg])
        assert np.allclose(Pl[2] + Pl[3] + Pl[4], [rs, 0, 0, 0], atol=1e-9 * rs)
        vals.append(O.me2_qqbar_ttbarg(AS, MT, Pl) * eg ** 2)
    assert abs(vals[2] / vals[1] - 1) < 1e-2 and abs(vals[1] / vals[0] - 1) < 1e-1


# ------------------------------------------------- formulation C and op counts
@pytest.mark.parametrize("rs,u", POINTS)
def test_ggttg_helicity_formulation_agrees(rs, u):
    """Formulation C (helicity amplitudes on spinors, one antitop spin doubled)
    equals formulation A (Dirac traces, every spin) and B (Feynman diagrams at
    explicit colours)."""
    P = ggttg_point(rs, np.array(u))
    a = O.me2_gg_ttbarg(AS, MT, P)
    c = O.me2_gg_ttbarg_helicity(AS, MT, P)
    b = O.me2_gg_ttbarg_brute(AS, MT, P)
    assert abs(c - a) < 1e-12 * abs(a)
    assert abs(c - b) < 1e-12 * abs(b)


def test_ggttg_helicity_formulation_random_points():
    rng = np.random.default_rng(7)
    for _ in range(20):
        rs = rng.uniform(400.0, 6000.0)
        P = ggttg_point(rs, rng.uniform(0.02, 0.98, 12))
        a = O.me2_gg_ttbarg(AS, MT, P)
        assert abs(O.me2_gg_ttbarg_helicity(AS, MT, P) - a) < 1e-12 * abs(a)


def test_operation_counts_of_the_event():
    """The counting harness runs the oracle's own arithmetic (its weights sum
    to orc_iterate's over the same events), the |M|^2 count is the same for
    every event, and the VEGAS map costs what its formula says:
    r = (2m + 1) 2^-(b+1) (1 multiplication), w = hi - lo, x = lo + r w,
    J *= N_b w: 6 operations per dimension."""
    from paper_2302_03343_b300 import workloads as W
    pdf = O.Pdf(W.synthetic_pdf_grid(0))
    itg = W.gg_ttbarg()
    edges = O.vegas_refine(W.uniform_grid(14, 50), np.random.default_rng(3).exponential(size=(14, 50)) ** 2, 1.0)
    per_event = []
    for first in (0, 5000):
        r = O.count_gg_ttbarg(itg, pdf, edges, 1, 4, 2, 0, first, 2000)
        it = O.iterate(itg, pdf, edges, 1, 4, 2, 0, first, 2000, nthreads=1)
        assert r["in_cuts"] == it["n_nonzero"] > 0
        assert abs(r["sum_w"] - it["sum"]) <= 1e-12 * abs(it["sum"])
        me = r["me2"]
        flop = me["add"] + me["mul"] + me["div"] + me["sqrt"]
        assert flop % r["in_cuts"] == 0
        per_event.append(flop // r["in_cuts"])
        m = r["map"]
        assert (m["add"], m["mul"], m["div"], m["sqrt"], m["fn"]) == (2 * 14 * 2000, 4 * 14 * 2000, 0, 0, 0)
    assert per_event[0] == per_event[1] > 0
