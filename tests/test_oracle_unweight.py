"""Pins of the oracle's unweighting (oracle/src/unweight.cpp; thesis Sec.
"Unweighted event exporter"): an event of weight w survives with probability
w / w_max, and the surviving events follow the weighted distribution."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import workloads as W


def test_acceptance_uniforms_are_uniform_and_distinct_from_the_event_stream():
    r = O.acceptance_uniforms(seed=3, iteration=1, gid=2, first=0, n=200000)
    assert r.min() > 0.0 and r.max() < 1.0
    assert abs(r.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(r))
    hist, _ = np.histogram(r, bins=20, range=(0, 1))
    expect = len(r) / 20
    assert ((hist - expect) ** 2 / expect).sum() < 45  # chi2, 19 dof
    # not the uniforms of the event itself (Philox calls 0.. of the same event)
    k = O.uniform_ints(3, 1, 2, 0, 4, 0, 1000)
    u0 = (2.0 * k[:, 0].astype(np.float64) + 1.0) * 2.0 ** -53
    assert not np.any(np.isclose(u0, r[:1000], rtol=0, atol=1e-15))


def test_acceptance_law_for_constant_weights():
    n = 200000
    for c in (0.0, 0.1, 0.5, 1.0):
        acc = O.unweight_accept(7, 0, 0, 0, np.full(n, 2.0 * c), 2.0)
        frac = acc.mean()
        if c in (0.0, 1.0):
            assert frac == c
        else:
            assert abs(frac - c) < 4 * math.sqrt(c * (1 - c) / n), (c, frac)


def test_unweighted_events_follow_the_weighted_distribution():
    """Weights w = 1 + 3 u^2 on the events' first uniform u: the accepted
    events' u follow the density (1 + 3 u^2) / 2, and the efficiency equals
    <w> / w_max = 2 / 4."""
    n = 200000
    k = O.uniform_ints(11, 5, 1, 0, 1, 0, n)[:, 0].astype(np.float64)
    u = (2.0 * k + 1.0) * 2.0 ** -53
    w = 1.0 + 3.0 * u * u
    acc = O.unweight_accept(11, 5, 1, 0, w, 4.0)
    assert abs(acc.mean() - 0.5) < 4 * math.sqrt(0.25 / n)
    ua = u[acc]
    edges = np.linspace(0.0, 1.0, 21)
    hist, _ = np.histogram(ua, bins=edges)
    cdf = lambda t: (t + t ** 3) / 2.0  # noqa: E731
    expect = len(ua) * (cdf(edges[1:]) - cdf(edges[:-1]))
    assert ((hist - expect) ** 2 / expect).sum() < 45  # chi2, 19 dof


def _lab_events(itg, prec, n, seed=0, pdf=None, wmax=0.0):
    edges = W.uniform_grid(O.process_ndim(itg), 50)
    w, wmax, evs, nacc = O.unweight_events(itg, pdf, edges, prec, seed, 0, 0, 0, n, wmax=wmax)
    assert nacc == len(evs)
    return w, wmax, evs


def _mass2(p):
    return p[0] ** 2 - p[1] ** 2 - p[2] ** 2 - p[3] ** 2


@pytest.mark.parametrize("maker", [W.gg_ttbarg, W.gg_ttbarg_7d], ids=["rambo", "hierarchical"])
def test_exported_gg_events_conserve_momentum_and_pass_the_lab_frame_cuts(maker):
    itg = maker(13000.0)
    pdf = O.Pdf(W.synthetic_pdf_grid(0))
    w, wmax, evs = _lab_events(itg, W.FP64, 4000, pdf=pdf)
    assert wmax == w.max() > 0
    acc = O.unweight_accept(0, 0, 0, 0, w, wmax)
    assert [e.event for e in evs] == list(np.nonzero(acc)[0])
    # a uniform grid leaves the efficiency at a fraction of a percent: take a
    # lower w_max (events above it are always kept) for a larger sample
    cut = float(np.quantile(w[w > 0], 0.7))
    w2, wmax2, evs = _lab_events(itg, W.FP64, 4000, pdf=pdf, wmax=cut)
    assert wmax2 == cut and np.array_equal(w2, w)
    acc = O.unweight_accept(0, 0, 0, 0, w, cut)
    assert [e.event for e in evs] == list(np.nonzero(acc)[0])
    assert len(evs) > 300
    half = itg.sqrt_s / 2
    mt = itg.m_top
    for e in evs:
        p = np.array([list(r) for r in e.p])
        assert e.nout == 3 and 0 < e.x1 <= 1 and 0 < e.x2 <= 1
        assert np.array_equal(p[0], [e.x1 * half, 0, 0, e.x1 * half])
        assert np.array_equal(p[1], [e.x2 * half, 0, 0, -e.x2 * half])
        # conservation in the laboratory frame: a boost with the wrong sign
        # or rapidity breaks the longitudinal and energy sums
        assert np.allclose(p[2:].sum(axis=0), p[0] + p[1], rtol=0, atol=1e-9 * itg.sqrt_s)
        assert abs(_mass2(p[2]) / mt ** 2 - 1) < 1e-9 and abs(_mass2(p[3]) / mt ** 2 - 1) < 1e-9
        assert abs(_mass2(p[4])) < 1e-9 * p[4][0] ** 2
        # the generation cuts, which are defined in the laboratory frame
        g = p[4]
        pt = math.hypot(g[1], g[2])
        eta = math.atanh(g[3] / math.sqrt(pt * pt + g[3] ** 2))
        assert pt > itg.ptcut_g and abs(eta) < itg.etacut_g
        assert e.weight == w[e.event] > 0


def test_exported_ee_events_follow_the_angular_distribution():
    """e+e- -> mu+mu- at the Z pole: the unweighted events' cos(theta(e-, mu-))
    follows 1 + c^2 + (A1/A0) c, the closed form of the averaged |M|^2."""
    itg = W.ee_mumu(91.0)
    w, wmax, evs = _lab_events(itg, W.FP64, 60000, seed=4)
    assert len(evs) > 30000  # efficiency <w>/w_max of 1 + c^2 is about 2/3
    c = []
    for e in evs:
        p = np.array([list(r) for r in e.p])
        assert e.nout == 2 and e.x1 == 1 and e.x2 == 1
        assert np.allclose(p[2] + p[3], [91.0, 0, 0, 0], rtol=0, atol=1e-12 * 91)
        c.append(p[2][3] / p[2][0])  # mu- along the e- beam (+z)
    c = np.array(c)
    # A1/A0 at 91 GeV is about -1.7e-3: the forward-backward asymmetry is
    # invisible at this statistics, the 1 + c^2 shape is not
    edges = np.linspace(-1, 1, 21)
    hist, _ = np.histogram(c, bins=edges)
    cdf = lambda t: t + t ** 3 / 3  # noqa: E731
    expect = len(c) * (cdf(edges[1:]) - cdf(edges[:-1])) / (cdf(1) - cdf(-1))
    assert ((hist - expect) ** 2 / expect).sum() < 45  # chi2, 19 dof
    flat = np.full(20, len(c) / 20)
    assert ((hist - flat) ** 2 / flat).sum() > 500  # a flat sample would fail


def test_export_of_processes_without_a_record_is_refused():
    with pytest.raises(ValueError):
        _lab_events(W.pp_ttbar(), W.FP64, 10, pdf=O.Pdf(W.synthetic_pdf_grid(0)))
