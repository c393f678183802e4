"""Pins of the oracle's unweighting (oracle/src/unweight.cpp; thesis Sec.
"Unweighted event exporter"): an event of weight w survives with probability
w / w_max, and the surviving events follow the weighted distribution."""
import math

import numpy as np

import oracle as O


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
