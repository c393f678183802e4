"""Pins of the oracle's VEGAS map, refinement and combination
(thesis Sec. "Adaptive Monte Carlo: VEGAS algorithm")."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import workloads as W


def test_map_on_uniform_grid_is_identity():
    nb = 50
    edges = W.uniform_grid(3, nb)
    for prec in (0, 1):
        bits = O.uniform_bits(prec)
        k = O.uniform_ints(11, 0, 0, prec, 3, 0, 200)
        for row in k:
            x, bins, jac = O.vegas_map(edges, prec, row)
            u = (2 * row.astype(np.float64) * nb + 1) / (nb * 2.0 ** (bits + 1))
            np.testing.assert_allclose(x, u, rtol=0, atol=1e-15)
            assert list(bins) == [int(v) * nb >> bits for v in row]
            assert abs(jac - 1.0) < 1e-12


def test_map_jacobian_is_inverse_density():
    # a random monotone grid: x lies inside its bin, J = nbins * width
    rng = np.random.default_rng(0)
    nb = 7
    e = np.concatenate([[0.0], np.sort(rng.uniform(size=nb - 1)), [1.0]])[None, :]
    k = O.uniform_ints(3, 0, 0, 0, 1, 0, 500)
    for row in k:
        x, bins, jac = O.vegas_map(e, 0, row)
        b = bins[0]
        assert e[0, b] < x[0] < e[0, b + 1]
        assert abs(jac - nb * (e[0, b + 1] - e[0, b])) < 1e-14


def test_refine_flat_histogram_is_a_fixed_point():
    edges = W.uniform_grid(2, 10)
    new = O.vegas_refine(edges, np.ones((2, 10)), alpha=1.5)
    np.testing.assert_allclose(new, edges, atol=1e-15)


def test_refine_support_by_hand():
    # With alpha = 0 every bin with non-zero smoothed weight has importance 1,
    # so new edges split the support uniformly.  A histogram with weight only in
    # bin 0 of 8 has smoothed support in bins 0 and 1: [0, 2/8].
    edges = W.uniform_grid(1, 8)
    h = np.zeros((1, 8))
    h[0, 0] = 3.0
    new = O.vegas_refine(edges, h, alpha=0.0)
    expect = np.concatenate([np.arange(8) * (0.25 / 8), [1.0]])
    np.testing.assert_allclose(new[0], expect, atol=1e-15)
    # empty histogram: grid kept
    np.testing.assert_array_equal(O.vegas_refine(edges, np.zeros((1, 8))), edges)


def test_refine_keeps_edges_monotone_and_pinned():
    rng = np.random.default_rng(1)
    edges = W.uniform_grid(3, 20)
    for _ in range(5):
        edges = O.vegas_refine(edges, rng.exponential(size=(3, 20)) ** 3, alpha=1.5)
        assert np.all(np.diff(edges, axis=1) > 0)
        assert np.all(edges[:, 0] == 0.0) and np.all(edges[:, -1] == 1.0)


def test_grid_approaches_quantiles_of_abs_f():
    # The thesis's target density is p_best = |f| / int |f|.  Refining with
    # noise-free histograms of f(x) = 1 + 3x (d_b = N nbins Delta_b int_b f^2)
    # brings the grid within a tenth of a bin of the quantiles of p ~ 1 + 3x
    # in three steps (later noise-free steps drift: the three-point smoothing
    # inverts alternating patterns, which sampling noise hides in practice).
    nb = 10
    f2 = lambda a, b: ((1 + 3 * b) ** 3 - (1 + 3 * a) ** 3) / 9.0
    e = W.uniform_grid(1, nb)
    for _ in range(3):
        d = np.array([[(e[0, b + 1] - e[0, b]) * f2(e[0, b], e[0, b + 1]) for b in range(nb)]])
        e = O.vegas_refine(e, d, alpha=1.5)
    k = np.arange(1, nb) / nb
    q = (-1 + np.sqrt(1 + 15 * k)) / 3  # CDF (x + 3x^2/2) / (5/2) = k
    width = np.diff(np.concatenate([[0.0], q, [1.0]]))
    err = np.abs(e[0, 1:-1] - q) / np.minimum(width[:-1], width[1:])
    assert np.max(err) < 0.1, err


def test_refinement_reduces_variance():
    # importance sampling with the adapted grid (eq. var_is) beats plain MC
    itg = W.gauss(4)
    r = O.integrate(itg, None, W.uniform_grid(4, 50), 0, seed=1, gid=0, niter=6, nevents=50000)
    s2 = r["per_iter"][:, 1]
    assert s2[-1] < s2[0] / 20.0, s2


def test_iteration_estimate_is_variance_of_the_mean():
    w = np.random.default_rng(2).exponential(size=1000)
    m, v = O.iteration_estimate(w.sum(), (w * w).sum(), w.size)
    assert abs(m - w.mean()) < 1e-14
    assert abs(v - w.var(ddof=1) / w.size) < 1e-12 * v


def test_combine_special_cases():
    m, s, c = O.combine([2.0, 2.0, 2.0], [0.04, 0.04, 0.04])
    assert abs(m - 2.0) < 1e-15 and abs(s - 0.2 / math.sqrt(3)) < 1e-15 and c == 0.0
    # two measurements: weighted mean and chi^2 with one degree of freedom
    m, s, c = O.combine([1.0, 3.0], [1.0, 4.0])
    assert abs(m - (1.0 + 3.0 / 4.0) / (1.0 + 0.25)) < 1e-15
    assert abs(s - math.sqrt(1.0 / 1.25)) < 1e-15
    assert abs(c - ((1.0 - m) ** 2 + (3.0 - m) ** 2 / 4.0)) < 1e-14


@pytest.mark.parametrize("dim", [4, 8])
def test_gaussian_closed_form(dim):
    itg = W.gauss(dim)
    r = O.integrate(itg, None, W.uniform_grid(dim, 50), 0, seed=0, gid=0, niter=6, nevents=60000)
    exact = W.gauss_exact(dim)
    assert abs(r["mean"] - exact) < 4 * r["sigma"], (r["mean"], exact, r["sigma"])
    assert r["chi2dof"] < 5.0


def test_histograms_account_for_every_event():
    itg = W.gauss(3)
    edges = W.uniform_grid(3, 10)
    r = O.iterate(itg, None, edges, 1, seed=4, iteration=0, gid=0, first=0, n=3000)
    assert np.all(r["hist_n"].sum(axis=1) == 3000)
    np.testing.assert_allclose(r["hist_w2"].sum(axis=1), r["sum2"], rtol=1e-12)
