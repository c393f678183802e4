"""Pins of the oracle's three-channel sampling of g g -> t tbar g
(oracle/src/channels.cpp; thesis Sec. "Multi-channel Monte Carlo").

Each check compares with something the channel code does not compute the
same way: the inverse of every map, the three-body phase-space volume by
quadrature of the Dalitz area, the normalisation of every channel density
integrated under another channel's sampling, the exact identity
sum_i alpha_i W_i = <w^2>, unbiasedness against the single-channel
generators, the channel frequencies, and the alpha update by hand.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import workloads as W
from test_oracle_phasespace import dalitz_volume

M_T, PTCUT, ETACUT = 173.0, 20.0, 2.5


def test_forward_then_inverse_is_the_identity():
    rng = np.random.default_rng(0)
    for rs, yb in ((400.0, 0.0), (800.0, 0.7), (3000.0, -1.9)):
        for ch in range(3):
            done = 0
            for _ in range(400):
                u = rng.random(5)
                r = O.channel_forward(ch, M_T, rs, PTCUT, ETACUT, yb, u)
                if r is None:
                    continue
                p, w = r
                # momentum conservation and masses of the generated point
                assert np.allclose(p.sum(axis=0), [rs, 0, 0, 0], rtol=0, atol=1e-9 * rs)
                m2 = p[:, 0] ** 2 - (p[:, 1:] ** 2).sum(axis=1)
                assert np.allclose(m2, [M_T ** 2, M_T ** 2, 0.0], rtol=0, atol=1e-7 * rs * rs)
                inv = O.channel_inverse(ch, M_T, rs, PTCUT, ETACUT, yb, p)
                assert inv is not None, (ch, u)
                u2, w2 = inv
                assert np.max(np.abs(u2 - u)) < 1e-8, (ch, u, u2)
                assert abs(w2 / w - 1) < 1e-8
                done += 1
            assert done > 300


def _mean_weight(ch, rs, yb, n, rng, indicator_of=None):
    ws = []
    for _ in range(n):
        r = O.channel_forward(ch, M_T, rs, PTCUT, ETACUT, yb, rng.random(5))
        if r is None:
            ws.append(0.0)
            continue
        p, w = r
        if indicator_of is not None:
            w = w if O.channel_inverse(indicator_of, M_T, rs, PTCUT, ETACUT, yb, p) is not None else 0.0
        ws.append(w)
    ws = np.array(ws)
    return ws.mean(), ws.std() / math.sqrt(n)


def test_full_support_channels_have_the_three_body_volume():
    """Channels 1 and 2 cover the whole phase space: their mean weight is the
    volume, by quadrature of the Dalitz area."""
    rng = np.random.default_rng(1)
    for rs in (500.0, 1500.0):
        vol = dalitz_volume(rs, M_T, M_T, 0.0)
        for ch in (1, 2):
            mean, err = _mean_weight(ch, rs, 0.3, 40000, rng)
            assert abs(mean - vol) < 4 * err, (rs, ch, mean, vol, err)


def test_channel_densities_integrate_to_one_under_the_others():
    """E_i[w_i / w_j] = integral of channel j's density = 1 for i = 1, 2
    (full support) and every j; channel 0's volume (its own mean weight) is
    the part of the phase space channel 1 finds inside channel 0's support."""
    rng = np.random.default_rng(2)
    rs, yb = 900.0, -0.4
    n = 30000
    for i in (1, 2):
        for j in range(3):
            vals = []
            for _ in range(n):
                r = O.channel_forward(i, M_T, rs, PTCUT, ETACUT, yb, rng.random(5))
                p, wi = r
                inv = O.channel_inverse(j, M_T, rs, PTCUT, ETACUT, yb, p)
                vals.append(wi / inv[1] if inv is not None else 0.0)
            vals = np.array(vals)
            assert abs(vals.mean() - 1.0) < 4 * vals.std() / math.sqrt(n) + 1e-12, (i, j, vals.mean())
    v0, e0 = _mean_weight(0, rs, yb, n, rng)
    v1, e1 = _mean_weight(1, rs, yb, n, rng, indicator_of=0)
    assert abs(v0 - v1) < 4 * math.hypot(e0, e1), (v0, v1)
    assert v0 < dalitz_volume(rs, M_T, M_T, 0.0)


@pytest.fixture(scope="module")
def pdf():
    return O.Pdf(W.synthetic_pdf_grid(0))


def test_channel_frequencies_and_update_sums(pdf):
    itg = W.gg_ttbarg_mc()
    edges = W.uniform_grid(17, 50)
    alpha = np.array([0.2, 0.5, 0.3])
    O.set_channel_alpha(alpha)
    n = 6000
    chans = []
    w2, wch = [], np.zeros(3)
    for ev in range(n):
        rec, dens = O.channels_event(itg, pdf, edges, W.FP64, 4, 1, 0, ev)
        chans.append(rec.channel)
        if rec.weight != 0.0:
            pden = alpha @ dens
            wch += rec.weight ** 2 * dens / pden
            assert dens[rec.channel] > 0
        w2.append(rec.weight ** 2)
    counts = np.bincount(chans, minlength=3)
    for i in range(3):
        assert abs(counts[i] - n * alpha[i]) < 4 * math.sqrt(n * alpha[i] * (1 - alpha[i]))
    sums, W_i = O.channels_iterate(itg, pdf, edges, W.FP64, 4, 1, 0, 0, n)
    assert np.allclose(W_i, wch / n, rtol=1e-12)
    # sum_i alpha_i W_i = <w^2> exactly: sum_i alpha_i p_i / p = 1
    assert abs(alpha @ W_i - sums[1] / n) <= 1e-12 * sums[1] / n
    O.set_channel_alpha([1 / 3, 1 / 3, 1 / 3])


def test_unbiased_against_the_single_channel_generators(pdf):
    """Every channel mixture estimates the same integral: three channels with
    equal and with skewed probabilities, and the hierarchical and RAMBO
    single-channel integrands, on uniform grids, agree within their errors."""
    n = 12000
    est = []
    for alpha in ([1 / 3, 1 / 3, 1 / 3], [0.7, 0.15, 0.15]):
        O.set_channel_alpha(alpha)
        sums, _ = O.channels_iterate(W.gg_ttbarg_mc(), pdf, W.uniform_grid(17, 50), W.FP64, 9, 0, 0, 0, n)
        m = sums[0] / n
        est.append((m, math.sqrt((sums[1] / n - m * m) / (n - 1))))
    O.set_channel_alpha([1 / 3, 1 / 3, 1 / 3])
    for itg in (W.gg_ttbarg_7d(), W.gg_ttbarg()):
        r = O.iterate(itg, pdf, W.uniform_grid(itg.ndim(), 50), W.FP64, 9, 0, 0, 0, n)
        m = r["sum"] / n
        est.append((m, math.sqrt((r["sum2"] / n - m * m) / (n - 1))))
    for a in range(len(est)):
        for b in range(a + 1, len(est)):
            assert abs(est[a][0] - est[b][0]) < 4 * math.hypot(est[a][1], est[b][1]), est


def test_alpha_update_by_hand():
    out = O.channel_update([1 / 3, 1 / 3, 1 / 3], [1.0, 4.0, 9.0], 0.5, 0.0)
    assert np.allclose(out, [1 / 6, 2 / 6, 3 / 6], rtol=1e-15)
    out = O.channel_update([0.5, 0.25, 0.25], [4.0, 1.0, 0.0], 1.0, 0.0)
    assert np.allclose(out, [2.0 / 2.25, 0.25 / 2.25, 0.0], rtol=1e-15)
    # floor, then renormalisation
    out = O.channel_update([0.5, 0.25, 0.25], [4.0, 1.0, 0.0], 1.0, 0.1)
    f = np.array([2.0 / 2.25, 0.25 / 2.25, 0.1])
    assert np.allclose(out, f / f.sum(), rtol=1e-15)
    # all sums zero: unchanged
    assert np.array_equal(O.channel_update([0.2, 0.3, 0.5], [0.0, 0.0, 0.0], 0.5, 0.0), [0.2, 0.3, 0.5])
