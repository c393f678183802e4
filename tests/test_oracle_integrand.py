"""Pins of the oracle's per-event integrand and full VEGAS integration
(thesis eq. mc_master_formula, eq. mc_est_is, Sec. "Adaptive Monte Carlo:
VEGAS algorithm")."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2302_03343_b300 import workloads as W


def mass2(p):
    return p[0] ** 2 - p[1] ** 2 - p[2] ** 2 - p[3] ** 2


def eemumu_total(itg):
    s = itg.sqrt_s ** 2
    f = lambda c: O.me2_eemumu(itg.alpha, itg.mz, itg.gz, itg.sw2, s, c)
    val, _ = integrate.quad(f, -1, 1, epsrel=1e-13)
    return val * 2 * math.pi / (64 * math.pi ** 2 * s) * itg.gev2pb


def test_eemumu_integration_matches_closed_form():
    itg = W.ee_mumu(91.0)
    exact = eemumu_total(itg)
    assert abs(exact - 1958.951) < 0.01  # thesis-configuration value, derived from the closed form
    r = O.integrate(itg, None, W.uniform_grid(2, 50), 0, seed=0, gid=0, niter=5, nevents=100000)
    assert abs(r["mean"] - exact) < 3 * r["sigma"]
    assert abs(r["mean"] / exact - 1) < 1e-3


@pytest.mark.parametrize("rs", [500.0, 13000.0])
def test_eemumu_other_energies(rs):
    itg = W.ee_mumu(rs)
    r = O.integrate(itg, None, W.uniform_grid(2, 20), 0, seed=3, gid=1, niter=3, nevents=20000)
    exact = eemumu_total(itg)
    assert abs(r["mean"] - exact) < 4 * r["sigma"]


def test_event_records_pp_ttbar(oracle_pdf):
    itg = W.pp_ttbar()
    edges = W.uniform_grid(4, 50)
    npass = 0
    for ev in range(400):
        r = O.event(itg, oracle_pdf, edges, 0, 0, 0, 0, ev)
        assert r.weight == r.f * r.jac
        assert abs(r.shat - r.x1 * r.x2 * itg.sqrt_s ** 2) <= 1e-12 * r.shat
        if r.pass_:
            npass += 1
            p = np.array(r.p)
            np.testing.assert_allclose(p[2] + p[3], p[0] + p[1], atol=1e-9 * math.sqrt(r.shat))
            assert abs(mass2(p[2]) - itg.m_top ** 2) < 1e-9 * r.shat
            assert r.f > 0
        else:
            assert r.f == 0 and r.shat <= 4 * itg.m_top ** 2
    assert 0 < npass < 400


def test_event_records_gg_ttbarg_and_cuts(oracle_pdf):
    itg = W.gg_ttbarg()
    edges = W.uniform_grid(14, 50)
    seen = {"pass": 0, "cut": 0}
    for ev in range(3000):
        r = O.event(itg, oracle_pdf, edges, 1, 0, 0, 0, ev)
        p = np.array(r.p)
        if r.shat <= 4 * itg.m_top ** 2:
            assert r.pass_ == 0 and r.weight == 0
            continue
        np.testing.assert_allclose(p[2] + p[3] + p[4], p[0] + p[1], atol=1e-9 * math.sqrt(r.shat))
        pt = math.hypot(p[4][1], p[4][2])
        eta = math.asinh(p[4][3] / pt) + 0.5 * math.log(r.x1 / r.x2)
        inside = pt > itg.ptcut_g and abs(eta) < itg.etacut_g
        assert bool(r.pass_) == inside
        seen["pass" if inside else "cut"] += 1
        if inside:
            # the bicubic interpolant can dip below zero where the sparse log-x
            # knots near x = 1 meet (1-x)^b; |M|^2 itself is positive
            assert r.f != 0 and r.me2 > 0
    assert seen["pass"] > 0 and seen["cut"] > 0


def test_iterate_threads_do_not_change_the_result(oracle_pdf):
    itg = W.pp_ttbar()
    edges = W.uniform_grid(4, 50)
    a = O.iterate(itg, oracle_pdf, edges, 0, 0, 1, 0, 0, 4000, nthreads=1)
    b = O.iterate(itg, oracle_pdf, edges, 0, 0, 1, 0, 0, 4000, nthreads=5)
    assert a["n_nonzero"] == b["n_nonzero"] and a["wmax"] == b["wmax"]
    assert abs(a["sum"] - b["sum"]) < 1e-13 * abs(a["sum"])
    np.testing.assert_array_equal(a["hist_n"], b["hist_n"])


def test_gg_ttbarg_rambo_and_hierarchical_integrate_alike(oracle_pdf):
    # one cross section, two phase-space parametrisations (Sec. "RAMBO" and
    # table tab:hierarchical): the VEGAS estimates agree within errors
    r14 = O.integrate(W.gg_ttbarg(), oracle_pdf, W.uniform_grid(14, 20), 0, seed=1, gid=0, niter=3, nevents=12000)
    r7 = O.integrate(W.gg_ttbarg_7d(), oracle_pdf, W.uniform_grid(7, 20), 0, seed=1, gid=0, niter=3, nevents=12000)
    assert abs(r14["mean"] - r7["mean"]) < 4 * math.hypot(r14["sigma"], r7["sigma"]), (r14, r7)


def test_pp_ttbarj_channel_sum():
    """p p -> t tbar + parton: with the quark densities set to zero it is the
    gg -> t tbar g integrand of the same generator, event by event; with
    only the u and ubar densities, the q qbar and qbar q channels (gluon
    density zero) give the sum of the two orientations, and swapping the
    beams' u and ubar swaps them."""
    import numpy as np
    import oracle as O
    from paper_2302_03343_b300 import workloads as W
    g = W.synthetic_pdf_grid(0)
    pids = list(g.pids)
    glue = g.xf.copy()
    for i, pid in enumerate(pids):
        if pid != 21:
            glue[:, :, i] = 0.0
    Pg = O.Pdf(W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=glue, params=g.params))
    edges = W.uniform_grid(7, 50)
    n_pass = 0
    for ev in range(300):
        a = O.event(W.pp_ttbarj(), Pg, edges, W.FP64, 1, 0, 0, ev)
        b = O.event(W.gg_ttbarg_7d(), Pg, edges, W.FP64, 1, 0, 0, ev)
        assert abs(a.weight - b.weight) <= 1e-14 * abs(b.weight)  # the luminosity's division order
        n_pass += a.pass_
    assert n_pass > 100
    uu = g.xf.copy()
    for i, pid in enumerate(pids):
        if pid not in (2, -2):
            uu[:, :, i] = 0.0
    Pu = O.Pdf(W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=uu, params=g.params))
    for ev in range(100):
        r = O.event(W.pp_ttbarj(), Pu, edges, W.FP64, 1, 0, 0, ev)
        if not r.pass_:
            continue
        l = list(r.lumi_x)
        # (an interpolated density may undershoot below zero near x -> 1)
        assert l[0] == 0 and l[3] == l[4] == l[5] == l[6] == 0 and l[1] != 0 and l[2] != 0
        p = np.array([list(q) for q in r.p])
        m12 = O.me2_qqbar_ttbarg(0.118, 173.0, p)
        m21 = O.me2_qqbar_ttbarg(0.118, 173.0, p[[1, 0, 2, 3, 4]])
        assert r.me2_qq == m12 and r.me2_x[0] == m21
        f = (l[1] * m12 + l[2] * m21) / (2 * r.shat) * r.ps_weight * 0.3893794e9
        assert abs(r.f / f - 1) < 1e-13
