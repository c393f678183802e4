"""GPU: the weights pass, device-side unweighting and LHE export (thesis Sec.
"Unweighted event exporter") against the FP64 oracle (oracle/src/unweight.cpp)
on the same Philox streams.

Bars: FP64 weights within 1e-12 relative with the same zero pattern (where
the synthetic PDF's interpolant crosses zero near x -> 1 a weight is small
and carries the rounding of the stencil, so the bound there is 1e-12 of
1e-3 of the sample's largest weight, as for the luminosities in
test_gpu_parity.py); the
accepted sets equal, except for events whose weight lies within rounding of
the acceptance threshold r_i w_max (both sides decide in FP64); exported
laboratory-frame records within 1e-12 of the oracle's (FP64) or FP32
rounding of the momenta (FP32+Kahan, the warp-specialised kernel).  At the
benchmark launch (gg -> t tbar g, FP32, 1e7 events) sampled decisions and
records are checked one by one against the oracle with a w_max fixed in
advance by the oracle.
"""
import math
import xml.etree.ElementTree as ET

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PROCS = {"ee": W.ee_mumu(91.0), "gg": W.gg_ttbarg(), "gg7": W.gg_ttbarg_7d()}


@pytest.fixture(scope="module")
def gpu(pdf_grid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    M.lib()
    torch.cuda.init()
    return M.mc_pdf_load(pdf_grid)


def random_grid(ndim, nbins, seed):
    rng = np.random.default_rng(seed)
    return O.vegas_refine(W.uniform_grid(ndim, nbins), rng.exponential(size=(ndim, nbins)) ** 2, alpha=1.0)


def rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def gpu_weights(gpdf, itg, prec, edges, n, iteration=0, seed=0):
    ndim, nb1 = edges.shape
    v = M.mc_vegas_init(ndim, nb1 - 1, seed, prec)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, iteration)
    w = torch.full((max(n, 1),), float("nan"), dtype=torch.float64, device="cuda")
    r = M.mc_vegas_iterate_weights(v, itg, gpdf, n, w)
    torch.cuda.synchronize()
    return v, w, r


def gpu_unweight(v, gpdf, itg, w, n, wmax, cap):
    ev = torch.zeros((max(cap, 1), M.EVENT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    nacc = M.mc_unweight(v, itg, gpdf, w, n, wmax, ev, cap)
    torch.cuda.synchronize()
    return nacc, M.events_from_bytes(ev[:min(nacc, cap)].cpu().numpy().tobytes())


def lab(e):
    return np.array([list(r) for r in e.p])


@pytest.mark.parametrize("name,prec,n", [("ee", M.MC_FP64, 20000), ("gg", M.MC_FP64, 6000), ("gg7", M.MC_FP64, 6000),
                                         ("ee", M.MC_FP32_KAHAN, 20000), ("gg", M.MC_FP32_KAHAN, 20000),
                                         ("gg7", M.MC_FP32_KAHAN, 20000)])
def test_weights_pass(gpu, oracle_pdf, name, prec, n):
    """Every event's weight, including 0 for cut events; the launch's sums are
    the sums of these weights."""
    itg = PROCS[name]
    edges = random_grid(O.process_ndim(itg), 50, 3)
    v, w, r = gpu_weights(gpu, itg, prec, edges, n, iteration=2, seed=7)
    wg = w.cpu().numpy()
    wo, _, _, _ = O.unweight_events(itg, oracle_pdf, edges, prec, 7, 2, 0, 0, n, cap=0)
    assert not np.isnan(wg).any()
    assert r.wmax == wg.max() and r.n_nonzero == np.count_nonzero(wg)
    assert abs(r.sum - math.fsum(wg)) <= 1e-12 * abs(r.sum)
    assert abs(r.sum2 - math.fsum(wg * wg)) <= 1e-12 * abs(r.sum2)
    both = (wg != 0) & (wo != 0)
    if prec == M.MC_FP64:
        assert np.array_equal(wg != 0, wo != 0)
        floor = 1e-3 * np.abs(wo).max()
        assert np.all(np.abs(wg - wo) <= 1e-12 * np.maximum(np.abs(wo), floor)), np.max(rel(wg[both], wo[both]))
    else:
        assert np.count_nonzero((wg != 0) != (wo != 0)) <= max(1, n // 1000)
        e = rel(wg[both], wo[both])
        assert np.median(e) < 1e-5 and np.quantile(e, 0.99) < 1e-3
    v.free()


@pytest.mark.parametrize("name,prec,n", [("ee", M.MC_FP64, 20000), ("gg", M.MC_FP64, 6000), ("gg7", M.MC_FP64, 6000),
                                         ("gg", M.MC_FP32_KAHAN, 20000), ("gg7", M.MC_FP32_KAHAN, 20000)])
def test_unweighted_sample_against_oracle(gpu, oracle_pdf, name, prec, n):
    """The accepted set and the laboratory-frame records.  w_max: 2% of each
    side's own largest weight (events above it are always kept), so that a
    hundred events or more survive on a grid that is far from adapted."""
    itg = PROCS[name]
    frac = 0.02
    edges = random_grid(O.process_ndim(itg), 50, 4)
    v, w, r = gpu_weights(gpu, itg, prec, edges, n, iteration=1, seed=3)
    nacc, ev = gpu_unweight(v, gpu, itg, w, n, frac * r.wmax, n)
    assert nacc == len(ev) > 50
    wo, wmax_o, evo, nacc_o = O.unweight_events(itg, oracle_pdf, edges, prec, 3, 1, 0, 0, n)
    wo2, _, evo, nacc_o = O.unweight_events(itg, oracle_pdf, edges, prec, 3, 1, 0, 0, n, wmax=frac * wmax_o)
    assert np.array_equal(wo, wo2)
    ig = [int(e) for e in ev["event"]]
    io = [e.event for e in evo]
    assert ig == sorted(ig) and len(set(ig)) == len(ig)  # event order, no repeats
    wg = w.cpu().numpy()
    assert np.array_equal(ev["weight"], wg[ig])
    # decisions that differ must sit at the threshold, within the weights' error
    r_acc = O.acceptance_uniforms(3, 1, 0, 0, n)
    tol = 1e-11 if prec == M.MC_FP64 else 2e-2
    diff = set(ig) ^ set(io)
    for i in diff:
        assert abs(wo[i] - r_acc[i] * frac * wmax_o) <= tol * max(wo[i], r_acc[i] * frac * wmax_o), i
    assert len(diff) <= (0 if prec == M.MC_FP64 else max(2, nacc // 50)) + 2
    # records of the events both accepted
    rec_o = {e.event: e for e in evo}
    for e in ev:
        o = rec_o.get(int(e["event"]))
        if o is None:
            continue
        po = lab(o)
        scale = po[:2, 0].sum()
        assert e["nout"] == o.nout and e["proc"] == o.proc
        if prec == M.MC_FP64:
            assert abs(e["x1"] - o.x1) <= 1e-12 * o.x1 and abs(e["x2"] - o.x2) <= 1e-12 * o.x2
            assert np.max(np.abs(e["p"] - po)) <= 1e-12 * scale
        else:
            assert abs(e["x1"] - o.x1) <= 1e-6 * o.x1 and abs(e["x2"] - o.x2) <= 1e-6 * o.x2
            assert np.max(np.abs(e["p"] - po)) <= 2e-5 * scale
        # laboratory-frame conservation of the device record itself
        p = e["p"]
        assert np.allclose(p[2:2 + e["nout"]].sum(axis=0), p[0] + p[1], rtol=0,
                           atol=(1e-10 if prec == M.MC_FP64 else 1e-4) * scale)
    v.free()


def test_capacity_count_only_and_argument_checks(gpu):
    itg = PROCS["ee"]
    n = 10000
    v, w, r = gpu_weights(gpu, itg, M.MC_FP64, W.uniform_grid(2, 50), n)
    full_n, full = gpu_unweight(v, gpu, itg, w, n, r.wmax, n)
    assert full_n > 1000
    part_n, part = gpu_unweight(v, gpu, itg, w, n, r.wmax, 100)
    assert part_n == full_n and np.array_equal(part, full[:100])
    assert gpu_unweight(v, gpu, itg, w, n, r.wmax, 0)[0] == full_n
    # w_max <= 0 keeps nothing; a tiny w_max keeps every event of positive weight
    assert gpu_unweight(v, gpu, itg, w, n, 0.0, n)[0] == 0
    assert gpu_unweight(v, gpu, itg, w, n, 1e-300, n)[0] == np.count_nonzero(w.cpu().numpy() > 0)
    with pytest.raises(M.McError):
        gpu_unweight(v, gpu, itg, w, n - 1, r.wmax, n)  # not the last iteration's size
    with pytest.raises(M.McError):
        gpu_unweight(v, gpu, W.pp_ttbar(), w, n, r.wmax, n)  # no event record
    M.mc_vegas_refine(v)
    with pytest.raises(M.McError):
        gpu_unweight(v, gpu, itg, w, n, r.wmax, n)  # grid changed since
    with pytest.raises(M.McError):
        M.mc_vegas_iterate_weights(v, itg, gpu, 1 << 32, w)
    v.free()


def test_decision_at_the_threshold_is_exact(gpu):
    """Weights set to RN(r_i w_max) exactly (w > r w_max is false: rejected)
    and to the next double above it (accepted), r_i from the oracle, for
    w_max on the device's integer path and for a w_max so small that the
    products are subnormal (its FP64 path): the decision is the FP64
    comparison, bit for bit."""
    itg = PROCS["ee"]
    n = 50000
    v, w, r = gpu_weights(gpu, itg, M.MC_FP64, W.uniform_grid(2, 50), n)
    racc = O.acceptance_uniforms(0, 0, 0, 0, n)
    for wmax in (1234.5678, 3.0e-10, 1.0, 2.0 ** -1000):
        thr = racc * wmax
        crafted = np.where(np.arange(n) % 2 == 0, thr, np.nextafter(thr, np.inf))
        w.copy_(torch.from_numpy(crafted))
        nacc, ev = gpu_unweight(v, gpu, itg, w, n, wmax, n)
        assert nacc == n // 2 and np.array_equal(ev["event"], np.arange(1, n, 2)), wmax
    v.free()


def test_full_size_gg_ttbarg_sampled(gpu, oracle_pdf):
    """At the benchmark launch (gg -> ttg, FP32+Kahan, 1e7 events, uniform
    grid): w_max fixed in advance from an oracle sample; sampled decisions and
    records against the oracle, one event at a time; the count against the
    expected number sum(min(w, w_max)) / w_max."""
    itg = PROCS["gg"]
    n = 10_000_000
    edges = W.uniform_grid(14, 50)
    wo_small, _, _, _ = O.unweight_events(itg, oracle_pdf, edges, M.MC_FP32_KAHAN, 0, 0, 0, 0, 20000, cap=0)
    wmax = float(np.quantile(wo_small[wo_small > 0], 0.99))
    v, w, r = gpu_weights(gpu, itg, M.MC_FP32_KAHAN, edges, n)
    nacc, ev = gpu_unweight(v, gpu, itg, w, n, wmax, n // 4)
    assert nacc <= n // 4
    wg = w.cpu().numpy()
    expect = np.minimum(wg, wmax).sum() / wmax
    p = np.minimum(wg, wmax) / wmax
    assert abs(nacc - expect) <= 6 * math.sqrt((p * (1 - p)).sum()) + 1
    ig = ev["event"]
    assert np.all(np.diff(ig) > 0)
    acc = np.zeros(n, dtype=bool)
    acc[ig] = True
    rng = np.random.default_rng(11)
    sample = np.concatenate([rng.choice(ig, 150, replace=False), rng.choice(n, 150, replace=False)])
    flips = 0
    for i in sample:
        wo, _, evo, k = O.unweight_events(itg, oracle_pdf, edges, M.MC_FP32_KAHAN, 0, 0, 0, int(i), 1, wmax=wmax)
        ro = O.acceptance_uniforms(0, 0, 0, int(i), 1)[0]
        if bool(k) != acc[i]:
            flips += 1
            assert abs(wo[0] - ro * wmax) <= 2e-2 * max(wo[0], ro * wmax)
            continue
        if k:
            e = ev[np.searchsorted(ig, i)]
            po = lab(evo[0])
            assert np.max(np.abs(e["p"] - po)) <= 2e-5 * po[:2, 0].sum()
    assert flips <= 3
    v.free()


def parse_lhe(path):
    root = ET.parse(path).getroot()
    init = [ln.split() for ln in root.find("init").text.split("\n") if ln.strip()]
    events = []
    for e in root.findall("event"):
        lines = [ln for ln in e.text.split("\n") if ln.strip() and not ln.startswith("#")]
        events.append(np.array([[float(t) for t in ln.split()] for ln in lines[1:]]))
    return init, events


def test_generate_lhe_ee_z_pole(gpu, tmp_path):
    """mc_generate_lhe end to end for e+e- -> mu+mu- at 91 GeV (FP64): the
    cross section written to <init> against the closed form 1958.95 pb, the
    event count against the efficiency, and the unweighted cos(theta)
    distribution against 1 + c^2."""
    itg = PROCS["ee"]
    path = tmp_path / "ee.lhe"
    res, st = M.mc_generate_lhe(itg, None, str(path), ntrain=2, niter=3, nevents=50000, prec=M.MC_FP64, threads=4)
    assert res.n_iter == 3 and st.n_weighted == 150000
    assert abs(res.mean - 1958.95) <= 5 * res.sigma + 1e-4 * 1958.95
    init, events = parse_lhe(path)
    assert len(events) == st.n_accepted > 75000  # efficiency of 1 + c^2 is about 2/3
    assert float(init[1][0]) == pytest.approx(res.mean, rel=1e-10)
    c = np.array([ev[2][8] / ev[2][9] for ev in events])  # mu- pz / E
    edges = np.linspace(-1, 1, 21)
    hist, _ = np.histogram(c, bins=edges)
    cdf = lambda t: t + t ** 3 / 3  # noqa: E731
    expect = len(c) * (cdf(edges[1:]) - cdf(edges[:-1])) / (cdf(1) - cdf(-1))
    assert ((hist - expect) ** 2 / expect).sum() < 50  # chi2, 19 dof
    print(f"\nee LHE: {st.n_accepted} events, eff {st.n_accepted / st.n_weighted:.3f}, "
          f"iterate {st.iterate_ms:.2f} ms, unweight {st.unweight_ms:.2f} ms, wall {st.wall_ms:.1f} ms")


def test_generate_lhe_gg_ttbarg_fp32(gpu, tmp_path):
    """gg -> t tbar g, FP32 (warp-specialised weights pass): every written
    event conserves momentum in the laboratory frame, has on-shell tops and
    passes the laboratory-frame gluon cuts."""
    itg = PROCS["gg"]
    path = tmp_path / "gg.lhe"
    res, st = M.mc_generate_lhe(itg, gpu, str(path), ntrain=3, niter=2, nevents=400000, prec=M.MC_FP32_KAHAN)
    init, events = parse_lhe(path)
    assert len(events) == st.n_accepted > 100 and res.mean > 0
    for ev in events:
        mom = ev[:, [9, 6, 7, 8]]  # E, px, py, pz
        s = mom[0, 0] + mom[1, 0]
        assert np.allclose(mom[2:].sum(axis=0), mom[0] + mom[1], rtol=0, atol=1e-4 * s)
        for k in (2, 3):
            m2 = mom[k, 0] ** 2 - (mom[k, 1:] ** 2).sum()
            assert abs(math.sqrt(max(m2, 0.0)) / itg.m_top - 1) < 1e-3
        g = mom[4]
        pt = math.hypot(g[1], g[2])
        eta = math.atanh(g[3] / math.sqrt(pt * pt + g[3] ** 2))
        assert pt > itg.ptcut_g * (1 - 1e-5) and abs(eta) < itg.etacut_g + 1e-5
    print(f"\ngg LHE: {st.n_accepted} events, eff {st.n_accepted / st.n_weighted:.4f}, "
          f"iterate {st.iterate_ms:.2f} ms, unweight {st.unweight_ms:.2f} ms, wall {st.wall_ms:.1f} ms")
