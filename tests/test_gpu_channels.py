"""GPU: three-channel sampling of g g -> t tbar g (MC_GG_TTBARG_MC; thesis Sec.
"Multi-channel Monte Carlo") against the FP64 oracle (oracle/src/channels.cpp)
on the same Philox streams.

Bars: the channel of every event identical (an integer decision taken in
FP64 on both sides from the same 24-bit uniform); FP64 mode: channel
densities within 1e-10, weights within 1e-12 (relative to 1e-3 of the
sample's largest weight where the synthetic PDF interpolant crosses zero),
bin counts of all 17 grid dimensions bit-exact, sums and the alpha-update
sums within 1e-10; FP32 mode: per-event error statistics, the median at
the FP32 rounding level (1e-5) as for the other processes, the 99th
percentile below 1e-2: the channels for radiation off the top quarks sample
the region where the gluon is collinear with a top, and there the |M|^2
propagators 1/(2 p_t.p_g), formed from FP32 momenta of energies E_t, E_g,
carry absolute errors of about 6e-8 E_t E_g, which RAMBO's flat sampling
rarely meets.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = M.REC
ALPHA = np.array([0.5, 0.3, 0.2])


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


def make_vegas(prec, edges, iteration=0, seed=0, alpha=ALPHA):
    v = M.mc_vegas_init(17, edges.shape[1] - 1, seed, prec)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, iteration)
    M.mc_vegas_set_channels(v, alpha)
    return v


def gpu_records(gpdf, prec, edges, k, iteration=0, seed=0):
    v = make_vegas(prec, edges, iteration, seed)
    out = torch.full((k, M.REC_STRIDE), float("nan"), dtype=torch.float64, device="cuda")
    M.mc_debug_events(v, W.gg_ttbarg_mc(), gpdf, 0, k, out)
    torch.cuda.synchronize()
    v.free()
    return out.cpu().numpy()


def oracle_records(opdf, prec, edges, k, iteration=0, seed=0):
    O.set_channel_alpha(ALPHA)
    recs = [O.channels_event(W.gg_ttbarg_mc(), opdf, edges, prec, seed, iteration, 0, ev) for ev in range(k)]
    O.set_channel_alpha([1 / 3, 1 / 3, 1 / 3])
    return recs


def test_fp64_events_against_oracle(gpu, oracle_pdf):
    edges = random_grid(17, 50, 5)
    k = 3000
    g = gpu_records(gpu, M.MC_FP64, edges, k, iteration=3, seed=2)
    recs = oracle_records(oracle_pdf, M.MC_FP64, edges, k, iteration=3, seed=2)
    ch_o = np.array([r.channel for r, _ in recs])
    assert np.array_equal(g[:, R["CHANNEL"]].astype(int), ch_o)
    assert set(ch_o) == {0, 1, 2}
    dens_o = np.array([d for _, d in recs])
    dens_g = g[:, R["DENS"]:R["DENS"] + 3]
    assert np.array_equal(dens_g > 0, dens_o > 0)
    nz = dens_o > 0
    assert np.max(np.abs(dens_g[nz] / dens_o[nz] - 1)) < 1e-10
    wo = np.array([r.weight for r, _ in recs])
    wg = g[:, R["W"]]
    assert np.array_equal(wg != 0, wo != 0)
    assert np.count_nonzero(wo) > k // 3
    floor = 1e-3 * np.abs(wo).max()
    assert np.all(np.abs(wg - wo) <= 1e-12 * np.maximum(np.abs(wo), floor))
    po = np.array([[list(r.p[i]) for i in range(2, 5)] for r, _ in recs])
    pg = g[:, R["P"] + 8:R["P"] + 20].reshape(k, 3, 4)
    ok = wo != 0
    scale = np.array([r.p[0][0] + r.p[1][0] for r, _ in recs])[ok]
    assert np.max(np.abs(pg[ok] - po[ok]).max(axis=(1, 2)) / scale) < 1e-12
    bins_o = np.array([list(r.bin)[:7] for r, _ in recs])
    assert np.array_equal(g[:, R["BIN"]:R["BIN"] + 7].astype(int), bins_o)


def test_fp32_events_error_statistics(gpu, oracle_pdf):
    # the grid in FP32 on both sides: the FP32 path maps through an FP32 copy
    # of the edges, and the channel densities of narrow bins would otherwise
    # compare the two roundings of the grid rather than the arithmetic
    edges = random_grid(17, 50, 6).astype(np.float32).astype(np.float64)
    k = 4000
    g = gpu_records(gpu, M.MC_FP32_KAHAN, edges, k, iteration=1, seed=4)
    recs = oracle_records(oracle_pdf, M.MC_FP32_KAHAN, edges, k, iteration=1, seed=4)
    assert np.array_equal(g[:, R["CHANNEL"]].astype(int), [r.channel for r, _ in recs])
    wo = np.array([r.weight for r, _ in recs])
    wg = g[:, R["W"]]
    both = (wo != 0) & (wg != 0)
    flips = np.count_nonzero((wo != 0) != (wg != 0))
    e = np.abs(wg[both] - wo[both]) / np.abs(wo[both])
    print(f"\nthree-channel FP32 per-event rel. error: median {np.median(e):.2e} p99 {np.quantile(e, .99):.2e} "
          f"max {e.max():.2e}; flips {flips}/{k}")
    assert flips <= max(2, k // 500)
    assert np.median(e) < 1e-5 and np.quantile(e, 0.99) < 1e-2
    # the large errors sit where the gluon is close to collinear with a top:
    # small 2 p_t.p_g / (E_t E_g) (oracle momenta)
    p = np.array([[list(r.p[i]) for i in range(2, 5)] for r, _ in recs])[both]

    def coll(a, b):
        return 2 * (a[:, 0] * b[:, 0] - (a[:, 1:] * b[:, 1:]).sum(axis=1)) / (a[:, 0] * b[:, 0])
    c = np.minimum(coll(p[:, 0], p[:, 2]), coll(p[:, 1], p[:, 2]))
    big = e > 1e-3
    print(f"collinearity: median {np.median(c):.2e}, at errors > 1e-3 {np.median(c[big]) if big.any() else 0:.2e}")
    if big.sum() >= 5:
        assert np.median(c[big]) < 0.1 * np.median(c)


def test_iteration_sums_histograms_and_channel_sums(gpu, oracle_pdf):
    edges = random_grid(17, 50, 7)
    n = 12000
    v = make_vegas(M.MC_FP64, edges, iteration=2, seed=8)
    r = M.mc_vegas_iterate(v, W.gg_ttbarg_mc(), gpu, n)
    w2, cnt = M.mc_vegas_get_hist(v)
    alpha, wch = M.mc_vegas_get_channels(v)
    v.free()
    assert np.allclose(alpha, ALPHA, rtol=1e-15)
    O.set_channel_alpha(ALPHA)
    sums, wch_o = O.channels_iterate(W.gg_ttbarg_mc(), oracle_pdf, edges, M.MC_FP64, 8, 2, 0, 0, n)
    ref = O.iterate(W.gg_ttbarg_mc(), oracle_pdf, edges, M.MC_FP64, 8, 2, 0, 0, n)
    O.set_channel_alpha([1 / 3, 1 / 3, 1 / 3])
    assert abs(r.sum - sums[0]) <= 1e-10 * abs(sums[0])
    assert abs(r.sum2 - sums[1]) <= 1e-10 * abs(sums[1])
    assert abs(r.wmax - sums[2]) <= 1e-12 * sums[2]
    assert np.max(np.abs(wch / wch_o - 1)) < 1e-10
    assert np.array_equal(cnt, ref["hist_n"])  # all 17 grid dimensions
    assert cnt[:2].sum(axis=1).tolist() == [n, n] and cnt[2:].sum() == 5 * n
    nzb = ref["hist_w2"] > 0
    assert np.max(np.abs(w2[nzb] / ref["hist_w2"][nzb] - 1)) < 1e-10


@pytest.mark.parametrize("nbins", [50, 256])
def test_fp32_warp_specialised_iteration_matches_the_event_records(gpu, nbins):
    """FP32 iterations run the warp-specialised kernel (producer warps: channel
    choice, maps, densities, cuts; consumer warps: |M|^2).  Against the
    per-event records of the one-event-per-thread path for the same events:
    the weights (from the weights pass) agree to FP32 rounding (the kernels
    evaluate the same amplitudes in different orders of operations: with 50
    bins the consumers keep each event's row spinors in shared memory, with
    256 bins that memory goes to the histograms and they recompute the rows
    as the one-event-per-thread path does), the launch's sums are the sums of
    its weights, and the bin counts of all 17 grid dimensions are identical."""
    itg = W.gg_ttbarg_mc()
    edges = random_grid(17, nbins, 12).astype(np.float32).astype(np.float64)
    n = 60000
    v = make_vegas(M.MC_FP32_KAHAN, edges, iteration=1, seed=6)
    rec = torch.empty((n, M.REC_STRIDE), dtype=torch.float64, device="cuda")
    M.mc_debug_events(v, itg, gpu, 0, n, rec)
    wd = torch.empty(n, dtype=torch.float64, device="cuda")
    r = M.mc_vegas_iterate_weights(v, itg, gpu, n, wd)
    _, cnt = M.mc_vegas_get_hist(v)
    alpha, wch = M.mc_vegas_get_channels(v)
    v.free()
    g = rec.cpu().numpy()
    w = g[:, R["W"]]
    ws = wd.cpu().numpy()
    assert np.array_equal(ws != 0, w != 0) and r.n_nonzero == np.count_nonzero(w)
    nz = w != 0
    e = np.abs(ws[nz] / w[nz] - 1)
    assert np.median(e) < 1e-6 and e.max() < 1e-3, (np.median(e), e.max())
    assert abs(r.sum - math.fsum(ws)) <= 1e-12 * abs(r.sum)
    assert abs(r.sum2 - math.fsum(ws * ws)) <= 1e-12 * r.sum2
    ch = g[:, R["CHANNEL"]].astype(int)
    ref = np.zeros((17, nbins), dtype=np.int64)
    for d in range(7):
        gd = np.where(d < 2, d, 2 + 5 * ch + (d - 2))
        np.add.at(ref, (gd, g[:, R["BIN"] + d].astype(int)), 1)
    assert np.array_equal(cnt, ref)
    dens = g[:, R["DENS"]:R["DENS"] + 3]
    pden = dens[nz] @ alpha
    wref = (ws[nz, None] ** 2 * dens[nz] / pden[:, None]).sum(axis=0) / n
    assert np.max(np.abs(wch / wref - 1)) < 1e-5


def test_adaptation_and_alpha_update(gpu):
    """From uniform grids and equal channel probabilities, FP32: the
    integral agrees with the hierarchical single-channel integrand's, the
    alpha update moves weight to the initial-state-radiation channel, and
    the variance per event ends below the single channel's."""
    n = 400_000
    res = {}
    for name, itg in (("mc", W.gg_ttbarg_mc()), ("7d", W.gg_ttbarg_7d())):
        v = M.mc_vegas_init(itg.ndim(), 50, 21, M.MC_FP32_KAHAN)
        est = []
        for it in range(10):
            r = M.mc_vegas_iterate(v, itg, gpu, n)
            mean = r.sum / r.n
            var = (r.sum2 / r.n - mean * mean) / (r.n - 1)
            if it >= 5:
                est.append((mean, var))
            if name == "mc":
                a, w = M.mc_vegas_get_channels(v)
                M.mc_vegas_set_channels(v, M.mc_channel_update(a, w))
            M.mc_vegas_refine(v)
        if name == "mc":
            res["alpha"] = M.mc_vegas_get_channels(v)[0]
        inv = sum(1 / s2 for _, s2 in est)
        res[name] = (sum(m / s2 for m, s2 in est) / inv, math.sqrt(1 / inv), (r.sum2 / r.n) / mean ** 2 - 1)
        v.free()
    print(f"\nthree-channel {res['mc']} alpha {res['alpha']}; hierarchical {res['7d']}")
    assert abs(res["mc"][0] - res["7d"][0]) < 4 * math.hypot(res["mc"][1], res["7d"][1])
    assert res["alpha"][0] > 0.5
    assert res["mc"][2] < res["7d"][2]


def test_unweighted_three_channel_sample(gpu, oracle_pdf):
    """Unweighting (w > r w_max) of the three-channel process in FP64: the
    accepted set and the lab-frame records against the oracle."""
    edges = random_grid(17, 50, 9)
    n = 4000
    v = make_vegas(M.MC_FP64, edges, iteration=1, seed=3)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    r = M.mc_vegas_iterate_weights(v, W.gg_ttbarg_mc(), gpu, n, w)
    ev = torch.zeros((n, M.EVENT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    nacc = M.mc_unweight(v, W.gg_ttbarg_mc(), gpu, w, n, 0.03 * r.wmax, ev, n)
    torch.cuda.synchronize()
    got = M.events_from_bytes(ev[:nacc].cpu().numpy().tobytes())
    v.free()
    O.set_channel_alpha(ALPHA)
    wo, wmax_o, _, _ = O.unweight_events(W.gg_ttbarg_mc(), oracle_pdf, edges, M.MC_FP64, 3, 1, 0, 0, n, cap=0)
    _, _, evo, nacc_o = O.unweight_events(W.gg_ttbarg_mc(), oracle_pdf, edges, M.MC_FP64, 3, 1, 0, 0, n,
                                          wmax=0.03 * wmax_o)
    O.set_channel_alpha([1 / 3, 1 / 3, 1 / 3])
    assert nacc > 50
    ig, io = [int(e) for e in got["event"]], [e.event for e in evo]
    r_acc = O.acceptance_uniforms(3, 1, 0, 0, n)
    for i in set(ig) ^ set(io):  # only at the threshold, within FP64 rounding of the two w_max
        assert abs(wo[i] - r_acc[i] * 0.03 * wmax_o) <= 1e-11 * wo[i], i
    rec_o = {e.event: e for e in evo}
    for a in got:
        b = rec_o.get(int(a["event"]))
        if b is None:
            continue
        pb = np.array([list(q) for q in b.p])
        assert a["proc"] == M.MC_GG_TTBARG_MC and a["nout"] == 3
        assert np.max(np.abs(a["p"] - pb)) <= 1e-12 * pb[:2, 0].sum()


def test_argument_checks(gpu):
    v = M.mc_vegas_init(17, 50, 0, M.MC_FP32_KAHAN)
    with pytest.raises(M.McError):
        M.mc_vegas_set_channels(v, [0.0, 0.0, 0.0])
    with pytest.raises(M.McError):
        M.mc_vegas_set_channels(v, [-0.1, 0.6, 0.5])
    itg = W.gg_ttbarg_mc()
    itg.ptcut_g = 0.0
    with pytest.raises(M.McError):
        M.mc_vegas_iterate(v, itg, gpu, 1000)
    with pytest.raises(M.McError):
        M.mc_vegas_iterate(v, W.gg_ttbarg_7d(), gpu, 1000)  # 7 dimensions against a 17-dimension grid
    v.free()
