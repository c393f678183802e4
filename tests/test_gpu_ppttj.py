"""GPU: p p -> t tbar + parton (MC_PP_TTBARJ: gg, q qbar, q g, qbar g and the
beam-swapped channels) against the FP64 oracle (oracle/src/integrand.cpp and
the q qbar -> t tbar g diagrams of oracle/src/matrix_elements.cpp).

The GPU evaluates the light-quark channels from helicity amplitudes with
physical spinors for every crossing; the oracle from Dirac traces of
q qbar -> t tbar g, crossing and charge conjugation.  Bars: FP64 |M|^2 of
all seven channels with a median difference at 1e-14 and at most 1e-11 (two
formulations of the same amplitudes: spinor products against Dirac traces,
whose roundings part by a few 1e-12 where propagators nearly cancel), the
weights the same (relative to 1e-3 of the sample's largest weight where the
synthetic PDF interpolant crosses zero), sums within 1e-10, bin counts
bit-exact; FP32 per-event error statistics.
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


def gpu_records(gpdf, itg, prec, edges, k, iteration=0, seed=0):
    v = M.mc_vegas_init(7, edges.shape[1] - 1, seed, prec)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, iteration)
    out = torch.full((k, M.REC_STRIDE), float("nan"), dtype=torch.float64, device="cuda")
    M.mc_debug_events(v, itg, gpdf, 0, k, out)
    torch.cuda.synchronize()
    v.free()
    return out.cpu().numpy()


def test_fp64_channels_against_oracle(gpu, oracle_pdf):
    itg = W.pp_ttbarj()
    edges = random_grid(7, 50, 3)
    k = 1500
    g = gpu_records(gpu, itg, M.MC_FP64, edges, k, iteration=2, seed=5)
    recs = [O.event(itg, oracle_pdf, edges, M.MC_FP64, 5, 2, 0, ev) for ev in range(k)]
    ok = np.array([r.pass_ for r in recs]) == 1
    assert np.array_equal(g[:, R["PASS"]].astype(int) == 1, ok) and ok.sum() > k // 3
    me_o = np.array([[r.me2, r.me2_qq, *r.me2_x] for r in recs])[ok]
    me_g = np.concatenate([g[:, [R["ME2"], R["ME2_QQ"]]], g[:, R["ME2_X"]:R["ME2_X"] + 5]], axis=1)[ok]
    assert np.all(me_o > 0)
    d = np.abs(me_g / me_o - 1)
    print(f"\npp->ttj FP64 |M|^2 by channel: median {np.median(d, axis=0)}, max {d.max(axis=0)}")
    assert np.median(d) < 1e-14 and d.max() < 1e-11
    wo = np.array([r.weight for r in recs])
    wg = g[:, R["W"]]
    floor = 1e-3 * np.abs(wo).max()
    dw = np.abs(wg - wo) / np.maximum(np.abs(wo), floor)
    print(f"weights: median {np.median(dw):.1e} max {dw.max():.1e}")
    assert np.median(dw) < 1e-14 and dw.max() < 1e-11
    po = np.array([[list(r.p[i]) for i in range(2, 5)] for r in recs])[ok]
    pg = g[:, R["P"] + 8:R["P"] + 20].reshape(k, 3, 4)[ok]
    assert np.max(np.abs(pg - po)) < 1e-12 * 14000


def test_fp32_error_statistics(gpu, oracle_pdf):
    itg = W.pp_ttbarj()
    edges = random_grid(7, 50, 4)
    k = 1500
    g = gpu_records(gpu, itg, M.MC_FP32_KAHAN, edges, k, iteration=1, seed=6)
    wo = np.array([O.event(itg, oracle_pdf, edges, M.MC_FP32_KAHAN, 6, 1, 0, ev).weight for ev in range(k)])
    wg = g[:, R["W"]]
    both = (wo != 0) & (wg != 0)
    flips = np.count_nonzero((wo != 0) != (wg != 0))
    e = np.abs(wg[both] - wo[both]) / np.abs(wo[both])
    print(f"\npp->ttj FP32 per-event rel. error: median {np.median(e):.2e} p99 {np.quantile(e, .99):.2e} "
          f"max {e.max():.2e}; flips {flips}/{k}")
    assert flips <= 2
    assert np.median(e) < 1e-5 and np.quantile(e, 0.99) < 1e-2


def test_iteration_sums_and_histograms(gpu, oracle_pdf):
    itg = W.pp_ttbarj()
    edges = random_grid(7, 50, 8)
    n = 3000
    v = M.mc_vegas_init(7, 50, 9, M.MC_FP64)
    M.mc_vegas_set_grid(v, edges)
    r = M.mc_vegas_iterate(v, itg, gpu, n)
    w2, cnt = M.mc_vegas_get_hist(v)
    v.free()
    ref = O.iterate(itg, oracle_pdf, edges, M.MC_FP64, 9, 0, 0, 0, n)
    assert abs(r.sum - ref["sum"]) <= 1e-10 * abs(ref["sum"])
    assert abs(r.sum2 - ref["sum2"]) <= 1e-10 * abs(ref["sum2"])
    assert np.array_equal(cnt, ref["hist_n"])


def test_gluon_only_densities_reduce_to_gg(gpu, pdf_grid):
    """With the quark densities set to zero the process is gg -> t tbar g with
    the hierarchical generator, event by event (FP64)."""
    g = pdf_grid
    xf = g.xf.copy()
    for i, pid in enumerate(g.pids):
        if pid != 21:
            xf[:, :, i] = 0.0
    gp = M.mc_pdf_load(W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=xf, params=g.params))
    edges = random_grid(7, 50, 10)
    a = gpu_records(gp, W.pp_ttbarj(), M.MC_FP64, edges, 2000, seed=3)[:, R["W"]]
    b = gpu_records(gp, W.gg_ttbarg_7d(), M.MC_FP64, edges, 2000, seed=3)[:, R["W"]]
    assert np.count_nonzero(a) > 500
    assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) < 1e-13


def test_integration_runs_and_agrees_between_precisions(gpu):
    itg = W.pp_ttbarj()
    r64, _ = M.mc_integrate(itg, gpu, 4, 200_000, prec=M.MC_FP64, seed=2)
    r32, _ = M.mc_integrate(itg, gpu, 4, 200_000, prec=M.MC_FP32_KAHAN, seed=2)
    assert r64.mean > 0 and r32.mean > 0
    assert abs(r64.mean - r32.mean) < 4 * math.hypot(r64.sigma, r32.sigma), (r64.mean, r32.mean)


def test_fp32_iteration_matches_event_records(gpu):
    """The FP32 iteration runs the warp-specialised kernel (producer warps:
    kinematics, cuts, the seven luminosities; consumer warps: the seven
    |M|^2); its sums equal those of the per-event weights that the per-thread
    debug path records for the same events.  Both kernels run the same
    kinematics, luminosity and |M|^2 source, but the compiler may contract
    multiply-adds differently in the two, so a weight may differ in its last
    FP32 bits: the bar is FP32 rounding (measured: sums 2.6e-9 apart, the
    counts and the largest weight identical)."""
    itg = W.pp_ttbarj()
    edges = random_grid(7, 50, 11)
    n = 20000
    v = M.mc_vegas_init(7, 50, 13, M.MC_FP32_KAHAN)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, 3)
    r = M.mc_vegas_iterate(v, itg, gpu, n)
    _, cnt = M.mc_vegas_get_hist(v)
    v.free()
    g = gpu_records(gpu, itg, M.MC_FP32_KAHAN, edges, n, iteration=3, seed=13)
    w = g[:, R["W"]]
    assert abs(r.n_nonzero - np.count_nonzero(w)) <= 2 and r.n_nonzero > 0
    assert abs(r.wmax - w.max()) <= 1e-6 * w.max()
    assert abs(r.sum - w.sum()) <= 1e-6 * abs(w.sum())
    assert np.all(cnt.sum(axis=1) == n)
