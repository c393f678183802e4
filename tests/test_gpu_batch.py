"""GPU: many integrands in one persistent launch (mc_batch_*).

Each integrand of the batch must reproduce, event for event, the
single-integrand path with the same seed, integrand id (gid = its index) and
iteration: identical bin counts, sums within 1e-12 (FP64) of
the weight scale (1e-4 for FP32: single events can carry ~1e-3 FP32
error and dominate the sum of squares), grids after refinement
within 1e-9 (FP64) or 1e-5 (FP32 block histograms).  The Gaussians integrate to their closed form.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpdf(pdf_grid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    torch.cuda.init()
    return M.mc_pdf_load(pdf_grid)


def small_batch(scale=0.01):
    itgs, counts = W.batch_configs(seed=0)
    return itgs, [max(1, int(c * scale)) for c in counts]


@pytest.mark.parametrize("prec", [M.MC_FP32_KAHAN, M.MC_FP64], ids=["fp32", "fp64"])
def test_batch_matches_single_path(gpdf, prec):
    itgs, counts = small_batch(0.002 if prec == M.MC_FP64 else 0.01)
    b = M.mc_batch_create(itgs, counts, gpdf, nbins=50, seed=7, prec=prec)
    singles = []
    for i, itg in enumerate(itgs):
        v = M.mc_vegas_init(itg.ndim(), 50, 7, prec)
        M.mc_vegas_set_gid(v, i)
        singles.append(v)
    for it in range(3):
        res = M.mc_batch_iterate(b, 1.5)
        for i, itg in enumerate(itgs):
            r = M.mc_vegas_iterate(singles[i], itg, gpdf, counts[i])
            hist_ref = M.mc_vegas_get_hist(singles[i])[1]
            M.mc_vegas_refine(singles[i], 1.5)
            assert res[i].n == r.n and res[i].n_nonzero == r.n_nonzero, (i, it)
            # the two kernels are compiled separately (FMA contraction may
            # differ): per-event agreement ~1e-15 in FP64, ~1e-7 in FP32; sums
            # can nearly cancel (negative PDF tails), so bound by the weight scale
            tol = 1e-12 if prec == M.MC_FP64 else 1e-4  # FP32 per-event errors reach ~1e-3 at worst
            scale = math.sqrt(r.n * r.sum2)
            assert abs(res[i].sum - r.sum) <= tol * scale, (i, it, res[i].sum, r.sum)
            assert abs(res[i].sum2 - r.sum2) <= tol * abs(r.sum2) + 1e-300
            # the two kernels may contract FMAs differently (weights agree to
            # ~1e-15) and sum histograms in different orders; refinement
            # amplifies that to ~1e-10 on the edges (FP64 histograms) or ~1e-6
            # (FP32 block histograms)
            assert abs(res[i].wmax - r.wmax) <= tol * abs(r.wmax)
            g_b = M.mc_batch_get_grid(b, i)
            g_s = M.mc_vegas_get_grid(singles[i])
            assert np.max(np.abs(g_b - g_s)) < (1e-9 if prec == M.MC_FP64 else 1e-5), (i, it)
            M.mc_vegas_set_grid(singles[i], g_b)  # continue both from the same grid
            assert hist_ref.sum() == itg.ndim() * counts[i]
    shape = M.mc_batch_shape(b)
    if prec == M.MC_FP64:
        assert shape["block"] in (64, 128, 256) and shape["events_per_thread"] in (2, 8, 32)
    else:  # warp-specialised batch kernel: 16 warps, tiles of 4, 16 or 64 events per thread
        assert shape["block"] == 512 and shape["events_per_thread"] in (4, 16, 64)
    assert shape["ntiles"] >= len(itgs)
    b.free()
    for v in singles:
        v.free()


def test_batch_many_gg_tiles_per_block(gpdf):
    """FP32 batch with enough gg -> t tbar g events that every block of the
    warp-specialised batch kernel runs several gg tiles in a row, whatever
    tile size the autotuner picks (at most 64 x 512 events): the ring of each
    block then reuses slots across tiles, end-marker slots included.  Every
    integrand matches the single-integrand path, as in the test above."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_gg = 4 * sms * 64 * 512  # four of the largest tiles per block
    itgs = [W.gg_ttbarg(sqrt_s=13000.0), W.gg_ttbarg_7d(sqrt_s=13000.0), W.gauss(8), W.gg_ttbarg(sqrt_s=7000.0)]
    counts = [n_gg // 2, n_gg // 4, 100000, n_gg // 4]
    b = M.mc_batch_create(itgs, counts, gpdf, nbins=50, seed=11, prec=M.MC_FP32_KAHAN)
    singles = []
    for i, itg in enumerate(itgs):
        v = M.mc_vegas_init(itg.ndim(), 50, 11, M.MC_FP32_KAHAN)
        M.mc_vegas_set_gid(v, i)
        singles.append(v)
    for it in range(2):
        res = M.mc_batch_iterate(b, 1.5)
        for i, itg in enumerate(itgs):
            r = M.mc_vegas_iterate(singles[i], itg, gpdf, counts[i])
            M.mc_vegas_refine(singles[i], 1.5)
            assert res[i].status == M.MC_OK and res[i].n == r.n and res[i].n_nonzero == r.n_nonzero, (i, it)
            scale = math.sqrt(r.n * r.sum2)
            assert abs(res[i].sum - r.sum) <= 1e-4 * scale, (i, it, res[i].sum, r.sum)
            M.mc_vegas_set_grid(singles[i], M.mc_batch_get_grid(b, i))
    shape = M.mc_batch_shape(b)
    assert shape["ntiles"] >= 4 * sms
    b.free()
    for v in singles:
        v.free()


def test_batch_first_iteration_against_oracle(gpdf, oracle_pdf):
    itgs, counts = small_batch(0.003)
    b = M.mc_batch_create(itgs, counts, gpdf, nbins=50, seed=0, prec=M.MC_FP64)
    res = M.mc_batch_iterate(b, 1.5)
    for i in (0, 4, 8, 12, 15):
        ref = O.iterate(itgs[i], oracle_pdf, W.uniform_grid(itgs[i].ndim(), 50), 0, 0, 0, i, 0, counts[i])
        assert abs(res[i].sum - ref["sum"]) <= 1e-10 * abs(ref["sum"]), i
        assert res[i].n_nonzero == ref["n_nonzero"]
    b.free()


def test_batch_gaussians_closed_form(gpdf):
    itgs = [W.gauss(d) for d in (4, 8, 12, 16)]
    counts = [200000, 300000, 400000, 500000]
    b = M.mc_batch_create(itgs, counts, None, nbins=50, seed=3, prec=M.MC_FP32_KAHAN)
    E = [[] for _ in itgs]
    S2 = [[] for _ in itgs]
    for _ in range(6):
        for i, r in enumerate(M.mc_batch_iterate(b, 1.5)):
            m = r.sum / r.n
            E[i].append(m)
            S2[i].append((r.sum2 / r.n - m * m) / (r.n - 1))
    for i, d in enumerate((4, 8, 12, 16)):
        mean, sigma, chi2 = O.combine(E[i], S2[i])
        exact = W.gauss_exact(d)
        assert abs(mean - exact) < 4 * sigma, (d, mean, exact, sigma)
    assert M.mc_batch_kernel_ms(b) > 0
    b.free()
