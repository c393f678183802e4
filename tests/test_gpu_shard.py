"""One iteration split into event ranges (mc_vegas_iterate_shard), as the
ranks of a multi-GPU run split it: the parts' sums and histograms add up to
the whole iteration's (bin counts exactly, sums to the order of the
additions), and the refinement of the added histograms (mc_vegas_set_hist)
gives the whole iteration's grid.  On one GPU the parts run one after the
other on separate handles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2302_03343_b300 import mcint as M  # noqa: E402
from paper_2302_03343_b300 import shard  # noqa: E402
from paper_2302_03343_b300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpdf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    return M.mc_pdf_load(W.synthetic_pdf_grid(0))


def _grid(ndim, seed):
    rng = np.random.default_rng(seed)
    e = np.sort(rng.uniform(0, 1, (ndim, 51)), axis=1)
    e[:, 0], e[:, -1] = 0.0, 1.0
    return e


def _handle(itg, prec, edges, seed=5, iteration=2):
    v = M.mc_vegas_init(itg.ndim(), edges.shape[1] - 1, seed, prec)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, iteration)
    return v


@pytest.mark.parametrize("name,prec", [("gg_ttbarg_7d", M.MC_FP64), ("gg_ttbarg", M.MC_FP32_KAHAN),
                                       ("ee_mumu", M.MC_FP64)])
def test_parts_add_up_to_the_whole(gpdf, name, prec):
    itg = getattr(W, name)()
    pdf = None if name == "ee_mumu" else gpdf
    edges = _grid(itg.ndim(), 3)
    n = 300007
    whole = _handle(itg, prec, edges)
    rw = M.mc_vegas_iterate(whole, itg, pdf, n)
    hw2, hn = M.mc_vegas_get_hist(whole)
    tot = dict(sum=0.0, sum2=0.0, n=0, nz=0, wmax=-np.inf)
    w2 = np.zeros_like(hw2)
    cnt = np.zeros_like(hn, dtype=np.int64)
    for rank in range(3):
        first, count = shard.shard_range(n, rank, 3)
        v = _handle(itg, prec, edges)
        r = M.mc_vegas_iterate_shard(v, itg, pdf, first, count)
        assert r.n == count and r.status in (M.MC_OK, M.MC_ENOCONV)
        a, b = M.mc_vegas_get_hist(v)
        w2 += a
        cnt += b
        tot["sum"] += r.sum
        tot["sum2"] += r.sum2
        tot["n"] += r.n
        tot["nz"] += r.n_nonzero
        tot["wmax"] = max(tot["wmax"], r.wmax)
        v.free()
    assert tot["n"] == n and tot["nz"] == rw.n_nonzero and tot["wmax"] == rw.wmax
    assert abs(tot["sum"] / rw.sum - 1) < 1e-12 and abs(tot["sum2"] / rw.sum2 - 1) < 1e-12
    assert np.array_equal(cnt, hn.astype(np.int64))
    assert np.allclose(w2, hw2, rtol=1e-6 if prec == M.MC_FP32_KAHAN else 1e-12, atol=0)
    # the refinement of the added histograms is the whole iteration's
    part = _handle(itg, prec, edges)
    M.mc_vegas_set_hist(part, w2, cnt.astype(np.uint32))
    M.mc_vegas_refine(part, 1.5)
    M.mc_vegas_refine(whole, 1.5)
    tol = 1e-6 if prec == M.MC_FP32_KAHAN else 1e-9  # FP32 block histograms add in launch order
    assert np.allclose(M.mc_vegas_get_grid(part), M.mc_vegas_get_grid(whole), rtol=0, atol=tol)
    part.free()
    whole.free()


def test_single_rank_helper_is_the_plain_iteration(gpdf):
    itg = W.gg_ttbarg_7d()
    edges = _grid(7, 4)
    a, b = _handle(itg, M.MC_FP64, edges), _handle(itg, M.MC_FP64, edges)
    r = M.mc_vegas_iterate(a, itg, gpdf, 100000)
    s = shard.iterate_sharded(b, itg, gpdf, 100000, 0, 1)
    assert s["n"] == r.n and s["n_nonzero"] == r.n_nonzero and s["sum"] == r.sum and s["sum2"] == r.sum2
    (wa, na), (wb, nb) = M.mc_vegas_get_hist(a), M.mc_vegas_get_hist(b)
    assert np.array_equal(na, nb)
    assert np.allclose(wa, wb, rtol=1e-12, atol=0)  # blocks add their partial histograms in any order
    a.free()
    b.free()


def test_argument_checks(gpdf):
    itg = W.gg_ttbarg_7d()
    v = _handle(itg, M.MC_FP64, _grid(7, 5))
    with pytest.raises(M.McError):
        M.mc_vegas_iterate_shard(v, itg, gpdf, -1, 10)
    with pytest.raises(M.McError):
        M.mc_vegas_iterate_shard(v, itg, gpdf, 2**62, 2**62)
    w2, n = M.mc_vegas_get_hist(v)
    w2[0, 0] = -1.0
    with pytest.raises(M.McError):
        M.mc_vegas_set_hist(v, w2, n)
    r = M.mc_vegas_iterate_shard(v, itg, gpdf, 10**12, 0)  # an empty part far along the stream
    assert r.n == 0 and r.sum == 0.0
    v.free()
