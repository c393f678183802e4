"""The allocation-free iteration entry point (mc_vegas_iterate_noalloc).

Some callers cannot allocate device memory while they run: code whose device
memory belongs to another pool that has reserved the device, and
latency-critical loops where a cudaMalloc/cudaFree would synchronise the
device.  The entry point keeps its only scratch (the per-block partial sums) in
a static device array and writes to buffers the caller owns.  This test calls
it through the C ABI twice in a row (two iterations, so the second call runs
over the scratch the first one left behind) and checks each call against the
ordinary mc_vegas_iterate on the same iteration: identical bin counts, sums
within the FP64 tolerance of the other tests (1e-12 relative), histograms
within 1e-10 (FP64 mode) or 1e-5 (FP32 mode, FP32 per-block histograms).  The file is collected last so a failure here cannot hide
failures elsewhere.
"""
import numpy as np
import pytest

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


# blocks = 0: the library picks the grid; 7: a caller's small grid; MC_NOALLOC_MAX_BLOCKS:
# the largest grid the scratch holds (for the warp-specialised FP32 gg -> ttg kernel, sized
# for one block per SM, that is many more blocks than SMs, most of them without events).
# The Philox counter of an event does not depend on the grid, so every shape must agree with
# mc_vegas_iterate.
@pytest.mark.parametrize("itg,prec,n,blocks", [(W.pp_ttbar(), M.MC_FP64, 30000, 0),
                                               (W.pp_ttbar(), M.MC_FP64, 30000, 7),
                                               (W.pp_ttbar(), M.MC_FP64, 30000, M.MC_NOALLOC_MAX_BLOCKS),
                                               (W.gg_ttbarg(), M.MC_FP32_KAHAN, 200000, 0),
                                               (W.gg_ttbarg(), M.MC_FP32_KAHAN, 200000, 7),
                                               (W.gg_ttbarg(), M.MC_FP32_KAHAN, 200000, M.MC_NOALLOC_MAX_BLOCKS),
                                               (W.pp_ttbarj(), M.MC_FP32_KAHAN, 30000, 0)])
def test_noalloc_matches_iterate_on_two_calls(gpdf, itg, prec, n, blocks):
    nd, nb, seed, gid = itg.ndim(), 50, 21, 3
    rng = np.random.default_rng(1)
    edges = np.sort(np.concatenate([np.zeros((nd, 1)), rng.uniform(size=(nd, nb - 1)), np.ones((nd, 1))], axis=1),
                    axis=1)
    dev = torch.device("cuda")
    e64 = torch.tensor(edges, dtype=torch.float64, device=dev)
    e32 = e64.float()
    hw2 = torch.zeros((nd, nb), dtype=torch.float64, device=dev)
    hn = torch.zeros((nd, nb), dtype=torch.int32, device=dev)
    sums = torch.zeros(8, dtype=torch.float64, device=dev)
    ref = M.mc_vegas_init(nd, nb, seed, prec)
    M.mc_vegas_set_grid(ref, edges)
    M.mc_vegas_set_gid(ref, gid)
    for it in (5, 6):
        hw2.zero_()
        hn.zero_()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        M.mc_vegas_iterate_noalloc(itg, gpdf, nd, nb, e64, e32, prec, seed, it, gid, n, blocks, hw2, hn, sums)
        torch.cuda.synchronize()
        if it == 6:  # after the first call (which may load the kernels' code): no device memory taken
            assert torch.cuda.mem_get_info()[0] == free0
        s = sums.cpu().numpy()
        counts = s.view(np.int64)[5:8]
        M.mc_vegas_set_iteration(ref, it)
        r = M.mc_vegas_iterate(ref, itg, gpdf, n)
        w2_ref, n_ref = M.mc_vegas_get_hist(ref)
        total, total2 = s[0] + s[1], s[2] + s[3]
        assert abs(total - r.sum) <= 1e-12 * abs(r.sum)
        assert abs(total2 - r.sum2) <= 1e-12 * abs(r.sum2)
        assert s[4] == r.wmax
        assert counts[0] == r.n_nonzero and counts[1] + counts[2] == r.n_bad
        np.testing.assert_array_equal(hn.cpu().numpy().astype(np.uint32), n_ref)
        nz = w2_ref > 0
        # FP32 mode sums w^2 per block in FP32 shared-memory atomics (order-dependent rounding)
        htol = 1e-10 if prec == M.MC_FP64 else 1e-5
        assert np.max(np.abs(hw2.cpu().numpy()[nz] - w2_ref[nz]) / w2_ref[nz]) < htol
        M.mc_vegas_refine(ref, 1.5)  # clears the reference histograms; keep its grid fixed
        M.mc_vegas_set_grid(ref, edges)
    ref.free()


def test_noalloc_rejects_oversized_launch(gpdf):
    itg = W.gauss(4)
    dev = torch.device("cuda")
    e64 = torch.tensor(W.uniform_grid(4, 10), dtype=torch.float64, device=dev)
    hw2 = torch.zeros((4, 10), dtype=torch.float64, device=dev)
    hn = torch.zeros((4, 10), dtype=torch.int32, device=dev)
    sums = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(M.McError) as e:
        M.mc_vegas_iterate_noalloc(itg, None, 4, 10, e64, None, M.MC_FP64, 0, 0, 0, 1000,
                                   M.MC_NOALLOC_MAX_BLOCKS + 1, hw2, hn, sums)
    assert "MC_NOALLOC_MAX_BLOCKS" in str(e.value)


def test_noalloc_rejects_unsupported_input(gpdf):
    """The three-channel process needs a VEGAS handle (its channel probabilities
    and update sums), and the Gaussian kernels stop at 16 dimensions: both are
    refused with EINVAL and a message that says why."""
    dev = torch.device("cuda")
    for itg, nd in ((W.gg_ttbarg_mc(), 17), (W.gauss(17), 17)):
        e64 = torch.tensor(W.uniform_grid(nd, 10), dtype=torch.float64, device=dev)
        hw2 = torch.zeros((nd, 10), dtype=torch.float64, device=dev)
        hn = torch.zeros((nd, 10), dtype=torch.int32, device=dev)
        sums = torch.zeros(8, dtype=torch.float64, device=dev)
        with pytest.raises(M.McError) as e:
            M.mc_vegas_iterate_noalloc(itg, gpdf, nd, 10, e64, e64.float(), M.MC_FP64, 0, 0, 0, 1000, 0, hw2, hn,
                                       sums)
        assert e.value.code == M.MC_EINVAL
        assert ("MC_GG_TTBARG_MC" in str(e.value)) == (itg.proc == M.MC_GG_TTBARG_MC)
