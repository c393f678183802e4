"""The benchmark configurations at their stated sizes against the oracle.

* p p -> t tbar, plain FP64 VEGAS (4 dims, 50 bins, 10 iterations x 1e6
  events, seed 0, uniform starting grid) through mc_integrate: the combined
  integral within 1e-10 and its standard error within 1e-8 of the oracle's
  run of the same configuration, and the closed-form cross section of the
  master formula (thesis eq. mc_master_formula) within 3 standard errors.
* g g -> t tbar g in FP32 mode, one full iteration of 1e7 events on a grid
  the oracle adapted: bin counts bit-exact, the integral's relative error
  against the FP64 oracle at identical points stated and bounded, and the
  per-event error statistics over the first 2e5 events.

The oracle's values for the full sizes are stored in tests/golden/ (written
by tests/golden/make_golden.py, which calls only the oracle); the per-event
sample is evaluated by the oracle here.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def gpu(pdf_grid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    M.lib()
    torch.cuda.init()
    return M.mc_pdf_load(pdf_grid)


def test_c2_pp_ttbar_fp64_at_config_size(gpu):
    g = golden("c2_pp_ttbar.json")
    p = g["params"]
    res, per = M.mc_integrate(W.pp_ttbar(), gpu, p["niter"], p["nevents"], nbins=p["nbins"], seed=p["seed"],
                              gid=p["gid"], prec=M.MC_FP64, alpha=p["alpha"])
    ref = g["oracle"]
    print(f"\nC2 GPU {res.mean:.10e} +- {res.sigma:.4e} pb, oracle {ref['mean_pb']:.10e} +- {ref['sigma_pb']:.4e}, "
          f"closed form {g['closed_form']['sigma_pb']:.10e}; {res.gpu_ms:.1f} ms")
    assert res.n_iter == p["niter"] and res.status == 0
    assert abs(res.mean - ref["mean_pb"]) <= 1e-10 * abs(ref["mean_pb"])
    assert abs(res.sigma - ref["sigma_pb"]) <= 1e-8 * ref["sigma_pb"]
    for i, r in enumerate(per):
        m = r.sum / r.n
        assert abs(m - ref["per_iteration"][i][0]) <= 1e-10 * abs(m)
    assert abs(res.mean - g["closed_form"]["sigma_pb"]) < 3 * res.sigma


def test_c3_full_iteration_against_fp64_oracle(gpu, oracle_pdf):
    g = golden("c3_ggttg_iteration.json")
    p = g["params"]
    edges = np.array(g["edges"])
    itg = W.gg_ttbarg()
    n = p["nevents"]
    v = M.mc_vegas_init(14, p["nbins"], p["seed"], M.MC_FP32_KAHAN)
    M.mc_vegas_set_grid(v, edges)
    M.mc_vegas_set_iteration(v, p["iteration"])
    M.mc_vegas_set_gid(v, p["gid"])
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    r = M.mc_vegas_iterate_weights(v, itg, gpu, n, w)
    _, cnt = M.mc_vegas_get_hist(v)
    ref = g["oracle"]
    np.testing.assert_array_equal(cnt, np.array(ref["hist_n"], dtype=np.uint32))
    rel_int = (r.sum - ref["sum"]) / ref["sum"]
    k = 200_000
    w_o = O.weights(itg, oracle_pdf, edges, M.MC_FP32_KAHAN, p["seed"], p["iteration"], p["gid"], 0, k)
    w_g = w[:k].cpu().numpy()
    both = (w_o != 0) & (w_g != 0)
    flips = int(np.count_nonzero((w_o != 0) != (w_g != 0)))
    e = np.abs(w_g[both] - w_o[both]) / np.abs(w_o[both])
    print(f"\nC3 FP32 iteration of {n} events: integral rel. error {rel_int:.3e}, in cuts {r.n_nonzero} "
          f"(oracle {ref['n_nonzero']}), w_max rel. {(r.wmax - ref['wmax']) / ref['wmax']:.2e}; per event "
          f"(first {k}): median {np.median(e):.2e} p99 {np.quantile(e, .99):.2e} max {e.max():.2e}, flips {flips}")
    assert abs(rel_int) < 1e-5
    assert abs(r.n_nonzero - ref["n_nonzero"]) <= n // 10000
    assert np.median(e) < 1e-5 and np.quantile(e, 0.99) < 1e-3
    assert flips <= k // 1000
    v.free()
