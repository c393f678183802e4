"""The flow's online training step split across devices (mc_flow_step_sample,
mc_flow_step_grads, mc_flow_step_apply; host side in shard.train_flow_sharded).

* With one rank the three calls are exactly one mc_flow_train step: the
  parameters after it are bitwise the same.
* Two ranks, emulated on one GPU by two flows with the same parameters and
  seed, each sampling half of the step's batch (their own events of the same
  Philox stream): the sum of their sums of w equals the whole batch's, and
  the sum of their gradients (each normalised by the total) equals the whole
  batch's gradient up to the FP32 summation order of the weight-gradient
  products (bars below); after the Adam step both ranks hold identical
  parameters, equal to the one-rank step except where a gradient component
  within rounding of zero takes the other sign of Adam's first step (+-lr).
"""
import numpy as np
import pytest

from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import shard
from paper_2302_03343_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D, L, K, BATCH, LR = 7, 6, 32, 8192, 1e-3


@pytest.fixture(scope="module")
def gpu(pdf_grid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    M.lib()
    torch.cuda.init()
    return M.mc_pdf_load(pdf_grid)


def make_flow(init):
    return M.mc_flow_create(D, L, K, init, BATCH, seed=5)


def trained_init(gpu):
    """Parameters after a few ordinary steps (every layer then has gradients)."""
    f = make_flow(W.flow_init_params(D, L=L, K=K, seed=2))
    M.mc_flow_train(f, W.gg_ttbarg_7d(), gpu, 3, BATCH, LR, losses=False)
    p = M.mc_flow_get_params(f)
    f.free()
    return p


def flat_params(f):
    return M.pack_flow_params(M.mc_flow_get_params(f))


def test_one_rank_step_equals_train_step(gpu):
    init = trained_init(gpu)
    itg = W.gg_ttbarg_7d()
    a, b = make_flow(init), make_flow(init)
    M.mc_flow_train(a, itg, gpu, 2, BATCH, LR, losses=False)
    shard.train_flow_sharded(b, itg, gpu, 2, BATCH, LR, rank=0, world=1)
    torch.cuda.synchronize()
    assert np.array_equal(flat_params(a), flat_params(b))
    a.free()
    b.free()


def test_two_ranks_equal_one(gpu):
    init = trained_init(gpu)
    itg = W.gg_ttbarg_7d()
    ref, r0, r1 = make_flow(init), make_flow(init), make_flow(init)
    n = M.mc_flow_grad_count(ref)
    g_ref = torch.empty(n, dtype=torch.float32, device="cuda")
    g0, g1 = torch.empty_like(g_ref), torch.empty_like(g_ref)
    w_ref = M.mc_flow_step_sample(ref, itg, gpu, 0, BATCH)
    M.mc_flow_step_grads(ref, w_ref, g_ref)
    (f0, c0), (f1, c1) = shard.shard_range(BATCH, 0, 2), shard.shard_range(BATCH, 1, 2)
    w0 = M.mc_flow_step_sample(r0, itg, gpu, f0, c0)
    w1 = M.mc_flow_step_sample(r1, itg, gpu, f1, c1)
    wtot = w0 + w1
    assert abs(wtot / w_ref - 1) < 1e-12
    M.mc_flow_step_grads(r0, wtot, g0)
    M.mc_flow_step_grads(r1, wtot, g1)
    g = g0 + g1
    torch.cuda.synchronize()
    gr, gs = g_ref.double(), g.double()
    cos = float(torch.dot(gr, gs) / (gr.norm() * gs.norm()))
    rel = float((gs - gr).norm() / gr.norm())
    print(f"\ntwo ranks vs one: gradient cosine {cos:.9f}, relative difference {rel:.2e}")
    assert cos > 0.99999 and rel < 1e-4
    for f, grads in ((ref, g_ref), (r0, g), (r1, g)):
        M.mc_flow_step_apply(f, grads, LR)
    torch.cuda.synchronize()
    p_ref, p0, p1 = flat_params(ref), flat_params(r0), flat_params(r1)
    assert np.array_equal(p0, p1)
    d = np.abs(p0.astype(np.float64) - p_ref)
    assert np.max(d) <= 2.0 * LR * 1.001
    assert np.count_nonzero(d > 1e-6) <= 1e-3 * d.size
    for f in (ref, r0, r1):
        f.free()
