"""bench.py's N > 1 path on CPU: two ranks as gloo processes (one process
per GPU on a GPU machine, over NCCL).  Every rank runs its own integration (a
replica with its own Philox seed) with no data-path collective; the job's
time is the slowest rank's (a MAX all-reduce after a barrier) and its rate
counts the events of all ranks.  The reference arm prints from rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_2302_03343_b300 import shard  # noqa: E402
from paper_2302_03343_b300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.ranks_barrier()
        slowest = bench.max_over_ranks(10.0 + 3.0 * rank)  # rank r took 10 + 3 r ms
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        out.put((rank, slowest, seeds, bench.job_rate(1e7, 10, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, seeds, rate in res:
        assert slowest == 13.0  # the slowest rank's time on every rank
        assert seeds == [1000, 1001]  # independent Philox streams
        assert rate == pytest.approx(1e7 * 10 * 2 / 13e-3)


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    bench.ranks_barrier()
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 2e-3)


def test_reference_arm_prints_from_rank_zero_only(capsys):
    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""


# ---- one iteration split across ranks (paper_2302_03343_b300/shard.py): the
# oracle stands in for each rank's device (same Philox streams, same events)
N_SHARD = 30001  # odd: the two parts differ in size


def _shard_rank(rank, world, port, out):
    import numpy as np
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        itg, pdf = W.gg_ttbarg_7d(), O.Pdf(W.synthetic_pdf_grid(0))
        edges = W.uniform_grid(7, 50)
        first, count = shard.shard_range(N_SHARD, rank, world)
        r = O.iterate(itg, pdf, edges, W.FP64, 5, 2, 0, first, count)
        sums = {k: r[k] for k in ("sum", "sum2", "n", "n_nonzero", "wmax")}
        sums["n_bad"] = 0
        tot, w2, cnt = shard.allreduce_iteration(sums, r["hist_w2"], r["hist_n"])
        out.put((rank, (first, count), tot, np.asarray(w2), np.asarray(cnt)))
    finally:
        dist.destroy_process_group()


def test_sharded_iteration_over_gloo_equals_the_whole():
    import numpy as np
    import oracle as O
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t[1] for t in res] == [(0, 15001), (15001, 15000)]
    itg, pdf = W.gg_ttbarg_7d(), O.Pdf(W.synthetic_pdf_grid(0))
    edges = W.uniform_grid(7, 50)
    whole = O.iterate(itg, pdf, edges, W.FP64, 5, 2, 0, 0, N_SHARD)
    for _, _, tot, w2, cnt in res:  # every rank holds the whole iteration
        assert tot["n"] == N_SHARD and tot["n_nonzero"] == whole["n_nonzero"] and tot["wmax"] == whole["wmax"]
        assert abs(tot["sum"] / whole["sum"] - 1) < 1e-12 and abs(tot["sum2"] / whole["sum2"] - 1) < 1e-12
        assert np.array_equal(cnt, whole["hist_n"])
        assert np.allclose(w2, whole["hist_w2"], rtol=1e-12, atol=0)
        # the refinement of the combined histogram is the whole iteration's
        assert np.allclose(O.vegas_refine(edges, w2, 1.5), O.vegas_refine(edges, whole["hist_w2"], 1.5),
                           rtol=0, atol=1e-12)


def test_shard_ranges_cover_the_iteration():
    for n in (0, 1, 7, 1000, 10**7 + 3):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and sum(c for _, c in parts) == n
            assert all(parts[k][0] + parts[k][1] == parts[k + 1][0] for k in range(world - 1))
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


# ---- the flow's data-parallel training step (paper_2302_03343_b300/shard.py):
# the FP64 oracle flow stands in for each rank's device.  Two ranks holding
# half a batch each, with the sum of w and the gradients all-reduced, give
# the one-rank gradient and Adam step.
N_FLOW, D_FLOW, L_FLOW, K_FLOW = 301, 4, 2, 8


def _flow_setup():
    import numpy as np
    from oracle import flow as OF
    arrays = W.flow_init_params(D_FLOW, L=L_FLOW, K=K_FLOW, seed=3)
    rng = np.random.default_rng(11)
    for layer in arrays:  # a non-zero last layer, so every parameter has a gradient
        layer["W4"] = 0.05 * rng.standard_normal(layer["W4"].shape)
        layer["b4"] = 0.05 * rng.standard_normal(layer["b4"].shape)
    params = OF.params_from_arrays(arrays)
    x = torch.tensor(rng.uniform(0.02, 0.98, size=(N_FLOW, D_FLOW)), dtype=torch.float64)
    w = torch.tensor(rng.exponential(size=N_FLOW) + 0.1, dtype=torch.float64)
    return params, x, w


def _flat(grads):
    return torch.cat([g[k].flatten() for g in grads for k in sorted(g)])


def _flow_rank(rank, world, port, out):
    from oracle import flow as OF
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        params, x, w = _flow_setup()
        first, count = shard.shard_range(N_FLOW, rank, world)
        xr, wr = x[first:first + count], w[first:first + count]
        wtot = shard.allreduce_sum(float(wr.sum()))
        _, g = OF.loss_and_grads(params, xr, wr, K_FLOW)  # normalised by this share's sum of w
        flat = _flat(g) * (float(wr.sum()) / wtot)
        shard.allreduce_grads_(flat)
        out.put((rank, wtot, flat.numpy()))
    finally:
        dist.destroy_process_group()


def test_flow_data_parallel_step_over_gloo():
    import numpy as np
    from oracle import flow as OF
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_flow_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    params, x, w = _flow_setup()
    _, g_full = OF.loss_and_grads(params, x, w, K_FLOW)
    ref = _flat(g_full).numpy()
    assert np.count_nonzero(ref) > 0.5 * ref.size  # zero only through inactive ReLU units
    scale = np.max(np.abs(ref))
    for _, wtot, flat in res:
        assert abs(wtot / float(w.sum()) - 1) < 1e-14
        assert np.max(np.abs(flat - ref)) < 1e-12 * scale
    # the same Adam step on every rank, equal to the one-rank step
    def unflat(v):
        out_, k = [], 0
        for g in g_full:
            d = {}
            for key in sorted(g):
                n = g[key].numel()
                d[key] = torch.tensor(v[k:k + n], dtype=torch.float64).reshape(g[key].shape)
                k += n
            out_.append(d)
        return out_
    p_full = OF.adam_step(params, g_full, OF.adam_state(params), 1)
    for _, _, flat in res:
        p_rank = OF.adam_step(params, unflat(flat), OF.adam_state(params), 1)
        # a gradient component within rounding of zero may take either sign of
        # the first Adam step (+-lr); every other one takes the same step
        d = np.abs(_flat(p_rank).numpy() - _flat(p_full).numpy())
        assert np.max(d) <= 2e-3 + 1e-12
        assert np.count_nonzero(d > 1e-12) <= np.count_nonzero(np.abs(ref) < 1e-10 * scale)
