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
