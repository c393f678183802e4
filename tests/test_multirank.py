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
