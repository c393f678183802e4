"""One VEGAS iteration split across processes (one per GPU).

The events of an iteration are independent and each is addressed by its
Philox counter, so rank r of W evaluates the contiguous range
shard_range(n, r, W) with mc_vegas_iterate_shard, and one all-reduce of the
iteration's sums and histograms (a few KB) makes every rank's state that of
the whole iteration: the estimate equals the single-device one up to the
order of the additions, the bin counts exactly, and mc_vegas_refine then
yields the same grid on every rank without a broadcast (thesis Sec. VEGAS:
the estimate, its variance and the refinement histogram are sums over the
iteration's events).
"""
import numpy as np

from . import mcint as M


def shard_range(n, rank, world):
    """(first, count) of rank `rank`'s events: contiguous, sizes differ by at most one."""
    if not (0 <= rank < world):
        raise ValueError("rank outside the world")
    base, extra = divmod(int(n), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def allreduce_iteration(sums, hist_w2, hist_n, device=None):
    """Adds the ranks' iteration sums and histograms over the default process
    group (wmax by maximum): sums is a dict with sum, sum2, n, n_nonzero,
    n_bad and wmax; the histograms are [ndim][nbins] arrays (FP64 sums of w^2
    and event counts).  Returns the combined (sums, hist_w2, hist_n)."""
    import torch
    import torch.distributed as dist
    f = torch.tensor([sums["sum"], sums["sum2"]], dtype=torch.float64, device=device)
    i = torch.tensor([sums["n"], sums["n_nonzero"], sums["n_bad"]], dtype=torch.int64, device=device)
    m = torch.tensor([sums["wmax"]], dtype=torch.float64, device=device)
    w2 = torch.as_tensor(np.ascontiguousarray(hist_w2, dtype=np.float64)).to(device)
    cnt = torch.as_tensor(np.ascontiguousarray(hist_n, dtype=np.int64)).to(device)
    for t in (f, i, w2, cnt):
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    f, i, m = f.cpu().tolist(), i.cpu().tolist(), m.cpu().tolist()
    out = {"sum": f[0], "sum2": f[1], "n": i[0], "n_nonzero": i[1], "n_bad": i[2], "wmax": m[0]}
    counts = cnt.cpu().numpy()
    if counts.max(initial=0) > np.iinfo(np.uint32).max:
        raise OverflowError("bin count beyond 2^32 - 1")
    return out, w2.cpu().numpy(), counts.astype(np.uint32)


def iterate_sharded(v, itg, pdf, n, rank, world, stream=None, device=None):
    """This rank's part of an n-event iteration, combined over all ranks: the
    handle's histograms become the whole iteration's, and the returned dict
    holds the whole iteration's sums.  Every rank calls it with the same n."""
    first, count = shard_range(n, rank, world)
    r = M.mc_vegas_iterate_shard(v, itg, pdf, first, count, stream)
    w2, cnt = M.mc_vegas_get_hist(v)
    sums = {"sum": r.sum, "sum2": r.sum2, "n": r.n, "n_nonzero": r.n_nonzero, "n_bad": r.n_bad, "wmax": r.wmax}
    if world > 1:
        sums, w2, cnt = allreduce_iteration(sums, w2, cnt, device)
        M.mc_vegas_set_hist(v, w2, cnt)
    return sums


# ---- the flow's online training split across processes (data parallel).
# The loss L = -sum_i w_i log q(x_i) / sum_i w_i is a sum over the batch's
# events divided by the sum of their weights, so with every rank holding the
# same parameters the step needs two all-reduces: one double (the sum of w,
# before differentiating, so each rank's part is normalised by the total)
# and the gradient (after); every rank then takes the same Adam step.

def allreduce_sum(value, device=None):
    """The sum over the default process group of one float (itself alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def allreduce_grads_(grads):
    """In-place SUM of a gradient tensor over the default process group."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(grads, op=dist.ReduceOp.SUM)
    return grads


def train_flow_sharded(f, itg, pdf, steps, batch, lr, rank, world, stream=None, device=None):
    """`steps` online training steps of the flow f with each batch split over
    the ranks (rank r samples the events shard_range(batch, r, world) of the
    step's batch).  Every rank calls it with the same arguments but its rank;
    afterwards every rank's flow holds the same parameters."""
    import torch
    grads = torch.empty(M.mc_flow_grad_count(f), dtype=torch.float32, device=device or "cuda")
    first, count = shard_range(batch, rank, world)
    for _ in range(steps):
        wsum = allreduce_sum(M.mc_flow_step_sample(f, itg, pdf, first, count, stream), device)
        M.mc_flow_step_grads(f, wsum, grads, stream)
        if world > 1:
            if stream is not None:
                stream.synchronize()
            allreduce_grads_(grads)
        M.mc_flow_step_apply(f, grads, lr, stream)
