"""Benchmark of the per-event Monte Carlo cross-section path on B300.

Workload (one "step" = one VEGAS iteration = the whole hot path over one batch):
gg -> t tbar g at sqrt(s) = 13 TeV, RAMBO phase space (2 + 12 sampled
dimensions, 7 physical), gluon pT > 20 GeV and |eta| < 2.5, synthetic
LHAPDF-shaped PDF grid, FP32 helicity-amplitude |M|^2 with Kahan FP64
accumulation, 1e7 events per iteration, 50 VEGAS bins per dimension, each step
followed by the grid refinement.  Inputs are synthetic and seeded.

The line also carries "time_to_target": the GPU time to a 1e-3 relative
error on gg -> t tbar g in 7 sampled dimensions for plain FP64 VEGAS, FP32
VEGAS, FP32 three-channel sampling (per-channel grids, Kleiss-Pittau channel
weights) and FP32 + normalizing-flow sampling with VEGAS as its judge and
fallback (200 online training steps and the judge's VEGAS iteration
included; mc_integrate_flow), each run from scratch, with the variance per
event and the unweighting efficiency of each (the flow's from a separately
timed train-then-sample breakdown); "batch16": sixteen integrands of uneven
dimension and event count in one persistent launch per iteration (CUDA
graph, autotuned shape) against the sum of their single launches; and
"pdf_members": the multi-member PDF evaluation of the thesis's Table
tab:fktable (400 members, 11 flavours, 2415 x points) against HBM; and
"unweighting": unweighted event generation on the benchmark workload (weights
pass, device-side acceptance-rejection and export of the accepted events,
and the native LHE writer's throughput on them); and "samplers": RAMBO, the
hierarchical generator and three-channel sampling side by side (time per
iteration, variance per event, unweighting efficiency); and "pp_ttbarj": the
higher-multiplicity process p p -> t tbar + parton (all partonic channels);
"c2": plain FP64 VEGAS of p p -> t tbar at its configured size (10 x 1e6)
against the oracle's run and the closed-form cross section; "oracle_check":
one full 1e7-event FP32 iteration of the benchmark workload against the FP64
oracle at identical points (integral, bin counts, and per-event errors over
the CPU-baseline sample); "fma_peaks": the measured FP32 / FP64 FMA rates, the
roofline's denominator; "sharded": one integration split across the ranks.

The roofline's numerator is the algorithmic FLOP of the event counted by the
oracle with an operation-counting scalar (tests/golden/ggttg_opcount.json);
the kernel's executed FLOP (ncu) is reported beside it.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead (a
bounded sample of events per step on the host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2302_03343_b300 import workloads as W  # noqa: E402

EVENTS = 10_000_000
NBINS = 50
ALPHA = 1.5
WORKLOAD = ("gg->ttg 13 TeV, RAMBO 2+12 dims (7 physical), gluon pT>20 GeV |eta|<2.5, synthetic 100x40x11 "
            "PDF grid, FP32 helicity |M|^2 + Kahan FP64 sums, VEGAS 50 bins, 1e7 events/iteration")
METRIC = "events/sec and GPU time to 1e-3 rel. error: FP32+flow vs plain FP64 VEGAS"
# Executed FP32 floating-point operations per in-cut gg -> ttg event of the
# warp-specialised fused kernel (packed |M|^2 over 16 polarisation
# configurations, RAMBO, PDFs and the map of every event, in-cut or not),
# counted by ncu over one full-size launch of this workload as
# 2 ffma + fmul + fadd + 4 ffma2 + 2 fmul2 + 2 fadd2 (1.668e11 FLOP) divided by
# the launch's 8 049 117 in-cut events; see profiles/.  The roofline's
# numerator is the algorithmic count (ggttg_opcount.json); this one measures
# how busy the pipes are.
EXECUTED_FLOP_PER_EVENT = 20720.0
# DRAM bytes (read + write) of one launch of that kernel, from an ncu capture
# of this workload (0.46 MB read + 3.24 MB written; see profiles/).  Nothing
# per event reaches DRAM: the kernel reads the grid and the PDF grid and
# writes histograms and per-block partials.
TRAFFIC_BYTES = 3700480
FP32_LANES_PER_SM = 128
# FP32 FLOP per FP32 lane operation of that launch: its ncu counts give
# 2 ffma + fmul + fadd + 4 ffma2 + 2 fmul2 + 2 fadd2 = 1.668e11 FLOP over
# ffma + fmul + fadd + 2 (ffma2 + fmul2 + fadd2) = 1.032e11 lane operations;
# a multiply or an add alone does one FLOP in a slot that could do two, so
# the kernel's mix caps it at this fraction of the FMA peak.
FLOP_PER_LANE_OP = 1.668e11 / 1.032e11
# time to a target relative error (gg -> t tbar g, 7 sampled dimensions):
# FP32 + normalizing flow (6 coupling layers, 32 bins, 3 x 256 BF16 hidden
# units, Adam lr 1e-3, 200 training steps of 65536 events, then 1e7 events per
# iteration) against plain FP64 VEGAS (1e7 events per iteration, 50 bins)
TTT_TARGET = 1e-3
TTT_EVENTS = 10_000_000
TTT_MAX_ITER = 15
FLOW_LAYERS, FLOW_BINS, FLOW_STEPS, FLOW_BATCH, FLOW_LR = 6, 32, 200, 65536, 1e-3


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, device_index=0):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[0] == str(device_index):
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden(name):
    """Stored oracle values (tests/golden/, written by tests/golden/make_golden.py)."""
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def cpu_baseline(seconds=15.0):
    """The FP64 oracle as it stands, timed on the host cores over a bounded
    sample of the same workload: the first events of the stored g g -> t tbar g
    iteration (the oracle-adapted 50-bin grid, FP32-mode uniforms evaluated in
    FP64).  Returns the baseline and the oracle's weights of the sample, which
    the per-event check compares with the GPU's weights of the same events."""
    import oracle as O
    g = golden("c3_ggttg_iteration.json")
    p = g["params"]
    grid = W.synthetic_pdf_grid(0)
    pdf = O.Pdf(grid)
    itg = W.gg_ttbarg()
    edges = np.array(g["edges"])
    cores = os.cpu_count() or 1

    def run(first, n):
        return O.weights(itg, pdf, edges, 1, p["seed"], p["iteration"], p["gid"], first, n, nthreads=cores)

    # calibrate on samples of at least a second (thread start-up dominates
    # smaller ones), then time a sample of about `seconds`
    n0, dt, parts = 200 * cores, 0.0, []
    while True:
        t0 = time.perf_counter()
        parts = [run(0, n0)]
        dt = time.perf_counter() - t0
        if dt >= 1.0 or n0 >= 1 << 30:
            break
        n0 *= 4
    n = max(n0, int(n0 * seconds / max(dt, 1e-3)))
    t0 = time.perf_counter()
    parts.append(run(n0, n))
    dt = time.perf_counter() - t0
    return ({"value": n / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
             "sample": f"events {n0}..{n0 + n - 1} of one gg->ttg iteration (seed {p['seed']}, iteration "
                       f"{p['iteration']}, the oracle-adapted 50-bin grid, FP32-mode uniforms, FP64 oracle), "
                       f"{cores} threads, {dt:.1f} s"},
            np.concatenate(parts))


def run_reference(args, rank, world):
    if rank != 0:
        return
    base, _ = cpu_baseline(seconds=max(2.0, 60.0 / max(args.steps + args.warmup, 1)))
    # each step: a bounded sample of the same workload on all host cores
    import oracle as O
    grid = W.synthetic_pdf_grid(0)
    pdf = O.Pdf(grid)
    itg = W.gg_ttbarg()
    edges = W.uniform_grid(14, NBINS)
    cores = os.cpu_count() or 1
    n = max(1000, int(base["value"] * 5.0))
    for i in range(args.warmup):
        O.iterate(itg, pdf, edges, 1, 0, i, 0, 0, max(1000, n // 10), nthreads=cores)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        r = O.iterate(itg, pdf, edges, 1, 0, args.warmup + i, 0, 0, n, nthreads=cores)
        times.append(time.perf_counter() - t0)
        edges = O.vegas_refine(edges, r["hist_w2"], ALPHA)
    value = n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": n, "sample": "bounded CPU sample per step"},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} events per step, {cores} threads"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


# ---- one process per GPU (torchrun): every rank runs its own integration
# (a replica with its own Philox stream, weak scaling, no data-path
# collective); the job's time is the slowest rank's and its rate counts the
# events of all ranks.
def replica_seed(rank):
    """Philox seed of rank `rank`'s integration."""
    return 1000 + rank


def ranks_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value, device=None):
    """The largest of the ranks' values (the value itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, steps, world, total_ms):
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return units_per_rank_step * steps * world / (total_ms / 1e3)


def _combine(res):
    """Inverse-variance combination of per-iteration (mean, variance of the mean)."""
    w = [1.0 / v for _, v in res if v > 0]
    if not w:
        return 0.0, float("inf")
    mean = sum(m / v for m, v in res if v > 0) / sum(w)
    return mean, (1.0 / sum(w)) ** 0.5


def _iter_stats(r):
    mean = r.sum / r.n
    var = max(r.sum2 / r.n - mean * mean, 0.0) / (r.n - 1)
    return mean, var


def batch16(M, pdf, stream, iterations=10):
    """Sixteen integrands of uneven dimension and event count in one
    persistent launch per iteration, captured in a CUDA graph (autotuned
    block size and events per thread), against the sum of the sixteen
    single-integrand launches of the same events."""
    import torch
    itgs, counts = W.batch_configs(seed=0)
    b = M.mc_batch_create(itgs, counts, pdf, NBINS, seed=0, prec=M.MC_FP32_KAHAN)
    M.mc_batch_iterate(b, ALPHA, stream)  # first iteration builds the graph
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(iterations):
        M.mc_batch_iterate(b, ALPHA, stream)
    t1.record(stream)
    torch.cuda.synchronize()
    batch_ms = t0.elapsed_time(t1) / iterations
    shape = M.mc_batch_shape(b)
    b.free()
    single_ms = 0.0
    for i, (itg, n) in enumerate(zip(itgs, counts)):
        v = M.mc_vegas_init(itg.ndim(), NBINS, 0, M.MC_FP32_KAHAN)
        M.mc_vegas_set_gid(v, i)
        M.mc_vegas_iterate(v, itg, pdf, n, stream)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(iterations):
            M.mc_vegas_iterate(v, itg, pdf, n, stream)
            M.mc_vegas_refine(v, ALPHA, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        single_ms += s0.elapsed_time(s1) / iterations
        v.free()
    total = int(sum(counts))
    return {"integrands": len(itgs), "events_per_iteration": total, "ms_per_iteration": batch_ms,
            "events_per_s": total / (batch_ms / 1e3), "single_launches_ms_per_iteration": single_ms,
            "speedup_vs_single_launches": single_ms / batch_ms, "autotuned": shape}


PDF_MEMBERS, PDF_POINTS, PDF_Q = 400, 2415, 100.0
PDF_SWEEP = (10, 14, 18, 22, 26)  # log2 of the batch sizes of the single-set sweep


def pdf_sweep_inputs(n, seed=0):
    """n query points log-uniform inside the synthetic grid: x in [1e-7, 1],
    Q in [1.65, 1e4] GeV (Q^2 passed), from a seeded torch generator."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    u = torch.rand((2, n), generator=g, dtype=torch.float64, device="cuda")
    x = torch.pow(10.0, -7.0 * (1.0 - u[0]))
    q = 1.65 * torch.pow(1e4 / 1.65, u[1])
    return x.contiguous(), (q * q).contiguous()


def pdf_xfxq2_sweep(M, pdf, stream, reps=10):
    """The PDF-only benchmark of the thesis (Sec. "Software design and
    benchmarks": PDFFlow against LHAPDF over growing numbers of query
    points): all 11 flavours of the synthetic grid at 2^10 .. 2^26 random
    (x, Q) points, FP32 and FP64, each launch timed alone with CUDA events
    after an L2 flush.  Roofline: HBM, algorithmic bytes = 16 B of input and
    8 B per flavour of output per point (the grid itself stays in L2)."""
    import torch
    nfl = 11
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    hbm = peaks().get("hbm_gbs", 6400.0)
    out = {"workload": "synthetic 100 x 40 x 11 grid, all 11 flavours, random (x, Q) log-uniform in the grid",
           "bytes_per_point": 16 + 8 * nfl, "hbm_peak_gbs": hbm,
           "thesis_context": "PDFFlow's xfxQ2 over growing batches of query points against LHAPDF"}
    for name, prec in (("fp32", M.MC_FP32_KAHAN), ("fp64", M.MC_FP64)):
        rows = []
        for lg in PDF_SWEEP:
            n = 1 << lg
            x, q2 = pdf_sweep_inputs(n, seed=lg)
            res = torch.empty((n, nfl), dtype=torch.float64, device="cuda")
            for _ in range(2):
                M.mc_pdf_xfxq2(pdf, prec, n, x, q2, res, stream)
            times = []
            for _ in range(reps):
                flush_l2(flush)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                M.mc_pdf_xfxq2(pdf, prec, n, x, q2, res, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            gbs = n * (16 + 8 * nfl) / (ms / 1e3) / 1e9
            rows.append({"points": n, "ms": ms, "points_per_s": n / (ms / 1e3), "achieved_gbs": gbs,
                         "hbm_frac": gbs / hbm})
            del x, q2, res
        out[name] = rows
    return out


def pdf_members(M, stream, reps=20):
    """Multi-member PDF evaluation (thesis Table tab:fktable): all 11 flavours
    of 400 members at 2415 x points (log-spaced on [1e-7, 1], Q = 100 GeV) of
    a two-sub-grid synthetic set, FP32 and FP64, each launch timed alone with
    CUDA events after an L2 flush.  Roofline: HBM, algorithmic bytes = output
    + the four Q rows of every flavour and member the points touch + inputs."""
    import torch
    pset = W.synthetic_pdf_set(nmem=PDF_MEMBERS, seed=0)
    ps = M.mc_pdfset_load(pset)
    x = np.array([10.0 ** (-7.0 * (1.0 - i / (PDF_POINTS - 1))) for i in range(PDF_POINTS)])
    x[-1] = 1.0
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    qd = torch.full_like(xd, PDF_Q * PDF_Q)
    nfl = len(pset.pids)
    nx = len(pset.x[1])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    hbm = peaks().get("hbm_gbs", 6400.0)
    out = {"workload": f"{PDF_MEMBERS} members x {nfl} flavours x {PDF_POINTS} x points at Q = {PDF_Q:g} GeV, "
                       "2 sub-grids (b threshold), 100 x knots", "hbm_peak_gbs": hbm,
           "thesis_context": "PDFFlow on an Nvidia Titan V: 1.69 s for 400 members (LHAPDF CPU 3.63 s), "
                             "thesis Table tab:fktable"}
    for name, prec, dt, size in (("fp32", M.MC_FP32_KAHAN, torch.float32, 4), ("fp64", M.MC_FP64, torch.float64, 8)):
        res = torch.empty((PDF_MEMBERS, PDF_POINTS, nfl), dtype=dt, device="cuda")
        for _ in range(3):
            M.mc_pdfset_xfxq2(ps, prec, 0, PDF_MEMBERS, PDF_POINTS, xd, qd, res, stream)
        times = []
        for _ in range(reps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M.mc_pdfset_xfxq2(ps, prec, 0, PDF_MEMBERS, PDF_POINTS, xd, qd, res, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        nbytes = PDF_MEMBERS * PDF_POINTS * nfl * size + 4 * nx * nfl * PDF_MEMBERS * size + 2 * PDF_POINTS * 8
        out[name] = {"ms": ms, "values_per_s": PDF_MEMBERS * PDF_POINTS * nfl / (ms / 1e3),
                     "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (ms / 1e3) / 1e9,
                     "hbm_frac": nbytes / (ms / 1e3) / 1e9 / hbm}
    ps.free()
    return out


def unweighting(M, pdf, stream, edges, plain_ms, reps=3):
    """Unweighted events on the benchmark workload (gg -> ttg, FP32, 1e7
    events per iteration).  (1) On the grid the timed steps adapted: the
    weights pass (the fused kernel writing every weight), the
    acceptance-rejection with the iteration's own w_max and the export of the
    accepted events in the laboratory frame, each timed with CUDA events.
    (2) The native LHE writer alone on 2^19 exported events (w_max lowered
    to the weight quantile that accepts them), device batch to a temporary
    file, min(16, cores) formatting threads.  (3) mc_generate_lhe end to end
    from a uniform grid: 5 adapting iterations, then 3 iterations whose
    accepted events are written while the next one runs (host wall time)."""
    import torch
    itg = W.gg_ttbarg()
    n = EVENTS
    cap = n // 4
    v = M.mc_vegas_init(14, NBINS, 7000, M.MC_FP32_KAHAN)
    M.mc_vegas_set_grid(v, edges)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    ev = torch.empty((cap, M.EVENT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    wp_ms, uw_ms, eff, nacc = [], [], [], 0
    for i in range(reps + 1):
        r = M.mc_vegas_iterate_weights(v, itg, pdf, n, w, stream)
        nacc = M.mc_unweight(v, itg, pdf, w, n, r.wmax, ev, cap, stream)
        if i == 0:
            continue  # warm-up
        wp_ms.append(M.mc_vegas_kernel_ms(v))
        uw_ms.append(M.mc_unweight_ms(v))
        eff.append(nacc / n)
    wpm, uwm = statistics.median(wp_ms), statistics.median(uw_ms)
    out = {"workload": "gg->ttg FP32, 1e7 events per iteration on the adapted grid, w_max = the iteration's "
                       "largest weight", "efficiency": statistics.mean(eff), "accepted_per_iteration": nacc,
           "weights_pass_ms": wpm, "plain_pass_ms": plain_ms, "unweight_ms": uwm,
           "unweight_frac_of_weights_pass": uwm / wpm,
           "weighted_events_per_s_device": n / ((wpm + uwm) / 1e3),
           "accepted_events_per_s_device": nacc / ((wpm + uwm) / 1e3),
           "thesis_context": "MadFlow's RAMBO sampling: unweighting efficiency about 5% (thesis Sec. "
                             "\"Unweighted event exporter\")"}
    # (2) the writer on 2^19 events
    k = 1 << 19
    wq = torch.sort(w[w > 0]).values
    wlow = float(wq[max(0, wq.numel() - 2 * k)].item())
    nk = min(M.mc_unweight(v, itg, pdf, w, n, wlow, ev, cap, stream), k)
    threads = max(1, min(16, os.cpu_count() or 1))
    fd, path = tempfile.mkstemp(suffix=".lhe")
    os.close(fd)
    try:
        t0 = time.perf_counter()
        lhe = M.mc_lhe_open(path, itg, threads)
        M.mc_lhe_write_device(lhe, ev, nk, stream)
        written = lhe.close(r.sum / r.n, 0.0, r.wmax)
        t_lhe = time.perf_counter() - t0
        size = os.path.getsize(path)
        out["lhe_writer"] = {"threads": threads, "events": written, "bytes": size, "s": t_lhe,
                             "events_per_s": written / t_lhe, "MB_per_s": size / t_lhe / 1e6}
        # (3) end to end
        res, st = M.mc_generate_lhe(itg, pdf, path, ntrain=5, niter=3, nevents=n, nbins=NBINS, seed=11,
                                    prec=M.MC_FP32_KAHAN, alpha=ALPHA, threads=threads, stream=stream)
        out["generate_lhe"] = {"train_iterations": 5, "export_iterations": 3, "events_per_iteration": n,
                               "written": st.n_accepted, "efficiency": st.n_accepted / st.n_weighted,
                               "xsec_pb": res.mean, "xsec_rel_err": res.sigma / res.mean,
                               "device_ms": st.iterate_ms + st.unweight_ms, "wall_ms": st.wall_ms,
                               "weighted_events_per_s_wall": st.n_weighted / (st.wall_ms / 1e3),
                               "unweighted_events_per_s_wall": st.n_accepted / (st.wall_ms / 1e3),
                               "file_bytes": os.path.getsize(path)}
    finally:
        os.unlink(path)
    v.free()
    return out


def samplers(M, pdf, stream, iterations=10):
    """The three phase-space samplers of gg -> t tbar g side by side, FP32,
    1e7 events per iteration, each adapted for `iterations` iterations from
    a uniform grid (the three-channel sampler also updating its channel
    probabilities): the fused kernel's time per iteration (median of the
    last 7), the relative variance per event and the unweighting efficiency
    <w>/w_max of the last iteration, and their product variance x time, the
    cost of a given precision (thesis Sec. "Multi-channel Monte Carlo" and
    Sec. "Unweighted event exporter": RAMBO's flat sampling against
    channels that follow the peaks of |M|^2)."""
    out = {}
    for name, itg in (("rambo_14d", W.gg_ttbarg()), ("hierarchical_7d", W.gg_ttbarg_7d()),
                      ("three_channel", W.gg_ttbarg_mc())):
        v = M.mc_vegas_init(itg.ndim(), NBINS, 2000, M.MC_FP32_KAHAN)
        ms = []
        for i in range(iterations):
            r = M.mc_vegas_iterate(v, itg, pdf, EVENTS, stream)
            if itg.proc == W.GG_TTBARG_MC:
                a, w = M.mc_vegas_get_channels(v)
                M.mc_vegas_set_channels(v, M.mc_channel_update(a, w, 0.5, 0.02))
            M.mc_vegas_refine(v, ALPHA, stream)
            if i >= iterations - 7:
                ms.append(M.mc_vegas_kernel_ms(v))
        mean = r.sum / r.n
        rv = (r.sum2 / r.n) / (mean * mean) - 1.0
        kms = statistics.median(ms)
        out[name] = {"kernel_ms": kms, "rel_var_per_event": rv, "unweighting_eff": mean / r.wmax,
                     "events_in_cuts": r.n_nonzero, "var_x_ms": rv * kms, "mean_pb": mean}
        if itg.proc == W.GG_TTBARG_MC:
            out[name]["alpha"] = [round(x, 4) for x in M.mc_vegas_get_channels(v)[0]]
        v.free()
    return out


def pp_ttbarj(M, pdf, stream, iterations=6):
    """p p -> t tbar + parton at LO (gg -> t tbar g and the six light-quark
    channels at every point; hierarchical phase space, 7 dims), FP32, 1e7
    events per iteration from a uniform grid: kernel time per iteration
    (median of the last 3), events per second, and the combined cross
    section of the last 3 iterations."""
    itg = W.pp_ttbarj()
    v = M.mc_vegas_init(7, NBINS, 3000, M.MC_FP32_KAHAN)
    ms, res = [], []
    with ClockSampler() as clk:
        for i in range(iterations):
            r = M.mc_vegas_iterate(v, itg, pdf, EVENTS, stream)
            M.mc_vegas_refine(v, ALPHA, stream)
            if i >= iterations - 3:
                ms.append(M.mc_vegas_kernel_ms(v))
                res.append(_iter_stats(r))
    v.free()
    mean, sig = _combine(res)
    kms = statistics.median(ms)
    return {"workload": "p p -> t tbar + parton, 13 TeV, parton pT > 20 GeV |eta| < 2.5, hierarchical 2->3, FP32, "
                        "1e7 events per iteration", "kernel_ms": kms, "events_per_s": EVENTS / (kms / 1e3),
            "xsec_pb": mean, "xsec_rel_err": sig / mean, "events_in_cuts": r.n_nonzero,
            "clocks": clk.summary(int(os.environ.get("LOCAL_RANK", "0")))}


def profile_case(case):
    """A small fixed workload for ncu captures (no timing output)."""
    import torch
    from paper_2302_03343_b300 import build
    from paper_2302_03343_b300 import mcint as M
    build.build()
    pdf = M.mc_pdf_load(W.synthetic_pdf_grid(0))
    if case == "integrand":
        v = M.mc_vegas_init(14, NBINS, 0, M.MC_FP32_KAHAN)
        for _ in range(3):
            M.mc_vegas_iterate(v, W.gg_ttbarg(), pdf, 1 << 20)
            M.mc_vegas_refine(v, ALPHA)
    elif case == "fp64_7d":  # plain FP64 VEGAS of gg -> ttg in 7 dims (the time-to-target arm): 2 x 2^20
        v = M.mc_vegas_init(7, NBINS, 0, M.MC_FP64)
        for _ in range(2):
            M.mc_vegas_iterate(v, W.gg_ttbarg_7d(), pdf, 1 << 20)
            M.mc_vegas_refine(v, ALPHA)
    elif case in ("mc", "ppttj"):  # three-channel gg -> ttg, or p p -> t tbar + parton: 3 iterations of 2^20
        itg = W.gg_ttbarg_mc() if case == "mc" else W.pp_ttbarj()
        v = M.mc_vegas_init(itg.ndim(), NBINS, 0, M.MC_FP32_KAHAN)
        for _ in range(3):
            M.mc_vegas_iterate(v, itg, pdf, 1 << 20)
            if case == "mc":
                a, w = M.mc_vegas_get_channels(v)
                M.mc_vegas_set_channels(v, M.mc_channel_update(a, w, 0.5, 0.02))
            M.mc_vegas_refine(v, ALPHA)
    elif case == "unweight":  # weights pass and unweighting of 2^24 events (134 MB of weights > L2)
        n = 1 << 24
        itg = W.gg_ttbarg()
        v = M.mc_vegas_init(14, NBINS, 0, M.MC_FP32_KAHAN)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        ev = torch.empty((n // 8, M.EVENT_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        for _ in range(2):
            r = M.mc_vegas_iterate_weights(v, itg, pdf, n, w)
            M.mc_unweight(v, itg, pdf, w, n, r.wmax, ev, n // 8)
    elif case == "pdf":  # the single-set batch interpolation, 2^24 points, FP32 then FP64
        x, q2 = pdf_sweep_inputs(1 << 24, seed=24)
        res = torch.empty((1 << 24, 11), dtype=torch.float64, device="cuda")
        for prec in (M.MC_FP32_KAHAN, M.MC_FP64):
            M.mc_pdf_xfxq2(pdf, prec, 1 << 24, x, q2, res)
    elif case == "pdfset":  # the multi-member PDF evaluation, FP32 then FP64
        import numpy as _np
        pset = W.synthetic_pdf_set(nmem=PDF_MEMBERS, seed=0)
        ps = M.mc_pdfset_load(pset)
        x = _np.array([10.0 ** (-7.0 * (1.0 - i / (PDF_POINTS - 1))) for i in range(PDF_POINTS)])
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        qd = torch.full_like(xd, PDF_Q * PDF_Q)
        for prec, dt in ((M.MC_FP32_KAHAN, torch.float32), (M.MC_FP64, torch.float64)):
            res = torch.empty((PDF_MEMBERS, PDF_POINTS, len(pset.pids)), dtype=dt, device="cuda")
            M.mc_pdfset_xfxq2(ps, prec, 0, PDF_MEMBERS, PDF_POINTS, xd, qd, res)
        ps.free()
    else:  # flow: two training steps of 65536 events, one sampling pass of 2^20 events
        itg = W.gg_ttbarg_7d()
        f = M.mc_flow_create(7, FLOW_LAYERS, FLOW_BINS, W.flow_init_params(7, FLOW_LAYERS, FLOW_BINS, seed=0),
                             FLOW_BATCH, seed=1)
        M.mc_flow_train(f, itg, pdf, 2, FLOW_BATCH, FLOW_LR, losses=False)
        M.mc_flow_iterate(f, itg, pdf, 1 << 20, iteration=0)
    torch.cuda.synchronize()
    print("profile case done:", case)


def fma_peaks(M, stream, reps=5):
    """FP32 and FP64 FMA throughput of this GPU (mc_fma_peak: a
    full-occupancy grid of independent FMA chains), best of `reps` launches
    timed with CUDA events: the measured denominators of the integrand
    kernels' roofline."""
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    threads = props.multi_processor_count * props.max_threads_per_multi_processor
    out = torch.empty(threads, dtype=torch.float32, device="cuda")
    res = {}
    for kind, name, iters in ((0, "fp32_fma", 1 << 16), (1, "fp32x2_fma", 1 << 15), (2, "fp64_fma", 1 << 11)):
        M.mc_fma_peak(kind, iters, out, stream)  # warm-up
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flop = M.mc_fma_peak(kind, iters, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res[name] = {"tflops": flop / (best / 1e3) / 1e12, "ms": best, "flop": flop}
    res["fp32_tflops"] = max(res["fp32_fma"]["tflops"], res["fp32x2_fma"]["tflops"])
    res["fp64_tflops"] = res["fp64_fma"]["tflops"]
    res["how"] = ("mc_fma_peak: SMs x 2048 threads, 8 independent chains of dependent FMAs per thread, "
                  "2 FLOP per lane operation, best of %d launches (CUDA events)" % reps)
    return res


def c2_pp_ttbar(M, pdf, stream):
    """Config: plain FP64 VEGAS of p p -> t tbar (gg + q qbar) at 13 TeV, 4
    dims, 50 bins, 10 iterations x 1e6 events, seed 0, from a uniform grid,
    through mc_integrate (GPU time from its CUDA events); the combined
    integral against the oracle's run of the same configuration and against
    the closed-form cross section of the master formula (stored values)."""
    g = golden("c2_pp_ttbar.json")
    p = g["params"]
    M.mc_integrate(W.pp_ttbar(), pdf, 1, p["nevents"], nbins=p["nbins"], seed=p["seed"], prec=M.MC_FP64,
                   stream=stream)  # warm-up
    res, _ = M.mc_integrate(W.pp_ttbar(), pdf, p["niter"], p["nevents"], nbins=p["nbins"], seed=p["seed"],
                            gid=p["gid"], prec=M.MC_FP64, alpha=p["alpha"], stream=stream)
    ref, cf = g["oracle"], g["closed_form"]["sigma_pb"]
    n = p["niter"] * p["nevents"]
    return {"workload": g["config"], "gpu_ms": res.gpu_ms, "events_per_s": n / (res.gpu_ms / 1e3),
            "mean_pb": res.mean, "sigma_pb": res.sigma, "chi2_dof": res.chi2_dof,
            "oracle_mean_pb": ref["mean_pb"], "rel_diff_vs_oracle": (res.mean - ref["mean_pb"]) / ref["mean_pb"],
            "closed_form_pb": cf, "pull_vs_closed_form": (res.mean - cf) / res.sigma}


def oracle_check(M, pdf, stream, keep=4_000_000):
    """Config: one full FP32 iteration of the benchmark workload (g g -> t tbar
    g, 1e7 events) on the grid the oracle adapted, against the FP64 oracle's
    iteration at the identical 23-bit points (stored values): the relative
    error of the integral, events in the cuts, w_max, and whether the bin
    counts are bit-exact.  Returns the result and the GPU's weights of the
    first `keep` events (host) for the per-event comparison with the
    CPU-baseline sample."""
    import torch
    g = golden("c3_ggttg_iteration.json")
    p = g["params"]
    n = p["nevents"]
    v = M.mc_vegas_init(14, p["nbins"], p["seed"], M.MC_FP32_KAHAN)
    M.mc_vegas_set_grid(v, np.array(g["edges"]))
    M.mc_vegas_set_iteration(v, p["iteration"])
    M.mc_vegas_set_gid(v, p["gid"])
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    r = M.mc_vegas_iterate_weights(v, W.gg_ttbarg(), pdf, n, w, stream)
    _, cnt = M.mc_vegas_get_hist(v)
    v.free()
    ref = g["oracle"]
    out = {"workload": g["config"], "events": n, "integral_pb": r.sum / n, "oracle_integral_pb": ref["sum"] / n,
           "integral_rel_err": (r.sum - ref["sum"]) / ref["sum"], "in_cuts": r.n_nonzero,
           "oracle_in_cuts": ref["n_nonzero"], "wmax_rel_err": (r.wmax - ref["wmax"]) / ref["wmax"],
           "bin_counts_bit_exact": bool(np.array_equal(cnt, np.array(ref["hist_n"], dtype=np.uint32)))}
    return out, w[:keep].cpu().numpy()


def per_event_stats(w_gpu, w_oracle):
    """Relative per-event errors of the FP32 weights against FP64 (events in
    the cuts on both sides) and the events whose cut decision differs."""
    k = min(len(w_gpu), len(w_oracle))
    wg, wo = w_gpu[:k], w_oracle[:k]
    both = (wg != 0) & (wo != 0)
    e = np.abs(wg[both] - wo[both]) / np.abs(wo[both])
    return {"events": int(k), "compared": int(both.sum()), "median": float(np.median(e)),
            "p99": float(np.quantile(e, 0.99)), "max": float(e.max()),
            "cut_flips": int(np.count_nonzero((wg != 0) != (wo != 0)))}


def time_to_target(M, pdf, stream, seed=0):
    """GPU time (CUDA events around every launch of the arm) from the first
    launch to the end of the first iteration whose combined relative error is
    at most TTT_TARGET, for plain FP64 VEGAS, FP32 VEGAS and FP32 + flow on
    gg -> t tbar g (7 dims), and FP32 three-channel sampling of the same
    process, each from scratch (uniform grids / identity flow)."""
    import torch
    itg = W.gg_ttbarg_7d()
    out = {"target_rel_err": TTT_TARGET, "events_per_iteration": TTT_EVENTS, "workload":
           "gg->ttg 13 TeV, hierarchical 2->3 phase space (7 dims), same cuts and PDF grid"}

    def vegas(prec, name, integrand=itg):
        v = M.mc_vegas_init(integrand.ndim(), NBINS, seed, prec)
        res, per_event, eff = [], None, None
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for it in range(TTT_MAX_ITER):
            r = M.mc_vegas_iterate(v, integrand, pdf, TTT_EVENTS, stream)
            if integrand.proc == W.GG_TTBARG_MC:  # Kleiss-Pittau step of the channel probabilities
                a, w = M.mc_vegas_get_channels(v)
                M.mc_vegas_set_channels(v, M.mc_channel_update(a, w, 0.5, 0.02))
            M.mc_vegas_refine(v, ALPHA, stream)
            res.append(_iter_stats(r))
            mean, sig = _combine(res)
            if sig <= TTT_TARGET * abs(mean):
                break
        t1.record(stream)
        torch.cuda.synchronize()
        m_it, v_it = res[-1]
        per_event = v_it * r.n / (m_it * m_it)
        eff = m_it / r.wmax if r.wmax > 0 else None
        arm = {"ms": t0.elapsed_time(t1), "iterations": len(res), "mean_pb": mean, "rel_err": sig / abs(mean),
               "rel_var_per_event_last": per_event, "unweighting_eff_last": eff}
        if integrand.proc == W.GG_TTBARG_MC:
            arm["alpha_final"] = [round(x, 4) for x in M.mc_vegas_get_channels(v)[0]]
        v.free()
        return arm

    out["vegas_fp64"] = vegas(M.MC_FP64, "fp64")
    out["vegas_fp32"] = vegas(M.MC_FP32_KAHAN, "fp32")
    # three-channel sampling (thesis Sec. "Multi-channel Monte Carlo"), FP32,
    # per-channel grids, channel probabilities updated after every iteration
    out["multichannel_fp32"] = vegas(M.MC_FP32_KAHAN, "mc", W.gg_ttbarg_mc())
    out["multichannel_fp32"]["workload"] = ("gg->ttg, three channels (initial-state radiation, radiation off t, "
                                            "off tbar), 7 uniforms per event, 17-dimension grid")
    # flow arm: training included in the timed region
    init = W.flow_init_params(7, L=FLOW_LAYERS, K=FLOW_BINS, seed=seed)
    f = M.mc_flow_create(7, FLOW_LAYERS, FLOW_BINS, init, FLOW_BATCH, seed=seed + 1)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    tt = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    M.mc_flow_train(f, itg, pdf, FLOW_STEPS, FLOW_BATCH, FLOW_LR, stream=stream, losses=False)
    tt.record(stream)
    res = []
    for it in range(TTT_MAX_ITER):
        r = M.mc_flow_iterate(f, itg, pdf, TTT_EVENTS, iteration=it, stream=stream)
        res.append(_iter_stats(r))
        mean, sig = _combine(res)
        if sig <= TTT_TARGET * abs(mean):
            break
    t1.record(stream)
    torch.cuda.synchronize()
    m_it, v_it = res[-1]
    flow = {"ms": t0.elapsed_time(t1), "train_ms": t0.elapsed_time(tt), "sample_ms": tt.elapsed_time(t1),
            "train_steps": FLOW_STEPS, "train_batch": FLOW_BATCH, "iterations": len(res), "mean_pb": mean,
            "rel_err": sig / abs(mean), "rel_var_per_event_last": v_it * r.n / (m_it * m_it),
            "unweighting_eff_last": m_it / r.wmax if r.wmax > 0 else None,
            "sample_events_per_s": TTT_EVENTS * len(res) / (tt.elapsed_time(t1) / 1e3)}
    f.free()
    out["flow_fp32_breakdown"] = flow
    # the method as a whole: flow sampling with plain VEGAS as judge and
    # fallback (one FP32 VEGAS iteration measures VEGAS's variance per event)
    res, used = M.mc_integrate_flow(itg, pdf, 7, FLOW_LAYERS, FLOW_BINS, init, FLOW_STEPS, FLOW_BATCH, FLOW_LR,
                                    niter=TTT_MAX_ITER, nevents=TTT_EVENTS, nbins=NBINS, seed=seed,
                                    target_rel_err=TTT_TARGET, stream=stream)
    flow = {"ms": res.gpu_ms, "sampler": "flow" if used else "vegas (fallback)", "iterations": res.n_iter,
            "mean_pb": res.mean, "rel_err": res.sigma / abs(res.mean), "chi2_dof": res.chi2_dof,
            "includes": f"{FLOW_STEPS} training steps x {FLOW_BATCH} events, the judge's FP32 VEGAS iteration"}
    out["flow_fp32"] = flow
    out["ratio_vegas_fp64_over_flow"] = out["vegas_fp64"]["ms"] / flow["ms"]
    comb = (out["vegas_fp64"]["mean_pb"] - flow["mean_pb"]) / (
        (out["vegas_fp64"]["rel_err"] * out["vegas_fp64"]["mean_pb"]) ** 2 +
        (flow["rel_err"] * flow["mean_pb"]) ** 2) ** 0.5
    out["flow_vs_vegas_fp64_pulls"] = comb
    return out


def sharded_integration(M, pdf, itg, args, rank, world, stream, dev, l2):
    """One integration of the benchmark workload split across the ranks (the
    multi-GPU split of the path): every iteration, rank r evaluates its
    contiguous share of the events (the same Philox counters as one device),
    one all-reduce adds the sums and histograms, and every rank refines the
    same grid.  Strong scaling: the events of an iteration are fixed as the
    ranks grow.  Device time per step from CUDA events (the all-reduce and the
    host round trips of the histograms included), slowest rank."""
    import torch
    from paper_2302_03343_b300 import shard
    v = M.mc_vegas_init(14, NBINS, 0, M.MC_FP32_KAHAN)
    for _ in range(args.warmup):
        shard.iterate_sharded(v, itg, pdf, args.events, rank, world, stream, dev)
        M.mc_vegas_refine(v, ALPHA, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ranks_barrier()
    torch.cuda.synchronize()
    last = None
    for i in range(args.steps):
        flush_l2(l2)
        ev[i][0].record(stream)
        last = shard.iterate_sharded(v, itg, pdf, args.events, rank, world, stream, dev)
        M.mc_vegas_refine(v, ALPHA, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev)
    v.free()
    nh = 14 * NBINS
    mean = last["sum"] / last["n"]
    return {"value": args.events * args.steps / (ms / 1e3), "unit": "events/s", "parallelism": f"sharded x{world}",
            "scaling": "strong", "ms_per_step": ms / args.steps, "events_per_step": args.events,
            "allreduce_bytes_per_step": (2 + 1) * 8 + 3 * 8 + nh * 8 * 2 if world > 1 else 0,
            "last_iteration_mean_pb": mean}


def run_native(args, rank, world):
    import torch
    from paper_2302_03343_b300 import build
    from paper_2302_03343_b300 import mcint as M

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    grid = W.synthetic_pdf_grid(0)
    pdf = M.mc_pdf_load(grid)
    itg = W.gg_ttbarg()
    l2 = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    # weak scaling: every rank runs its own integration (its own Philox stream)
    v = M.mc_vegas_init(14, NBINS, replica_seed(rank), M.MC_FP32_KAHAN)
    for _ in range(args.warmup):
        M.mc_vegas_iterate(v, itg, pdf, args.events, stream)
        M.mc_vegas_refine(v, ALPHA, stream)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms, nnz, results = [], [], []
    ranks_barrier()
    torch.cuda.synchronize()
    with ClockSampler() as clk:
        for i in range(args.steps):
            flush_l2(l2)
            ev[i][0].record(stream)
            r = M.mc_vegas_iterate(v, itg, pdf, args.events, stream)
            M.mc_vegas_refine(v, ALPHA, stream)
            ev[i][1].record(stream)
            kernel_ms.append(M.mc_vegas_kernel_ms(v))
            nnz.append(r.n_nonzero)
            results.append(r)
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in ev]
    ranks_barrier()
    total_ms = max_over_ranks(sum(step_ms), dev)
    clocks = clk.summary(local)

    # end to end through the public API with host buffers: upload the host
    # grid, iterate (sums back to the host), refine, read the grid back
    edges = M.mc_vegas_get_grid(v)
    ve = M.mc_vegas_init(14, NBINS, replica_seed(rank) + 4000, M.MC_FP32_KAHAN)
    e2e_s = []
    ranks_barrier()
    for i in range(args.steps):
        flush_l2(l2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.mc_vegas_set_grid(ve, edges)
        M.mc_vegas_iterate(ve, itg, pdf, args.events, stream)
        M.mc_vegas_refine(ve, ALPHA, stream)
        edges = M.mc_vegas_get_grid(ve)
        e2e_s.append(time.perf_counter() - t0)
    ngrid = 14 * (NBINS + 1)
    h2d = ngrid * 8 + ngrid * 4
    d2h = 64 + ngrid * 8
    e2e_ms = max_over_ranks(1e3 * sum(e2e_s), dev)
    sharded = sharded_integration(M, pdf, itg, args, rank, world, stream, dev, l2)

    if rank != 0:
        return
    value = job_rate(args.events, args.steps, world, total_ms)
    measured = fma_peaks(M, stream)
    pk = peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = pk.get("sm_max_mhz", 2032.0)
    fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s
    mean_kernel_ms = sum(kernel_ms) / len(kernel_ms)
    mean_nnz = sum(nnz) / len(nnz)
    # algorithmic work of one launch: the oracle's operation counts per event
    # (map, RAMBO, cuts) and per event inside the cuts (PDFs, |M|^2 from
    # helicity amplitudes, weight), times this launch's events
    oc = golden("ggttg_opcount.json")
    algo_flop = (sum(oc["flop_per_event"].values()) * args.events +
                 sum(oc["flop_per_event_in_cuts"].values()) * mean_nnz)
    achieved = algo_flop / (mean_kernel_ms / 1e3) / 1e12
    executed = EXECUTED_FLOP_PER_EVENT * mean_nnz / (mean_kernel_ms / 1e3) / 1e12
    peak = measured["fp32_tflops"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC_BYTES,
            "algorithmic_flop_per_launch": algo_flop,
            "algorithmic_source": "oracle operation counts (tests/golden/ggttg_opcount.json): "
                                  f"{sum(oc['flop_per_event'].values()):.0f} FLOP per event (map, RAMBO, cuts) + "
                                  f"{sum(oc['flop_per_event_in_cuts'].values()):.0f} per event in the cuts "
                                  "(PDFs, |M|^2 from helicity amplitudes, weight)",
            "peak_source": "measured (fma_peaks: the larger of the f32 and f32x2 FMA rates)",
            "executed": executed, "frac_executed": executed / peak,
            "executed_note": f"{EXECUTED_FLOP_PER_EVENT:.0f} FP32 FLOP per in-cut event executed (ncu): the "
                             "kernel shares sub-amplitudes across orderings, spins and polarisations that "
                             "the oracle's formulation recomputes",
            "peak_nominal": fp32_peak,
            "nominal_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz",
            "frac_executed_of_mix_bound": executed / (fp32_peak * FLOP_PER_LANE_OP / 2.0),
            "mix_bound_note": "the nominal peak times the kernel's FLOP per FP32 lane operation / 2 "
                              f"({FLOP_PER_LANE_OP:.3f} / 2): the executed rate if every lane slot issued its mix"}
    roof["kernel_ms"] = mean_kernel_ms
    roof["events_in_cuts_per_launch"] = mean_nnz
    r_last = results[-1]
    mean = r_last.sum / r_last.n
    var = (r_last.sum2 / r_last.n - mean * mean) / (r_last.n - 1)
    line = {"metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (|M|^2) + f64 (sums, RAMBO boosts)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "events_per_step": args.events, "nbins": NBINS,
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                       "other_mode": "sharded (one integration split across the ranks): the 'sharded' object"},
            "clocks": clocks,
            "e2e": {"value": job_rate(args.events, args.steps, world, e2e_ms), "unit": "events/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 3 * args.steps,
            "sharded": sharded,
            "roofline": roof,
            "fma_peaks": measured,
            "last_iteration": {"mean_pb": mean, "rel_err": (var ** 0.5) / abs(mean) if mean else None,
                               "n_nonzero": r_last.n_nonzero, "unweighting_eff": mean / r_last.wmax
                               if r_last.wmax > 0 else None}}
    w_check = None
    if not args.no_time_to_target:
        line["c2"] = c2_pp_ttbar(M, pdf, stream)
        line["oracle_check"], w_check = oracle_check(M, pdf, stream)
        line["time_to_target"] = time_to_target(M, pdf, stream)
        line["batch16"] = batch16(M, pdf, stream)
        line["pdf_members"] = pdf_members(M, stream)
        line["pdf_xfxq2"] = pdf_xfxq2_sweep(M, pdf, stream)
        line["unweighting"] = unweighting(M, pdf, stream, M.mc_vegas_get_grid(v), mean_kernel_ms)
        line["samplers"] = samplers(M, pdf, stream)
        line["pp_ttbarj"] = pp_ttbarj(M, pdf, stream)
    if not args.no_cpu_baseline:
        line["cpu_baseline"], w_oracle = cpu_baseline()
        if w_check is not None:
            line["oracle_check"]["per_event"] = per_event_stats(w_check, w_oracle)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--events", type=int, default=EVENTS)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-target", action="store_true")
    ap.add_argument("--profile-case", choices=["integrand", "flow", "pdf", "pdfset", "unweight", "mc", "ppttj", "fp64_7d"], default=None,
                    help="run a small fixed workload for profiling and exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world)


if __name__ == "__main__":
    main()
