"""Writes the stored oracle values of tests/golden/ (calls only oracle/).

c2_pp_ttbar.json: plain FP64 VEGAS of p p -> t tbar at 13 TeV (4 dims, 50
bins, 10 iterations x 1e6 events, Philox seed 0, uniform starting grid), as
the oracle runs it (thesis Sec. "Adaptive Monte Carlo: VEGAS algorithm":
per-iteration estimates combined by inverse variance, eq. vegas-check), and
the closed-form cross section of the same master formula (Sec. "The MadFlow
event generator", eq. mc_master_formula) by quadrature (oracle/hadronic.py).

c3_ggttg_iteration.json: one full iteration of 1e7 events of g g -> t tbar g
(RAMBO, 14 sampled dimensions, gluon pT > 20 GeV, |eta| < 2.5) with the
23-bit uniforms of the FP32 mode, evaluated by the FP64 oracle on a grid
that the oracle itself adapted (5 iterations x 2e5 events, FP32-mode
uniforms, seed 0), for the check of the FP32 path against FP64 at identical
points (eq. mc_est_is): the grid, the sums, the count of events in the cuts,
the largest weight and the bin counts.

ggttg_opcount.json: the algorithmic operation counts of that workload's
event (oracle/src/opcount.cpp: the oracle's VEGAS map, RAMBO, cuts, PDFs,
|M|^2 from helicity amplitudes (formulation C) and weight, run with an
operation-counting scalar) over the first 20 000 events of the stored
iteration, per event and per event inside the cuts.

Run: python tests/golden/make_golden.py [c2] [c3] [opcount]   (c3 takes several minutes;
opcount reads c3's grid)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from oracle import hadronic as H  # noqa: E402
from paper_2302_03343_b300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
C2 = dict(niter=10, nevents=1_000_000, nbins=50, seed=0, gid=0, alpha=1.5)
C3 = dict(adapt_iter=5, adapt_events=200_000, nbins=50, seed=0, gid=0, alpha=1.5, iteration=5,
          nevents=10_000_000)


def c2():
    grid = W.synthetic_pdf_grid(0)
    pdf = O.Pdf(grid)
    itg = W.pp_ttbar()
    t0 = time.time()
    r = O.integrate(itg, pdf, W.uniform_grid(4, C2["nbins"]), 0, C2["seed"], C2["gid"], C2["niter"], C2["nevents"],
                    alpha=C2["alpha"])
    t_mc = time.time() - t0
    q = H.pp_ttbar_sigma(pdf, grid, itg.alpha_s, itg.m_top, itg.mu_f, itg.sqrt_s, itg.gev2pb)
    out = {"config": "p p -> t tbar LO, 13 TeV, m_t = mu_F = 173 GeV, alpha_s = 0.118, FP64, 4 dims, "
                     "50 bins, 10 iterations x 1e6 events, seed 0, uniform starting grid, synthetic PDF grid seed 0",
           "params": C2, "oracle": {"mean_pb": r["mean"], "sigma_pb": r["sigma"], "chi2_dof": r["chi2dof"],
                                    "per_iteration": r["per_iter"].tolist(), "seconds": t_mc},
           "closed_form": q,
           "citation": "thesis eq. mc_master_formula; VEGAS combination eq. vegas-check"}
    with open(os.path.join(HERE, "c2_pp_ttbar.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("c2", out["oracle"]["mean_pb"], out["oracle"]["sigma_pb"], q["sigma_pb"])


def c3():
    grid = W.synthetic_pdf_grid(0)
    pdf = O.Pdf(grid)
    itg = W.gg_ttbarg()
    a = O.integrate(itg, pdf, W.uniform_grid(14, C3["nbins"]), 1, C3["seed"], C3["gid"], C3["adapt_iter"],
                    C3["adapt_events"], alpha=C3["alpha"])
    edges = a["edges"]
    t0 = time.time()
    r = O.iterate(itg, pdf, edges, 1, C3["seed"], C3["iteration"], C3["gid"], 0, C3["nevents"])
    t_it = time.time() - t0
    out = {"config": "g g -> t tbar g, 13 TeV, RAMBO 2 + 12 dims, gluon pT > 20 GeV |eta| < 2.5, FP32-mode "
                     "(23-bit) uniforms evaluated in FP64, 1e7 events, seed 0, iteration 5, on the grid the "
                     "oracle adapted in 5 iterations x 2e5 events",
           "params": C3, "edges": edges.tolist(),
           "oracle": {"sum": r["sum"], "sum2": r["sum2"], "n": r["n"], "n_nonzero": r["n_nonzero"],
                      "wmax": r["wmax"], "hist_n": r["hist_n"].astype(np.int64).tolist(), "seconds": t_it},
           "citation": "thesis eq. mc_est_is (the iteration's estimate is the mean of w = f J)"}
    with open(os.path.join(HERE, "c3_ggttg_iteration.json"), "w") as f:
        json.dump(out, f)
    print("c3", r["sum"] / r["n"], r["n_nonzero"], t_it)


def opcount(n=20_000):
    with open(os.path.join(HERE, "c3_ggttg_iteration.json")) as f:
        g = json.load(f)
    p = g["params"]
    pdf = O.Pdf(W.synthetic_pdf_grid(0))
    r = O.count_gg_ttbarg(W.gg_ttbarg(), pdf, np.array(g["edges"]), 1, p["seed"], p["iteration"], p["gid"], 0, n)
    flop = {st: sum(r[st][k] for k in ("add", "mul", "div", "sqrt")) for st in O.COUNT_STEPS}
    every = ("map", "rambo", "cuts")  # run for every event (cuts: every event above threshold)
    out = {"config": "g g -> t tbar g, RAMBO 2 + 12 dims, the first %d events of the stored FP32-mode iteration" % n,
           "events": r["events"], "in_cuts": r["in_cuts"], "counts": {st: r[st] for st in O.COUNT_STEPS},
           "flop_per_event": {st: flop[st] / r["events"] for st in every},
           "flop_per_event_in_cuts": {st: flop[st] / r["in_cuts"] for st in O.COUNT_STEPS if st not in every},
           "convention": "additions, subtractions, multiplications, divisions and square roots count one FLOP each; "
                         "special functions (log, exp, sin, cos, pow) are counted apart, not as FLOP",
           "citation": "thesis Sec. \"The MadFlow event generator\" (|M|^2 from helicity amplitudes), Sec. \"RAMBO\", "
                       "Sec. \"LHAPDF: the Les Houches Accord PDF\", eq. mc_est_is"}
    with open(os.path.join(HERE, "ggttg_opcount.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("opcount", out["flop_per_event"], out["flop_per_event_in_cuts"])


if __name__ == "__main__":
    which = sys.argv[1:] or ["c2", "c3", "opcount"]
    if "c2" in which:
        c2()
    if "c3" in which:
        c3()
    if "opcount" in which:
        opcount()
