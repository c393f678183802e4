"""Pins of the oracle's log-bicubic PDF interpolation (thesis Sec. "LHAPDF:
the Les Houches Accord PDF")."""
import math

import numpy as np

import oracle as O
from paper_2302_03343_b300 import workloads as W


def test_nodes_reproduced_exactly(pdf_grid, oracle_pdf):
    g = pdf_grid
    for fl, pid in enumerate(g.pids):
        for i in range(0, len(g.x), 3):
            for j in range(0, len(g.q), 3):
                got = oracle_pdf.xfxq2(int(pid), g.x[i], g.q[j] ** 2)
                assert got == g.xf[i, j, fl], (pid, i, j)


def test_quadratic_reproduced_in_interior_cells(pdf_grid):
    # cubic Hermite with centred divided-difference slopes is exact for
    # functions quadratic in (log x, log Q^2) on the uniform log grid
    g = pdf_grid
    t = np.log(g.x)[:, None]
    s = np.log(g.q ** 2)[None, :]
    f = 2.0 + 0.3 * t + 0.05 * t * t - 0.2 * s + 0.01 * s * s
    xf = np.repeat(f[:, :, None], len(g.pids), axis=2)
    pdf = O.Pdf(W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=xf, params=g.params))
    rng = np.random.default_rng(0)
    for _ in range(300):
        lt = rng.uniform(np.log(g.x[1]), np.log(g.x[-2]))
        ls = rng.uniform(np.log(g.q[1] ** 2), np.log(g.q[-2] ** 2))
        expect = 2.0 + 0.3 * lt + 0.05 * lt * lt - 0.2 * ls + 0.01 * ls * ls
        got = pdf.xfxq2(21, math.exp(lt), math.exp(ls))
        assert abs(got - expect) < 1e-12 * abs(expect)


def test_accuracy_metric_against_the_generating_function(pdf_grid, oracle_pdf):
    # eq. pdfflow-diff: r = |xf_interp - xf_exact| / (|xf_exact| + 1e-16) stays
    # below the 1e-3 threshold where the log-x knots resolve (1-x)^b (x <= 0.1)
    g = pdf_grid
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(2000):
        x = 10 ** rng.uniform(-4, -1)
        q = 10 ** rng.uniform(math.log10(2.0), 3.9)
        fl = int(rng.integers(len(g.pids)))
        A, a, b, c = g.params[fl]
        exact = A * x ** (-a) * (1 - x) ** b * (1 + c * math.log(q * q / 1.65 ** 2))
        got = oracle_pdf.xfxq2(int(g.pids[fl]), x, q * q)
        worst = max(worst, abs(got - exact) / (abs(exact) + 1e-16))
    assert worst < 1e-3, worst


def test_out_of_grid_and_unknown_flavour_are_nan(oracle_pdf):
    assert math.isnan(oracle_pdf.xfxq2(21, 1e-9, 100.0))
    assert math.isnan(oracle_pdf.xfxq2(21, 0.1, 1e10))
    assert math.isnan(oracle_pdf.xfxq2(6, 0.1, 100.0))
