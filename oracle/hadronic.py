"""Closed-form LO p p -> t tbar cross section by quadrature (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): an independent check of
the Monte Carlo estimate of the master formula (thesis Sec. "The MadFlow
event generator", eq. mc_master_formula)

    sigma = sum_ab int dx1 dx2 f_a(x1, mu_F) f_b(x2, mu_F) sigma_ab(x1 x2 s),

with the textbook total partonic cross sections (Combridge; Ellis, Stirling &
Webber) in place of the phase-space integral over (cos theta, phi):

    sigma_qqbar(s) = 8 pi alpha_s^2 / (27 s) beta (1 + rho / 2),
    sigma_gg(s)    = pi alpha_s^2 / (3 s) [(1 + rho + rho^2 / 16) ln((1 + beta) / (1 - beta))
                                           - beta (7 / 4 + 31 rho / 16)],

rho = 4 m^2 / s, beta = sqrt(1 - rho), times 0.3893794e9 pb GeV^2.

The densities are the oracle's own interpolation (oracle.Pdf).  At a fixed
factorisation scale, x f(x) is a cubic polynomial in t = ln x on every cell of
a log-spaced x grid (a Hermite cubic in t at each Q knot, then a fixed linear
combination of the Q knots), so each cell's cubic is recovered exactly from
four evaluations.  With L = ln(x1 x2) and y = (ln x1 - ln x2) / 2,

    sigma = int_{L0}^{0} dL  sum_ab Lum_ab(L) sigma_ab(e^L s),
    Lum_ab(L) = int_{L/2}^{-L/2} dy  (x f_a)(L/2 + y) (x f_b)(L/2 - y),

L0 = ln(4 m^2 / s).  For fixed L the y integrand is a polynomial of degree 6
between the points where ln x1 or ln x2 crosses a knot, so four-point
Gauss-Legendre per piece is exact.  Lum(L) is a polynomial between the points
L = t_i + t_j, which on a uniform log grid are spaced by the knot spacing;
each such panel gets 16-point Gauss-Legendre, and the first one, where sigma
grows like beta ~ sqrt(L - L0), is integrated in u = sqrt(L - L0), in which
the integrand is smooth.
"""
import math

import numpy as np

GEV2PB = 0.3893794e9


def sigma_hat_qqbar(alpha_s, mt, s, gev2pb=GEV2PB):
    """Total partonic q qbar -> t tbar cross section (pb) at squared energy s."""
    rho = 4.0 * mt * mt / s
    if rho >= 1.0:
        return 0.0
    beta = math.sqrt(1.0 - rho)
    return 8.0 * math.pi * alpha_s ** 2 / (27.0 * s) * beta * (1.0 + rho / 2.0) * gev2pb


def sigma_hat_gg(alpha_s, mt, s, gev2pb=GEV2PB):
    """Total partonic g g -> t tbar cross section (pb) at squared energy s."""
    rho = 4.0 * mt * mt / s
    if rho >= 1.0:
        return 0.0
    beta = math.sqrt(1.0 - rho)
    lg = math.log((1.0 + beta) / (1.0 - beta))
    return math.pi * alpha_s ** 2 / (3.0 * s) * ((1.0 + rho + rho * rho / 16.0) * lg
                                                 - beta * (7.0 / 4.0 + 31.0 * rho / 16.0)) * gev2pb


class CellCubics:
    """x f(x, Q^2) of one flavour as a cubic in s = (ln x - t_i) / h on every
    cell [t_i, t_i + h] of a uniform ln x grid, recovered from the oracle's
    interpolation at four points of each cell."""

    NODES = np.array([0.1, 0.4, 0.6, 0.9])

    def __init__(self, pdf, pid, t, q2):
        self.t0, self.h, self.n = float(t[0]), float(t[1] - t[0]), len(t) - 1
        V = np.vander(self.NODES, 4)  # rows: s^3, s^2, s, 1
        coef = np.empty((self.n, 4))
        for i in range(self.n):
            tt = self.t0 + self.h * (i + self.NODES)
            vals = np.array([pdf.xfxq2(pid, math.exp(v), q2) for v in tt])
            coef[i] = np.linalg.solve(V, vals)
        self.coef = coef

    def __call__(self, tt):
        tt = np.asarray(tt, dtype=np.float64)
        i = np.clip(np.floor((tt - self.t0) / self.h).astype(np.int64), 0, self.n - 1)
        s = (tt - (self.t0 + self.h * i)) / self.h
        c = self.coef[i]
        return ((c[..., 0] * s + c[..., 1]) * s + c[..., 2]) * s + c[..., 3]


def _uniform_log_knots(x):
    t = np.log(np.asarray(x, dtype=np.float64))
    h = (t[-1] - t[0]) / (len(t) - 1)
    if np.max(np.abs(np.diff(t) - h)) > 1e-9 * abs(h):
        raise ValueError("the quadrature needs log-spaced x knots")
    return t[0] + h * np.arange(len(t)), h


def luminosities(cubics_pairs, L, t, h):
    """sum over the (a, b) pairs of Lum_ab(L) for each L (exact)."""
    g4, w4 = np.polynomial.legendre.leggauss(4)
    out = np.empty(len(L))
    tmax = t[-1]
    for k, Lk in enumerate(L):
        lo, hi = Lk / 2.0 - tmax, tmax - Lk / 2.0  # y range: ln x1, ln x2 <= t_max (= 0)
        br = np.concatenate([t - Lk / 2.0, Lk / 2.0 - t])
        br = np.unique(np.concatenate([[lo, hi], br[(br > lo) & (br < hi)]]))
        a, b = br[:-1], br[1:]
        y = (0.5 * (b - a))[:, None] * g4[None, :] + (0.5 * (a + b))[:, None]
        wy = (0.5 * (b - a))[:, None] * w4[None, :]
        t1, t2 = Lk / 2.0 + y, Lk / 2.0 - y
        acc = 0.0
        for fa, fb in cubics_pairs:
            acc += float(np.sum(wy * fa(t1) * fb(t2)))
        out[k] = acc
    return out


def pp_ttbar_sigma(pdf, grid, alpha_s=0.118, mt=173.0, mu_f=173.0, sqrt_s=13000.0, gev2pb=GEV2PB):
    """sigma(p p -> t tbar) at LO (pb): g g plus q qbar and qbar q of the five
    light flavours, with the oracle's densities at mu_F."""
    t, h = _uniform_log_knots(grid.x)
    q2 = mu_f * mu_f
    s = sqrt_s * sqrt_s
    cub = {int(p): CellCubics(pdf, int(p), t, q2) for p in grid.pids}
    gg = [(cub[21], cub[21])]
    qq = []
    for q in range(1, 6):
        qq += [(cub[q], cub[-q]), (cub[-q], cub[q])]
    L0 = math.log(4.0 * mt * mt / s)
    # panel ends: L0, the points 2 t_0 + k h above it, and t_max + t_max (= 0)
    kmin = math.floor((L0 - 2.0 * t[0]) / h) + 1
    ends = [L0] + [2.0 * t[0] + k * h for k in range(kmin, int(round((2 * t[-1] - 2 * t[0]) / h)) + 1)]
    ends = np.array(sorted(set(e for e in ends if e > L0 and e <= 2 * t[-1] + 1e-12) | {L0}))
    g16, w16 = np.polynomial.legendre.leggauss(16)
    Ls, Ws = [], []
    for j in range(len(ends) - 1):
        a, b = ends[j], ends[j + 1]
        if j == 0:  # L = L0 + u^2, dL = 2 u du
            umax = math.sqrt(b - a)
            u = 0.5 * umax * (g16 + 1.0)
            Ls.append(a + u * u)
            Ws.append(0.5 * umax * w16 * 2.0 * u)
        else:
            Ls.append(0.5 * (b - a) * g16 + 0.5 * (a + b))
            Ws.append(0.5 * (b - a) * w16)
    L = np.concatenate(Ls)
    W = np.concatenate(Ws)
    lum_gg = luminosities(gg, L, t, h)
    lum_qq = luminosities(qq, L, t, h)
    sg = np.array([sigma_hat_gg(alpha_s, mt, math.exp(l) * s, gev2pb) for l in L])
    sq = np.array([sigma_hat_qqbar(alpha_s, mt, math.exp(l) * s, gev2pb) for l in L])
    return {"sigma_pb": float(np.sum(W * (lum_gg * sg + lum_qq * sq))),
            "gg_pb": float(np.sum(W * lum_gg * sg)), "qqbar_pb": float(np.sum(W * lum_qq * sq))}
