"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle side.

This module holds no arithmetic of the method itself: it draws the synthetic
PDF grid (the thesis's LHAPDF sets are not available, so a grid of the same
shape stands in for them) and names the integrand configurations.

PDF grid recipe (stand-in for an LHAPDF set such as NNPDF3.1, thesis
Sec. "LHAPDF: the Les Houches Accord PDF"): 100 x knots x_i = 10^(-7 + 7 i/99)
with x_99 = 1, 40 Q knots Q_j = 1.65 (1e4/1.65)^(j/39) GeV, 11 flavours in
LHAPDF order (-5..-1, 21, 1..5), values
    x f(x, Q) = A x^-a (1 - x)^b (1 + c ln(Q^2 / Q0^2)),  Q0 = 1.65 GeV,
with (A, a, b, c) drawn per flavour from SplitMix64(seed):
A in [0.5, 2] (times 3 for the gluon), a in [0, 0.3], b in [2, 6], c in [0, 0.2].
synthetic_pdf_set adds sub-grids (a b-quark threshold) and members, and
synthetic_alphas_knots the alpha_s(Q) knots of such a set.
"""
from dataclasses import dataclass, asdict
import math

import numpy as np

PIDS = (-5, -4, -3, -2, -1, 21, 1, 2, 3, 4, 5)
GEV2_TO_PB = 0.3893794e9

EE_MUMU, PP_TTBAR, GG_TTBARG, GAUSS, GG_TTBARG_7D, GG_TTBARG_MC, PP_TTBARJ = 0, 1, 2, 3, 4, 5, 6
FP64, FP32 = 0, 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): seeds the synthetic inputs."""

    def __init__(self, seed):
        self.state = seed & 0xFFFFFFFFFFFFFFFF

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0):
        return lo + (hi - lo) * (self.next_u64() >> 11) * 2.0 ** -53


@dataclass
class PdfGrid:
    x: np.ndarray        # [nx]
    q: np.ndarray        # [nq] (GeV)
    pids: np.ndarray     # [nflav] int32
    xf: np.ndarray       # [nx][nq][nflav] float64 (LHAPDF data-block order)
    params: np.ndarray   # [nflav][4] (A, a, b, c)


def synthetic_pdf_grid(seed=0, nx=100, nq=40, xmin=1e-7, qmin=1.65, qmax=1e4):
    x = np.array([10.0 ** (math.log10(xmin) * (1.0 - i / (nx - 1))) for i in range(nx)])
    x[-1] = 1.0
    q = np.array([qmin * (qmax / qmin) ** (j / (nq - 1)) for j in range(nq)])
    rng = SplitMix64(seed)
    params = []
    for pid in PIDS:
        A = rng.uniform(0.5, 2.0) * (3.0 if pid == 21 else 1.0)
        a = rng.uniform(0.0, 0.3)
        b = rng.uniform(2.0, 6.0)
        c = rng.uniform(0.0, 0.2)
        params.append((A, a, b, c))
    params = np.array(params)
    xf = np.empty((nx, nq, len(PIDS)))
    q0 = qmin
    for fl, (A, a, b, c) in enumerate(params):
        for i, xi in enumerate(x):
            for j, qj in enumerate(q):
                xf[i, j, fl] = A * xi ** (-a) * (1.0 - xi) ** b * (1.0 + c * math.log(qj * qj / (q0 * q0)))
    return PdfGrid(x=x, q=q, pids=np.array(PIDS, dtype=np.int32), xf=xf, params=params)


@dataclass
class PdfSet:
    """A PDF set of several sub-grids and members (LHAPDF layout)."""
    x: list              # per sub-grid: x knots
    q: list              # per sub-grid: Q knots (GeV); adjacent sub-grids share the threshold knot
    pids: np.ndarray     # [nflav] int32
    xf: np.ndarray       # [nmem][sum over sub-grids of nx*nq*nflav]: per sub-grid [x][q][flav]
    params: np.ndarray   # [nmem][nflav][4]

    def member_subgrid(self, m, s):
        """Values of member m on sub-grid s as [nx][nq][nflav]."""
        off = 0
        for t in range(s):
            off += len(self.x[t]) * len(self.q[t]) * len(self.pids)
        nx, nq = len(self.x[s]), len(self.q[s])
        return self.xf[m, off:off + nx * nq * len(self.pids)].reshape(nx, nq, len(self.pids))


MB_THRESHOLD = 4.92   # GeV, the sub-grid boundary (b-quark mass, as in NNPDF3.1)


def synthetic_pdf_set(nmem=1, seed=0, nx=100, nq_low=8, nq_high=32, xmin=1e-7, qmin=1.65, qmax=1e4,
                      spread=0.05):
    """A multi-member, two-sub-grid stand-in for an LHAPDF set with a b-quark
    threshold: the x knots of synthetic_pdf_grid; Q knots log-spaced on
    [qmin, m_b] (nq_low) and [m_b, qmax] (nq_high), the threshold knot in both;
    member m draws its flavour parameters as synthetic_pdf_grid(seed) does and
    multiplies A, a, b, c by 1 + spread u, u uniform in [-1, 1] from
    SplitMix64(seed + 1000 + m) (member 0 is the central set, unperturbed);
    the b and b-bar densities vanish below the threshold."""
    x = np.array([10.0 ** (math.log10(xmin) * (1.0 - i / (nx - 1))) for i in range(nx)])
    x[-1] = 1.0
    q_lo = np.array([qmin * (MB_THRESHOLD / qmin) ** (j / (nq_low - 1)) for j in range(nq_low)])
    q_hi = np.array([MB_THRESHOLD * (qmax / MB_THRESHOLD) ** (j / (nq_high - 1)) for j in range(nq_high)])
    q_lo[-1] = q_hi[0] = MB_THRESHOLD
    base = synthetic_pdf_grid(seed).params
    nfl = len(PIDS)
    size = nx * (nq_low + nq_high) * nfl
    xf = np.empty((nmem, size))
    params = np.empty((nmem, nfl, 4))
    for m in range(nmem):
        rng = SplitMix64(seed + 1000 + m)
        pm = base.copy()
        if m > 0:
            for fl in range(nfl):
                for k in range(4):
                    pm[fl, k] *= 1.0 + spread * rng.uniform(-1.0, 1.0)
        params[m] = pm
        blocks = []
        for s, qk in enumerate((q_lo, q_hi)):
            v = np.empty((nx, len(qk), nfl))
            for fl, (A, a, b, c) in enumerate(pm):
                heavy_b = abs(PIDS[fl]) == 5
                for j, qj in enumerate(qk):
                    if heavy_b and s == 0:
                        v[:, j, fl] = 0.0
                        continue
                    lq = math.log(qj * qj / (qmin * qmin))
                    v[:, j, fl] = A * x ** (-a) * (1.0 - x) ** b * (1.0 + c * lq)
            blocks.append(v.reshape(-1))
        xf[m] = np.concatenate(blocks)
    return PdfSet(x=[x, x.copy()], q=[q_lo, q_hi], pids=np.array(PIDS, dtype=np.int32), xf=xf, params=params)


ALPHAS_MZ, MZ, MC_THRESHOLD = 0.118, 91.1876, 1.51


def synthetic_alphas_knots(qmin=1.0, qmax=1e4, per_segment=(6, 10, 40)):
    """alpha_s knots shaped like an LHAPDF set's: one-loop running
    alpha_s(Q) = 1 / (b0(nf) ln(Q^2 / Lambda_nf^2)), b0 = (33 - 2 nf) / (12 pi),
    with nf = 3 below m_c = 1.51 GeV, 4 up to m_b = 4.92 GeV and 5 above,
    Lambda_5 fixed by alpha_s(M_Z) = 0.118 and Lambda_4, Lambda_3 by continuity
    at the thresholds; Q knots log-spaced per segment, each threshold knot
    repeated (the end of one segment, the start of the next).  Returns (q, a)."""
    def b0(nf):
        return (33.0 - 2.0 * nf) / (12.0 * math.pi)
    lam2 = {5: MZ * MZ * math.exp(-1.0 / (b0(5) * ALPHAS_MZ))}
    a_b = 1.0 / (b0(5) * math.log(MB_THRESHOLD ** 2 / lam2[5]))
    lam2[4] = MB_THRESHOLD ** 2 * math.exp(-1.0 / (b0(4) * a_b))
    a_c = 1.0 / (b0(4) * math.log(MC_THRESHOLD ** 2 / lam2[4]))
    lam2[3] = MC_THRESHOLD ** 2 * math.exp(-1.0 / (b0(3) * a_c))
    edges = [(qmin, MC_THRESHOLD, 3), (MC_THRESHOLD, MB_THRESHOLD, 4), (MB_THRESHOLD, qmax, 5)]
    qs, als = [], []
    for (lo, hi, nf), n in zip(edges, per_segment):
        for j in range(n):
            qj = lo * (hi / lo) ** (j / (n - 1))
            qs.append(qj)
            als.append(1.0 / (b0(nf) * math.log(qj * qj / lam2[nf])))
    return np.array(qs), np.array(als)


@dataclass
class Integrand:
    """One integrand of the cross-section family (field order = C struct order)."""
    proc: int
    gauss_dim: int = 0
    sqrt_s: float = 13000.0
    m_top: float = 173.0
    alpha: float = 1.0 / 128.0
    alpha_s: float = 0.118
    mz: float = 91.1876
    gz: float = 2.4952
    sw2: float = 0.2312
    mu_f: float = 173.0
    ptcut_g: float = 20.0
    etacut_g: float = 2.5
    gauss_sigma: float = 0.1
    gev2pb: float = GEV2_TO_PB

    def ndim(self):
        return {EE_MUMU: 2, PP_TTBAR: 4, GG_TTBARG: 14, GG_TTBARG_7D: 7, GG_TTBARG_MC: 17, PP_TTBARJ: 7}.get(self.proc, self.gauss_dim)

    def asdict(self):
        return asdict(self)


def ee_mumu(sqrt_s=91.0):
    """e+e- -> mu+mu- via gamma + Z (2 dims: cos theta, phi)."""
    return Integrand(proc=EE_MUMU, sqrt_s=sqrt_s)


def pp_ttbar(sqrt_s=13000.0):
    """pp -> t tbar at LO, gg + q qbar (4 dims: x1, x2, cos theta, phi)."""
    return Integrand(proc=PP_TTBAR, sqrt_s=sqrt_s)


def gg_ttbarg(sqrt_s=13000.0):
    """gg -> t tbar g with RAMBO (2 + 12 dims), gluon pT > 20 GeV, |eta| < 2.5."""
    return Integrand(proc=GG_TTBARG, sqrt_s=sqrt_s)


def gg_ttbarg_7d(sqrt_s=13000.0):
    """gg -> t tbar g with the hierarchical three-body generator (2 + 5 = 7 dims), same cuts."""
    return Integrand(proc=GG_TTBARG_7D, sqrt_s=sqrt_s)


def gg_ttbarg_mc(sqrt_s=13000.0):
    """gg -> t tbar g with three-channel sampling (7 uniforms per event; a
    17-dimension VEGAS grid: x1, x2 and 5 dimensions per channel), same cuts."""
    return Integrand(proc=GG_TTBARG_MC, sqrt_s=sqrt_s)


def pp_ttbarj(sqrt_s=13000.0):
    """p p -> t tbar + one parton at LO (gg -> t tbar g, q qbar -> t tbar g,
    q g -> t tbar q and the charge conjugates), hierarchical 2 -> 3 phase
    space (2 + 5 = 7 dims), the parton with pT > 20 GeV, |eta| < 2.5."""
    return Integrand(proc=PP_TTBARJ, sqrt_s=sqrt_s)


def gauss(dim, sigma=0.1):
    """Normalised Gaussian centred at 1/2; integral over the cube erf(1/(2 sqrt2 sigma))^d."""
    return Integrand(proc=GAUSS, gauss_dim=dim, gauss_sigma=sigma, sqrt_s=0.0)


def gauss_exact(dim, sigma=0.1):
    return math.erf(0.5 / (sigma * math.sqrt(2.0))) ** dim


def batch_configs(seed=0):
    """Sixteen integrands of uneven dimension and size: e+e- -> mu+mu-, pp -> tt and
    gg -> ttg at sqrt(s) = 0.5, 2, 7, 13 TeV plus Gaussians in d = 4, 8, 12, 16; event
    counts N_i = round(10^(4 + 3 U_i)) with U_i from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    items = []
    for mk in (ee_mumu, pp_ttbar, gg_ttbarg):
        for rs in (500.0, 2000.0, 7000.0, 13000.0):
            items.append(mk(rs))
    for d in (4, 8, 12, 16):
        items.append(gauss(d))
    counts = [int(round(10.0 ** (4.0 + 3.0 * rng.uniform()))) for _ in items]
    return items, counts


def uniform_grid(ndim, nbins):
    """Initial VEGAS grid: nbins equal bins per dimension, [ndim][nbins+1]."""
    return np.tile(np.linspace(0.0, 1.0, nbins + 1), (ndim, 1))


def splitmix64_uniform(seed, n, offset=0):
    """n uniforms in [0, 1) from the SplitMix64 sequence of `seed` (vectorised)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def flow_layer_masks(D, L):
    """(conditioning dims, transformed dims) of each coupling layer: layer l
    transforms the dimensions d with d % 2 == l % 2."""
    return [([d for d in range(D) if d % 2 != l % 2], [d for d in range(D) if d % 2 == l % 2]) for l in range(L)]


def flow_init_params(D, L=6, K=32, hidden=256, seed=0, last_scale=0.0):
    """Initial flow parameters (FP32), one dict per coupling layer:
    W1 [hidden, d_A], b1, W2 [hidden, hidden], b2, W3, b3, W4 [d_B (2K+1), hidden], b4.
    Glorot-uniform weights from SplitMix64(seed), zero biases; the last layer is
    scaled by last_scale (0: the initial flow is the identity map)."""
    out = []
    off = 0
    for a, b in flow_layer_masks(D, L):
        shapes = [("W1", (hidden, len(a))), ("W2", (hidden, hidden)), ("W3", (hidden, hidden)),
                  ("W4", (len(b) * (2 * K + 1), hidden))]
        layer = {}
        for name, (fo, fi) in shapes:
            lim = math.sqrt(6.0 / (fo + fi))
            u = splitmix64_uniform(seed, fo * fi, off)
            off += fo * fi
            w = (2.0 * u - 1.0) * lim
            if name == "W4":
                w = w * last_scale
            layer[name] = w.reshape(fo, fi).astype(np.float32)
        for name, n in (("b1", hidden), ("b2", hidden), ("b3", hidden), ("b4", len(b) * (2 * K + 1))):
            layer[name] = np.zeros(n, dtype=np.float32)
        out.append(layer)
    return out
