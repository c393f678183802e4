"""FP64 CPU oracle (ctypes wrapper over oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA path is checked
against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
may import this package.  It shares no code with the CUDA path.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


class IntegrandC(ctypes.Structure):
    _fields_ = [("proc", ctypes.c_int32), ("gauss_dim", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in ("sqrt_s", "m_top", "alpha", "alpha_s", "mz", "gz", "sw2",
                                       "mu_f", "ptcut_g", "etacut_g", "gauss_sigma", "gev2pb")]


class EventRecord(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * 16), ("bin", ctypes.c_int32 * 16), ("jac", ctypes.c_double),
                ("p", (ctypes.c_double * 4) * 7), ("x1", ctypes.c_double), ("x2", ctypes.c_double),
                ("shat", ctypes.c_double), ("lumi", ctypes.c_double), ("lumi_qq", ctypes.c_double),
                ("me2", ctypes.c_double), ("me2_qq", ctypes.c_double), ("ps_weight", ctypes.c_double),
                ("f", ctypes.c_double), ("weight", ctypes.c_double), ("pass_", ctypes.c_int32),
                ("status", ctypes.c_int32), ("channel", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("me2_x", ctypes.c_double * 5), ("lumi_x", ctypes.c_double * 7)]


class LabEvent(ctypes.Structure):
    _fields_ = [("event", ctypes.c_int64), ("weight", ctypes.c_double), ("x1", ctypes.c_double),
                ("x2", ctypes.c_double), ("p", (ctypes.c_double * 4) * 5), ("proc", ctypes.c_int32),
                ("nout", ctypes.c_int32)]


class IterResult(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_double), ("sum2", ctypes.c_double), ("n", ctypes.c_int64),
                ("n_nonzero", ctypes.c_int64), ("wmax", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_d = ctypes.c_double


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_uniform_ints.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _u64p]
        L.orc_vegas_map.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _u64p, _dp, _i32p, _dp]
        L.orc_vegas_refine.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _d, _dp]
        L.orc_iteration_estimate.argtypes = [_d, _d, ctypes.c_int64, _dp, _dp]
        L.orc_combine.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.orc_two_body.argtypes = [_d, _d, _d, _d, _d, _dp, _dp]
        L.orc_rambo.argtypes = [ctypes.c_int, _dp, _d, _dp, _dp, _dp]
        L.orc_rambo.restype = ctypes.c_int
        L.orc_hierarchical.argtypes = [ctypes.c_int, _dp, _d, _dp, _dp, _dp]
        L.orc_hierarchical.restype = ctypes.c_int
        L.orc_pdf_new.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int, _i32p, _dp]
        L.orc_pdf_new.restype = ctypes.c_void_p
        L.orc_pdf_free.argtypes = [ctypes.c_void_p]
        L.orc_pdf_xfxq2.argtypes = [ctypes.c_void_p, ctypes.c_int, _d, _d]
        L.orc_pdf_xfxq2.restype = _d
        L.orc_pdfset_new.argtypes = [ctypes.c_int, _i32p, _i32p, _dp, _dp, ctypes.c_int, _i32p, ctypes.c_int, _dp]
        L.orc_pdfset_new.restype = ctypes.c_void_p
        L.orc_pdfset_free.argtypes = [ctypes.c_void_p]
        L.orc_pdfset_xfxq2.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _d, _d]
        L.orc_pdfset_xfxq2.restype = _d
        L.orc_alphas_new.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_alphas_new.restype = ctypes.c_void_p
        L.orc_alphas_free.argtypes = [ctypes.c_void_p]
        L.orc_alphas_q2.argtypes = [ctypes.c_void_p, _d]
        L.orc_alphas_q2.restype = _d
        L.orc_acceptance_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                              ctypes.c_int64, _dp]
        L.orc_unweight_accept.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                          ctypes.c_int64, _dp, _d, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_unweight_events.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp,
                                          ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int64, ctypes.c_int64, _d, _dp, ctypes.POINTER(LabEvent),
                                          ctypes.c_int64, _dp]
        L.orc_unweight_events.restype = ctypes.c_int64
        L.orc_set_channel_alpha.argtypes = [_dp]
        L.orc_channel_forward.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _dp, _dp, _dp]
        L.orc_channel_forward.restype = ctypes.c_int
        L.orc_channel_inverse.argtypes = [ctypes.c_int, _d, _d, _d, _d, _d, _dp, _dp, _dp]
        L.orc_channel_inverse.restype = ctypes.c_int
        L.orc_channels_event.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                         ctypes.POINTER(EventRecord), _dp]
        L.orc_channels_iterate.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_int64, ctypes.c_int64, _dp, _dp]
        L.orc_channel_update.argtypes = [ctypes.c_int, _dp, _dp, _d, _d, _dp]
        for name, args in [("orc_me2_eemumu", [_d] * 6), ("orc_me2_eemumu_trace", [_d] * 4 + [_dp]),
                           ("orc_me2_qqbar_ttbar", [_d] * 4), ("orc_me2_qqbar_ttbar_trace", [_d, _d, _dp]),
                           ("orc_me2_gg_ttbar", [_d] * 4), ("orc_me2_gg_ttbar_colour_ordered", [_d, _d, _dp]),
                           ("orc_me2_gg_ttbarg", [_d, _d, _dp]), ("orc_me2_gg_ttbarg_brute", [_d, _d, _dp]),
                           ("orc_me2_gg_ttbarg_helicity", [_d, _d, _dp])]:
            getattr(L, name).argtypes = args
            getattr(L, name).restype = _d
        for name in ("orc_me2_qqbar_ttbarg", "orc_me2_qg_ttbarq"):
            getattr(L, name).argtypes = [_d, _d, _dp]
            getattr(L, name).restype = _d
        L.orc_me2_qqbar_ttbarg_eps.argtypes = [_d, _d, _dp, _dp]
        L.orc_me2_qqbar_ttbarg_eps.restype = _d
        L.orc_ggttg_partial_amplitudes.argtypes = [_d, _d, _dp, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.orc_process_ndim.argtypes = [ctypes.POINTER(IntegrandC)]
        L.orc_process_ndim.restype = ctypes.c_int
        L.orc_event.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                ctypes.POINTER(EventRecord)]
        L.orc_weights.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int, _dp]
        L.orc_count_gg_ttbarg.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                          ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                          ctypes.c_int64, _dp]
        L.orc_iterate.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                  ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int, ctypes.POINTER(IterResult), _dp, _u32p]
        L.orc_integrate.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int,
                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, _d,
                                    ctypes.c_int, _dp, _dp, _dp, _dp]
        L.orc_integrand_at.argtypes = [ctypes.POINTER(IntegrandC), ctypes.c_void_p, ctypes.c_int64, _dp, _dp,
                                       ctypes.POINTER(ctypes.c_int32)]
        _LIB = L
    return _LIB


# ----------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def uniform_ints(seed, iteration, gid, prec, ndim, first, n):
    out = np.zeros((n, ndim), dtype=np.uint64)
    lib().orc_uniform_ints(seed, iteration, gid, prec, ndim, first, n, _ptr(out, _u64p))
    return out


def uniform_bits(prec):
    return 52 if prec == 0 else 23


# ----------------------------------------------------------------- VEGAS
def vegas_map(edges, prec, k):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    ndim, nb1 = edges.shape
    k = np.ascontiguousarray(k, dtype=np.uint64)
    x = np.zeros(ndim)
    bins = np.zeros(ndim, dtype=np.int32)
    jac = ctypes.c_double()
    lib().orc_vegas_map(ndim, nb1 - 1, _ptr(edges), prec, _ptr(k, _u64p), _ptr(x), _ptr(bins, _i32p),
                        ctypes.byref(jac))
    return x, bins, jac.value


def vegas_refine(edges, hist_w2, alpha=1.5):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    hist = np.ascontiguousarray(hist_w2, dtype=np.float64)
    ndim, nb1 = edges.shape
    out = np.zeros_like(edges)
    lib().orc_vegas_refine(ndim, nb1 - 1, _ptr(edges), _ptr(hist), alpha, _ptr(out))
    return out


def iteration_estimate(s, s2, n):
    m, v = ctypes.c_double(), ctypes.c_double()
    lib().orc_iteration_estimate(s, s2, n, ctypes.byref(m), ctypes.byref(v))
    return m.value, v.value


def combine(e, s2):
    e = np.ascontiguousarray(e, dtype=np.float64)
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    m, s, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_combine(len(e), _ptr(e), _ptr(s2), ctypes.byref(m), ctypes.byref(s), ctypes.byref(c))
    return m.value, s.value, c.value


# ----------------------------------------------------------------- phase space
def two_body(sqrt_s, m1, m2, cos_theta, phi):
    p = np.zeros((2, 4))
    w = ctypes.c_double()
    lib().orc_two_body(sqrt_s, m1, m2, cos_theta, phi, _ptr(p), ctypes.byref(w))
    return p, w.value


def rambo(masses, sqrt_s, u):
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = len(masses)
    p = np.zeros((n, 4))
    w = ctypes.c_double()
    rc = lib().orc_rambo(n, _ptr(masses), sqrt_s, _ptr(u), _ptr(p), ctypes.byref(w))
    return p, w.value, rc


def hierarchical(masses, sqrt_s, u):
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = len(masses)
    p = np.zeros((n, 4))
    w = ctypes.c_double()
    rc = lib().orc_hierarchical(n, _ptr(masses), sqrt_s, _ptr(u), _ptr(p), ctypes.byref(w))
    return p, w.value, rc


# ----------------------------------------------------------------- PDF
class Pdf:
    def __init__(self, grid):
        self.grid = grid
        x = np.ascontiguousarray(grid.x, dtype=np.float64)
        q = np.ascontiguousarray(grid.q, dtype=np.float64)
        pids = np.ascontiguousarray(grid.pids, dtype=np.int32)
        xf = np.ascontiguousarray(grid.xf, dtype=np.float64)
        self.handle = lib().orc_pdf_new(len(x), _ptr(x), len(q), _ptr(q), len(pids), _ptr(pids, _i32p),
                                        _ptr(xf))

    def xfxq2(self, pid, x, q2):
        return lib().orc_pdf_xfxq2(self.handle, pid, x, q2)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.orc_pdf_free(self.handle)
            self.handle = None


class PdfSet:
    """A PDF set of sub-grids and members (workloads.PdfSet) with LHAPDF's
    interpolation and extrapolation (oracle/src/pdfset.cpp)."""

    def __init__(self, pset):
        self.pset = pset
        nx = np.array([len(x) for x in pset.x], dtype=np.int32)
        nq = np.array([len(q) for q in pset.q], dtype=np.int32)
        x = np.ascontiguousarray(np.concatenate(pset.x), dtype=np.float64)
        q = np.ascontiguousarray(np.concatenate(pset.q), dtype=np.float64)
        pids = np.ascontiguousarray(pset.pids, dtype=np.int32)
        xf = np.ascontiguousarray(pset.xf, dtype=np.float64)
        self.handle = lib().orc_pdfset_new(len(nx), _ptr(nx, _i32p), _ptr(nq, _i32p), _ptr(x), _ptr(q), len(pids),
                                           _ptr(pids, _i32p), xf.shape[0], _ptr(xf))

    def xfxq2(self, member, pid, x, q2):
        return lib().orc_pdfset_xfxq2(self.handle, member, pid, x, q2)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.orc_pdfset_free(self.handle)
            self.handle = None


class AlphaS:
    """alpha_s(Q^2) interpolation on LHAPDF-style knots (oracle/src/pdfset.cpp)."""

    def __init__(self, q, a):
        q = np.ascontiguousarray(q, dtype=np.float64)
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.handle = lib().orc_alphas_new(len(q), _ptr(q), _ptr(a))

    def __call__(self, q2):
        return lib().orc_alphas_q2(self.handle, q2)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.orc_alphas_free(self.handle)
            self.handle = None


# ----------------------------------------------------------------- unweighting
def acceptance_uniforms(seed, iteration, gid, first, n):
    """The acceptance-rejection uniforms r_i of events first .. first+n-1."""
    r = np.empty(n)
    lib().orc_acceptance_uniforms(seed, iteration, gid, first, n, _ptr(r))
    return r


def unweight_accept(seed, iteration, gid, first, weights, wmax):
    """Boolean mask of the events accepted by w_i > r_i w_max."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    acc = np.zeros(len(w), dtype=np.uint8)
    lib().orc_unweight_accept(seed, iteration, gid, first, len(w), _ptr(w), wmax,
                              acc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return acc.astype(bool)


def unweight_events(itg, pdf, edges, prec, seed, iteration, gid, first, n, wmax=0.0, cap=None):
    """Unweighted sample of events first .. first+n-1 of one iteration:
    returns (weights [n], w_max used, list of accepted LabEvent in event
    order, number accepted).  wmax <= 0: the largest weight of the sample."""
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    cap = n if cap is None else cap
    w = np.zeros(n)
    out = (LabEvent * max(cap, 1))()
    wm = ctypes.c_double()
    nacc = lib().orc_unweight_events(ctypes.byref(c), pdf.handle if pdf is not None else None, edges.shape[1] - 1,
                                     _ptr(edges), prec, seed, iteration, gid, first, n, wmax, _ptr(w), out, cap,
                                     ctypes.byref(wm))
    if nacc < 0:
        raise ValueError("process has no event record")
    return w, wm.value, list(out[:min(nacc, cap)]), nacc


# ----------------------------------------------------------------- channels
def set_channel_alpha(alpha):
    """Channel probabilities of the multi-channel process (normalised)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    lib().orc_set_channel_alpha(_ptr(a))


def channel_forward(ch, m, rs, ptcut, etacut, yb, u):
    """Channel ch's map of u[5] at partonic energy rs (cuts pT > ptcut,
    |eta + yb| < etacut): (momenta [3][4] t, tbar, g, weight) or None."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.zeros((3, 4))
    w = ctypes.c_double()
    if lib().orc_channel_forward(ch, m, rs, ptcut, etacut, yb, _ptr(u), _ptr(p), ctypes.byref(w)):
        return None
    return p, w.value


def channel_inverse(ch, m, rs, ptcut, etacut, yb, p):
    """The channel-ch variables of the momenta p [3][4] and the channel's
    weight there, or None outside its support."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.zeros(5)
    w = ctypes.c_double()
    if lib().orc_channel_inverse(ch, m, rs, ptcut, etacut, yb, _ptr(p), _ptr(u), ctypes.byref(w)):
        return None
    return u, w.value


def channels_event(itg, pdf, edges, prec, seed, iteration, gid, ev):
    """One multi-channel event: (EventRecord, densities of the three channels)."""
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    rec = EventRecord()
    dens = np.zeros(3)
    lib().orc_channels_event(ctypes.byref(c), pdf.handle if pdf is not None else None, edges.shape[1] - 1,
                             _ptr(edges), prec, seed, iteration, gid, ev, ctypes.byref(rec), _ptr(dens))
    return rec, dens


def channels_iterate(itg, pdf, edges, prec, seed, iteration, gid, first, n):
    """(sum w, sum w^2, w_max) and the alpha-update sums W[3] of n events."""
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    sums = np.zeros(3)
    wch = np.zeros(3)
    lib().orc_channels_iterate(ctypes.byref(c), pdf.handle if pdf is not None else None, edges.shape[1] - 1,
                               _ptr(edges), prec, seed, iteration, gid, first, n, _ptr(sums), _ptr(wch))
    return sums, wch


def channel_update(alpha, w, beta=0.5, amin=0.0):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(len(a))
    lib().orc_channel_update(len(a), _ptr(a), _ptr(ww), beta, amin, _ptr(out))
    return out


# ----------------------------------------------------------------- |M|^2
def me2_eemumu(alpha, mz, gz, sw2, s, c):
    return lib().orc_me2_eemumu(alpha, mz, gz, sw2, s, c)


def me2_eemumu_trace(alpha, mz, gz, sw2, p):
    return lib().orc_me2_eemumu_trace(alpha, mz, gz, sw2, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


def me2_qqbar_ttbar(alpha_s, mt, s, t):
    return lib().orc_me2_qqbar_ttbar(alpha_s, mt, s, t)


def me2_qqbar_ttbar_trace(alpha_s, mt, p):
    return lib().orc_me2_qqbar_ttbar_trace(alpha_s, mt, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


def me2_gg_ttbar(alpha_s, mt, s, t):
    return lib().orc_me2_gg_ttbar(alpha_s, mt, s, t)


def me2_gg_ttbar_colour_ordered(alpha_s, mt, p):
    return lib().orc_me2_gg_ttbar_colour_ordered(alpha_s, mt, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


def me2_gg_ttbarg(alpha_s, mt, p):
    return lib().orc_me2_gg_ttbarg(alpha_s, mt, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


def me2_qqbar_ttbarg(alpha_s, mt, p):
    """<|M|^2> of q(p0) qbar(p1) -> t(p2) tbar(p3) g(p4); p [5][4]."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    return lib().orc_me2_qqbar_ttbarg(alpha_s, mt, _ptr(p))


def me2_qg_ttbarq(alpha_s, mt, p):
    """<|M|^2> of q(p0) g(p1) -> t(p2) tbar(p3) q(p4) (crossing); p [5][4]."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    return lib().orc_me2_qg_ttbarq(alpha_s, mt, _ptr(p))


def me2_qqbar_ttbarg_eps(alpha_s, mt, p, eps):
    """Spin- and colour-summed |M|^2 /36 with the gluon polarisation replaced by eps [4] (complex)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    e = np.ascontiguousarray(np.stack([np.real(eps), np.imag(eps)], axis=1).reshape(-1), dtype=np.float64)
    return lib().orc_me2_qqbar_ttbarg_eps(alpha_s, mt, _ptr(p), _ptr(e))


def me2_gg_ttbarg_helicity(alpha_s, mt, p):
    """Formulation C: helicity amplitudes on spinors (oracle/src/helicity_t.h)."""
    return lib().orc_me2_gg_ttbarg_helicity(alpha_s, mt, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


COUNT_STEPS = ("map", "rambo", "cuts", "pdf", "me2", "weight")
COUNT_KINDS = ("add", "mul", "div", "sqrt", "fn")


def count_gg_ttbarg(itg, pdf, edges, prec, seed, iteration, gid, first, n):
    """Algorithmic operation counts of events [first, first + n) of one g g ->
    t tbar g (RAMBO) iteration: {"events", "in_cuts", step: {kind: total}}."""
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros(3 + 5 * len(COUNT_STEPS))
    lib().orc_count_gg_ttbarg(ctypes.byref(c), pdf.handle, edges.shape[1] - 1, _ptr(edges), prec, seed, iteration,
                              gid, first, n, _ptr(out))
    res = {"events": int(out[0]), "in_cuts": int(out[1]), "sum_w": float(out[-1])}
    for k, st in enumerate(COUNT_STEPS):
        res[st] = {kind: int(out[2 + 5 * k + j]) for j, kind in enumerate(COUNT_KINDS)}
    return res


def me2_gg_ttbarg_brute(alpha_s, mt, p):
    return lib().orc_me2_gg_ttbarg_brute(alpha_s, mt, _ptr(np.ascontiguousarray(p, dtype=np.float64)))


def ggttg_partial_amplitudes(alpha_s, mt, q_in, eps, ubar, v):
    """q_in: [n+1][4] incoming gluon momenta then the top momentum; eps: [n][4]
    complex; ubar, v: [4] complex (Dirac representation).  Returns n! amplitudes
    in lexicographic order of the gluon orderings."""
    n = len(eps)
    q = np.ascontiguousarray(q_in, dtype=np.float64)
    e = np.ascontiguousarray(np.stack([np.asarray(eps).real, np.asarray(eps).imag], -1), dtype=np.float64)
    ub = np.ascontiguousarray(np.stack([np.asarray(ubar).real, np.asarray(ubar).imag], -1), dtype=np.float64)
    vv = np.ascontiguousarray(np.stack([np.asarray(v).real, np.asarray(v).imag], -1), dtype=np.float64)
    out = np.zeros((6, 2))
    lib().orc_ggttg_partial_amplitudes(alpha_s, mt, _ptr(q), _ptr(e), n, _ptr(ub), _ptr(vv), _ptr(out))
    k = 2 if n == 2 else 6
    return out[:k, 0] + 1j * out[:k, 1]


# ----------------------------------------------------------------- integrand
def _integrand_c(itg):
    d = itg.asdict() if hasattr(itg, "asdict") else dict(itg)
    return IntegrandC(**d)


def process_ndim(itg):
    c = _integrand_c(itg)
    return lib().orc_process_ndim(ctypes.byref(c))


def event(itg, pdf, edges, prec, seed, iteration, gid, ev):
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    rec = EventRecord()
    lib().orc_event(ctypes.byref(c), pdf.handle if pdf is not None else None, edges.shape[1] - 1,
                    _ptr(edges), prec, seed, iteration, gid, ev, ctypes.byref(rec))
    return rec


def integrand_at(itg, pdf, x):
    """Integrand f at the points x [n, ndim] of the unit hypercube; returns (f, status)."""
    c = _integrand_c(itg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    f = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    lib().orc_integrand_at(ctypes.byref(c), pdf.handle if pdf is not None else None, n, _ptr(x), _ptr(f),
                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return f, st


def iterate(itg, pdf, edges, prec, seed, iteration, gid, first, n, nthreads=0):
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    ndim, nb1 = edges.shape
    hist = np.zeros((ndim, nb1 - 1))
    cnt = np.zeros((ndim, nb1 - 1), dtype=np.uint32)
    res = IterResult()
    lib().orc_iterate(ctypes.byref(c), pdf.handle if pdf is not None else None, nb1 - 1, _ptr(edges), prec,
                      seed, iteration, gid, first, n, nthreads, ctypes.byref(res), _ptr(hist), _ptr(cnt, _u32p))
    return dict(sum=res.sum, sum2=res.sum2, n=res.n, n_nonzero=res.n_nonzero, wmax=res.wmax,
                hist_w2=hist, hist_n=cnt)


def weights(itg, pdf, edges, prec, seed, iteration, gid, first, n, nthreads=0):
    """Per-event weights w = f J of events [first, first + n) of one iteration."""
    c = _integrand_c(itg)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    w = np.zeros(n)
    lib().orc_weights(ctypes.byref(c), pdf.handle if pdf is not None else None, edges.shape[1] - 1, _ptr(edges),
                      prec, seed, iteration, gid, first, n, nthreads, _ptr(w))
    return w


def integrate(itg, pdf, edges, prec, seed, gid, niter, nevents, alpha=1.5, nthreads=0):
    c = _integrand_c(itg)
    edges = np.array(edges, dtype=np.float64, copy=True)
    ndim, nb1 = edges.shape
    per = np.zeros((niter, 2))
    m, s, chi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_integrate(ctypes.byref(c), pdf.handle if pdf is not None else None, nb1 - 1, _ptr(edges), prec,
                        seed, gid, niter, nevents, alpha, nthreads, _ptr(per), ctypes.byref(m), ctypes.byref(s),
                        ctypes.byref(chi))
    return dict(mean=m.value, sigma=s.value, chi2dof=chi.value, per_iter=per, edges=edges)
