"""Thin ctypes binding of libmcint.so (C ABI in include/mcint.h).

Argument marshalling only: every step of the Monte Carlo path runs in the CUDA
library.  Device buffers are passed as raw pointers (e.g. a torch tensor's
data_ptr()), streams as the integer handle of a cudaStream_t.  A non-zero
status raises McError with the library's message.  The library must have been
built (python -m paper_2302_03343_b300.build); there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import workloads

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmcint.so")

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ENAN, MC_ENOCONV, MC_ETIMEOUT, MC_EIO = 0, -1, -2, -3, -4, -5, -6, -7
MC_FP64, MC_FP32_KAHAN = 0, 1
MC_EE_MUMU, MC_PP_TTBAR, MC_GG_TTBARG, MC_GAUSS, MC_GG_TTBARG_7D, MC_GG_TTBARG_MC, MC_PP_TTBARJ = 0, 1, 2, 3, 4, 5, 6
MC_MAX_DIM, MC_MAX_BINS = 17, 256
REC = dict(K=0, X=16, BIN=32, JAC=48, P=49, X1=77, X2=78, SHAT=79, LUMI=80, LUMI_QQ=81, ME2=82, ME2_QQ=83,
           PSW=84, F=85, W=86, PASS=87, STATUS=88, CHANNEL=89, DENS=90, ME2_X=89)
REC_STRIDE = 96

# exported symbols (each declared in include/mcint.h)
SYMBOLS = ("mc_last_error", "mc_pdf_load", "mc_pdf_free", "mc_pdf_xfxq2", "mc_vegas_init", "mc_vegas_free",
           "mc_vegas_set_grid", "mc_vegas_get_grid", "mc_vegas_get_hist", "mc_vegas_set_hist",
           "mc_vegas_iterate_shard", "mc_vegas_set_iteration",
           "mc_vegas_get_iteration", "mc_vegas_set_gid", "mc_vegas_iterate", "mc_vegas_refine", "mc_integrate",
           "mc_debug_events", "mc_launch_shape", "mc_vegas_kernel_ms", "mc_vegas_iterate_noalloc",
           "mc_batch_create", "mc_batch_iterate", "mc_batch_get_grid", "mc_batch_shape", "mc_batch_kernel_ms",
           "mc_batch_free", "mc_gemm_bf16", "mc_gemm_bf16_rs", "mc_gemm_bf16_tn", "mc_gemm_bf16_xn", "mc_flow_param_count", "mc_flow_create", "mc_flow_free",
           "mc_flow_set_params", "mc_flow_get_params", "mc_flow_forward", "mc_flow_loss_grad", "mc_flow_adam_step",
           "mc_flow_train", "mc_flow_iterate", "mc_flow_set_fused", "mc_integrate_flow", "mc_pdfset_load",
           "mc_pdfset_free", "mc_pdfset_xfxq2", "mc_alphas_load", "mc_alphas_free", "mc_alphas_q2",
           "mc_vegas_iterate_weights", "mc_unweight", "mc_unweight_ms", "mc_lhe_open", "mc_lhe_write",
           "mc_lhe_write_device", "mc_lhe_close", "mc_generate_lhe", "mc_vegas_set_channels", "mc_vegas_get_channels",
           "mc_channel_update", "mc_fma_peak", "mc_flow_grad_count", "mc_flow_step_sample", "mc_flow_step_grads",
           "mc_flow_step_apply")

# mc_event (include/mcint.h): one accepted event in the laboratory frame, 200 bytes
EVENT_DTYPE = np.dtype([("event", "<i8"), ("weight", "<f8"), ("x1", "<f8"), ("x2", "<f8"), ("p", "<f8", (5, 4)),
                        ("proc", "<i4"), ("nout", "<i4")])
assert EVENT_DTYPE.itemsize == 200


class McError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mcint error {code}: {msg}")
        self.code = code


class Integrand(ctypes.Structure):
    _fields_ = [("proc", ctypes.c_int32), ("gauss_dim", ctypes.c_int32)] + [
        (n, ctypes.c_double) for n in ("sqrt_s", "m_top", "alpha", "alpha_s", "mz", "gz", "sw2", "mu_f", "ptcut_g",
                                       "etacut_g", "gauss_sigma", "gev2pb")]


class IterResult(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_double), ("sum2", ctypes.c_double), ("n", ctypes.c_int64),
                ("n_nonzero", ctypes.c_int64), ("wmax", ctypes.c_double), ("n_bad", ctypes.c_int64),
                ("status", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class FlowCfg(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("layers", ctypes.c_int32), ("bins", ctypes.c_int32),
                ("hidden", ctypes.c_int32)]


class GenStats(ctypes.Structure):
    _fields_ = [("n_weighted", ctypes.c_int64), ("n_accepted", ctypes.c_int64), ("iterate_ms", ctypes.c_double),
                ("unweight_ms", ctypes.c_double), ("wall_ms", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
                ("n_iter", ctypes.c_int32), ("status", ctypes.c_int32), ("gpu_ms", ctypes.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def lib():
    """Load libmcint.so; raises if it is missing (no CPU fallback exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise McError(MC_EINVAL, f"{LIB_PATH} not built: run python -m paper_2302_03343_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        L.mc_last_error.restype = ctypes.c_char_p
        i64, i32, u32, u64, d = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        sig = {
            "mc_pdf_load": [_dp, i32, _dp, i32, ctypes.POINTER(ctypes.c_int32), i32, _dp, ctypes.POINTER(_vp)],
            "mc_pdf_free": [_vp],
            "mc_pdf_xfxq2": [_vp, i32, i64, _vp, _vp, _vp, _vp],
            "mc_vegas_init": [i32, i32, u64, i32, ctypes.POINTER(_vp)],
            "mc_vegas_free": [_vp],
            "mc_vegas_set_grid": [_vp, _dp],
            "mc_vegas_get_grid": [_vp, _dp],
            "mc_vegas_get_hist": [_vp, _dp, ctypes.POINTER(ctypes.c_uint32)],
            "mc_vegas_set_hist": [_vp, _dp, ctypes.POINTER(ctypes.c_uint32)],
            "mc_vegas_iterate_shard": [_vp, _vp, _vp, i64, i64, _vp, _vp],
            "mc_vegas_set_iteration": [_vp, u32],
            "mc_vegas_get_iteration": [_vp, ctypes.POINTER(ctypes.c_uint32)],
            "mc_vegas_set_gid": [_vp, u32],
            "mc_vegas_iterate": [_vp, ctypes.POINTER(Integrand), _vp, i64, _vp, ctypes.POINTER(IterResult)],
            "mc_vegas_refine": [_vp, d, _vp],
            "mc_integrate": [ctypes.POINTER(Integrand), _vp, i32, i64, i32, u64, u32, i32, d, d, _vp,
                             ctypes.POINTER(Result), ctypes.POINTER(IterResult)],
            "mc_debug_events": [_vp, ctypes.POINTER(Integrand), _vp, i64, i64, _vp, _vp],
            "mc_launch_shape": [ctypes.POINTER(Integrand), i32, i64, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)],
            "mc_vegas_kernel_ms": [_vp, ctypes.POINTER(ctypes.c_float)],
            "mc_fma_peak": [i32, i32, _vp, i64, _dp, _vp],
            "mc_batch_create": [i32, ctypes.POINTER(Integrand), ctypes.POINTER(ctypes.c_int64), _vp, i32, u64, i32,
                                ctypes.POINTER(_vp)],
            "mc_batch_iterate": [_vp, d, _vp, ctypes.POINTER(IterResult)],
            "mc_batch_get_grid": [_vp, i32, _dp],
            "mc_batch_shape": [_vp] + [ctypes.POINTER(ctypes.c_int)] * 4,
            "mc_batch_kernel_ms": [_vp, ctypes.POINTER(ctypes.c_float)],
            "mc_batch_free": [_vp],
            "mc_gemm_bf16": [i32, i32, i32, i32, i32, _vp, i32, _vp, i32, _vp, _vp, i32, _vp, i32, i32, _vp, _vp],
            "mc_gemm_bf16_tn": [i32, i32, i32, i32, i32, _vp, i32, _vp, i32, _vp, i32, i32, _vp, _vp],
            "mc_gemm_bf16_xn": [i32, i32, i32, i32, i32, _vp, i32, _vp, i32, _vp, i32, i32, _vp, _vp],
            "mc_gemm_bf16_rs": [i32, i32, i32, i32, i32, _vp, i32, _vp, i32, _vp, _vp, i32, _vp, i32, _vp, i32, _vp,
                                _vp],
            "mc_vegas_iterate_noalloc": [ctypes.POINTER(Integrand), _vp, i32, i32, _vp, _vp, i32, u64, u32, u32,
                                         i64, i32, _vp, _vp, _vp, _vp],
            "mc_flow_grad_count": [_vp, ctypes.POINTER(ctypes.c_int64)],
            "mc_flow_step_sample": [_vp, ctypes.POINTER(Integrand), _vp, i64, i64, _vp, _dp],
            "mc_flow_step_grads": [_vp, d, _vp, _vp],
            "mc_flow_step_apply": [_vp, _vp, d, _vp],
            "mc_flow_param_count": [ctypes.POINTER(FlowCfg), ctypes.POINTER(ctypes.c_int64)],
            "mc_flow_create": [ctypes.POINTER(FlowCfg), _fp, i64, u64, ctypes.POINTER(_vp)],
            "mc_flow_free": [_vp],
            "mc_flow_set_params": [_vp, _fp],
            "mc_flow_get_params": [_vp, _fp],
            "mc_flow_forward": [_vp, i64, _vp, _vp, _vp, _vp],
            "mc_flow_loss_grad": [_vp, i64, _vp, _vp, _dp, _fp, _vp],
            "mc_flow_adam_step": [_vp, d, _vp],
            "mc_flow_set_fused": [_vp, i32],
            "mc_integrate_flow": [ctypes.POINTER(Integrand), _vp, ctypes.POINTER(FlowCfg), _fp, i32, i64, d, i32, i64,
                                  i32, u64, d, _vp, ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_int)],
            "mc_flow_train": [_vp, ctypes.POINTER(Integrand), _vp, i32, i64, d, _vp, _dp],
            "mc_flow_iterate": [_vp, ctypes.POINTER(Integrand), _vp, i64, u32, _vp, ctypes.POINTER(IterResult)],
            "mc_pdfset_load": [i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp, _dp, i32,
                               ctypes.POINTER(ctypes.c_int), i32, _dp, ctypes.POINTER(_vp)],
            "mc_pdfset_free": [_vp],
            "mc_pdfset_xfxq2": [_vp, i32, i32, i32, i64, _vp, _vp, _vp, _vp],
            "mc_alphas_load": [i32, _dp, _dp, ctypes.POINTER(_vp)],
            "mc_alphas_free": [_vp],
            "mc_alphas_q2": [_vp, i64, _vp, _vp, _vp],
            "mc_vegas_iterate_weights": [_vp, ctypes.POINTER(Integrand), _vp, i64, _vp, _vp,
                                         ctypes.POINTER(IterResult)],
            "mc_unweight": [_vp, ctypes.POINTER(Integrand), _vp, _vp, i64, d, _vp, i64, ctypes.POINTER(ctypes.c_int64),
                            _vp],
            "mc_unweight_ms": [_vp, ctypes.POINTER(ctypes.c_float)],
            "mc_lhe_open": [ctypes.c_char_p, ctypes.POINTER(Integrand), i32, ctypes.POINTER(_vp)],
            "mc_lhe_write": [_vp, _vp, i64],
            "mc_lhe_write_device": [_vp, _vp, i64, _vp],
            "mc_lhe_close": [_vp, d, d, d, ctypes.POINTER(ctypes.c_int64)],
            "mc_vegas_set_channels": [_vp, _dp],
            "mc_vegas_get_channels": [_vp, _dp, _dp],
            "mc_channel_update": [i32, _dp, _dp, d, d, _dp],
            "mc_generate_lhe": [ctypes.POINTER(Integrand), _vp, i32, i32, i64, i32, u64, i32, d, ctypes.c_char_p, i32,
                                _vp, ctypes.POINTER(Result), ctypes.POINTER(GenStats)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(rc):
    if rc != MC_OK:
        raise McError(rc, lib().mc_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(x):
    """Device pointer of a torch tensor (or an int)."""
    return ctypes.c_void_p(x.data_ptr() if hasattr(x, "data_ptr") else int(x))


def _integrand(itg):
    if isinstance(itg, Integrand):
        return itg
    d = itg.asdict() if hasattr(itg, "asdict") else dict(itg)
    return Integrand(**d)


# ------------------------------------------------------------------ PDF
class Pdf:
    """Owns an mc_pdf handle (device copy of an LHAPDF-style grid)."""

    def __init__(self, handle, nflav, pids):
        self.handle, self.nflav, self.pids = handle, nflav, pids

    def free(self):
        if self.handle:
            mc_pdf_free(self)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_pdf_load(grid):
    x = np.ascontiguousarray(grid.x, dtype=np.float64)
    q = np.ascontiguousarray(grid.q, dtype=np.float64)
    pids = np.ascontiguousarray(grid.pids, dtype=np.int32)
    xf = np.ascontiguousarray(grid.xf, dtype=np.float64)
    h = _vp()
    _check(lib().mc_pdf_load(x.ctypes.data_as(_dp), len(x), q.ctypes.data_as(_dp), len(q),
                             pids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(pids), xf.ctypes.data_as(_dp),
                             ctypes.byref(h)))
    return Pdf(h, len(pids), tuple(int(p) for p in pids))


def mc_pdf_free(pdf):
    _check(lib().mc_pdf_free(pdf.handle))


def mc_pdf_xfxq2(pdf, prec, n, x_dev, q2_dev, out_dev, stream=None):
    _check(lib().mc_pdf_xfxq2(pdf.handle, prec, n, _ptr(x_dev), _ptr(q2_dev), _ptr(out_dev), _stream(stream)))


# ---------------------------------------------------------------- PDF sets
class PdfSet:
    """Owns an mc_pdfset handle (sub-grids and members on the device)."""

    def __init__(self, handle, nflav, nmem, pids):
        self.handle, self.nflav, self.nmem, self.pids = handle, nflav, nmem, pids

    def free(self):
        if self.handle:
            mc_pdfset_free(self)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_pdfset_load(pset):
    """Load a workloads.PdfSet (x, q per sub-grid; xf [member][...])."""
    nx = np.array([len(x) for x in pset.x], dtype=np.int32)
    nq = np.array([len(q) for q in pset.q], dtype=np.int32)
    x = np.ascontiguousarray(np.concatenate(pset.x), dtype=np.float64)
    q = np.ascontiguousarray(np.concatenate(pset.q), dtype=np.float64)
    pids = np.ascontiguousarray(pset.pids, dtype=np.int32)
    xf = np.ascontiguousarray(pset.xf, dtype=np.float64)
    ip = ctypes.POINTER(ctypes.c_int)
    h = _vp()
    _check(lib().mc_pdfset_load(len(nx), nx.ctypes.data_as(ip), nq.ctypes.data_as(ip), x.ctypes.data_as(_dp),
                                q.ctypes.data_as(_dp), len(pids), pids.ctypes.data_as(ip), xf.shape[0],
                                xf.ctypes.data_as(_dp), ctypes.byref(h)))
    return PdfSet(h, len(pids), xf.shape[0], tuple(int(p) for p in pids))


def mc_pdfset_free(pset):
    _check(lib().mc_pdfset_free(pset.handle))


def mc_pdfset_xfxq2(pset, prec, member0, nmem, n, x_dev, q2_dev, out_dev, stream=None):
    _check(lib().mc_pdfset_xfxq2(pset.handle, prec, member0, nmem, n, _ptr(x_dev), _ptr(q2_dev), _ptr(out_dev),
                                 _stream(stream)))


class AlphaS:
    """Owns an mc_alphas handle."""

    def __init__(self, handle):
        self.handle = handle

    def free(self):
        if self.handle:
            _check(lib().mc_alphas_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_alphas_load(q, alphas):
    q = np.ascontiguousarray(q, dtype=np.float64)
    a = np.ascontiguousarray(alphas, dtype=np.float64)
    h = _vp()
    _check(lib().mc_alphas_load(len(q), q.ctypes.data_as(_dp), a.ctypes.data_as(_dp), ctypes.byref(h)))
    return AlphaS(h)


def mc_alphas_free(a):
    a.free()


def mc_alphas_q2(a, n, q2_dev, out_dev, stream=None):
    _check(lib().mc_alphas_q2(a.handle, n, _ptr(q2_dev), _ptr(out_dev), _stream(stream)))


# ---------------------------------------------------------------- VEGAS
class Vegas:
    """Owns an mc_vegas handle."""

    def __init__(self, handle, ndim, nbins, prec):
        self.handle, self.ndim, self.nbins, self.prec = handle, ndim, nbins, prec

    def free(self):
        if self.handle:
            _check(lib().mc_vegas_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_vegas_init(ndim, nbins, seed, prec):
    h = _vp()
    _check(lib().mc_vegas_init(ndim, nbins, seed, prec, ctypes.byref(h)))
    return Vegas(h, ndim, nbins, prec)


def mc_vegas_free(v):
    v.free()


def mc_vegas_set_grid(v, edges):
    e = np.ascontiguousarray(edges, dtype=np.float64)
    assert e.shape == (v.ndim, v.nbins + 1)
    _check(lib().mc_vegas_set_grid(v.handle, e.ctypes.data_as(_dp)))


def mc_vegas_get_grid(v):
    e = np.zeros((v.ndim, v.nbins + 1))
    _check(lib().mc_vegas_get_grid(v.handle, e.ctypes.data_as(_dp)))
    return e


def mc_vegas_get_hist(v):
    w2 = np.zeros((v.ndim, v.nbins))
    n = np.zeros((v.ndim, v.nbins), dtype=np.uint32)
    _check(lib().mc_vegas_get_hist(v.handle, w2.ctypes.data_as(_dp), n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return w2, n


def mc_vegas_set_hist(v, w2, counts):
    w2 = np.ascontiguousarray(w2, dtype=np.float64)
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    if w2.shape != (v.ndim, v.nbins) or counts.shape != (v.ndim, v.nbins):
        raise ValueError("histograms must be [ndim][nbins]")
    _check(lib().mc_vegas_set_hist(v.handle, w2.ctypes.data_as(_dp),
                                   counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))


def mc_vegas_set_iteration(v, it):
    _check(lib().mc_vegas_set_iteration(v.handle, it))


def mc_vegas_get_iteration(v):
    it = ctypes.c_uint32()
    _check(lib().mc_vegas_get_iteration(v.handle, ctypes.byref(it)))
    return it.value


def mc_vegas_set_gid(v, gid):
    _check(lib().mc_vegas_set_gid(v.handle, gid))


def mc_vegas_iterate(v, itg, pdf, nevents, stream=None):
    r = IterResult()
    c = _integrand(itg)
    _check(lib().mc_vegas_iterate(v.handle, ctypes.byref(c), pdf.handle if pdf else None, nevents,
                                  _stream(stream), ctypes.byref(r)))
    return r


def mc_vegas_iterate_shard(v, itg, pdf, first, count, stream=None):
    r = IterResult()
    c = _integrand(itg)
    _check(lib().mc_vegas_iterate_shard(v.handle, ctypes.byref(c), pdf.handle if pdf else None, first, count,
                                        _stream(stream), ctypes.byref(r)))
    return r


def mc_vegas_iterate_weights(v, itg, pdf, nevents, weights_dev, stream=None):
    """mc_vegas_iterate that also writes every event's weight to weights_dev
    (device FP64 [nevents])."""
    r = IterResult()
    c = _integrand(itg)
    _check(lib().mc_vegas_iterate_weights(v.handle, ctypes.byref(c), pdf.handle if pdf else None, nevents,
                                          _ptr(weights_dev), _stream(stream), ctypes.byref(r)))
    return r


def mc_unweight(v, itg, pdf, weights_dev, nevents, wmax, events_dev, capacity, stream=None):
    """Unweighted sample of the last iteration: writes up to `capacity` mc_event
    records (device buffer of capacity * 200 bytes) and returns the number
    accepted."""
    c = _integrand(itg)
    n = ctypes.c_int64()
    _check(lib().mc_unweight(v.handle, ctypes.byref(c), pdf.handle if pdf else None, _ptr(weights_dev), nevents,
                             wmax, _ptr(events_dev) if capacity else None, capacity, ctypes.byref(n),
                             _stream(stream)))
    return n.value


def mc_unweight_ms(v):
    ms = ctypes.c_float()
    _check(lib().mc_unweight_ms(v.handle, ctypes.byref(ms)))
    return ms.value


class Lhe:
    """Owns an mc_lhe writer; close() returns the number of events written."""

    def __init__(self, handle):
        self.handle = handle

    def close(self, xsec=0.0, xerr=0.0, wmax=0.0):
        n = ctypes.c_int64()
        h, self.handle = self.handle, None
        _check(lib().mc_lhe_close(h, xsec, xerr, wmax, ctypes.byref(n)))
        return n.value

    def __del__(self):
        if self.handle:
            try:
                self.close()
            except Exception:
                pass


def mc_lhe_open(path, itg, threads=4):
    h = _vp()
    c = _integrand(itg)
    _check(lib().mc_lhe_open(os.fsencode(path), ctypes.byref(c), threads, ctypes.byref(h)))
    return Lhe(h)


def mc_lhe_write(lhe, events):
    """Queue host events (a numpy array of EVENT_DTYPE)."""
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    _check(lib().mc_lhe_write(lhe.handle, ev.ctypes.data_as(_vp), len(ev)))


def mc_lhe_write_device(lhe, events_dev, n, stream=None):
    _check(lib().mc_lhe_write_device(lhe.handle, _ptr(events_dev), n, _stream(stream)))


def mc_lhe_close(lhe, xsec=0.0, xerr=0.0, wmax=0.0):
    return lhe.close(xsec, xerr, wmax)


def mc_generate_lhe(itg, pdf, path, ntrain, niter, nevents, nbins=50, seed=0, prec=MC_FP64, alpha=1.5, threads=4,
                    stream=None):
    """Train the grid, then generate unweighted events to an LHE file; returns
    (Result, GenStats)."""
    c = _integrand(itg)
    out, st = Result(), GenStats()
    _check(lib().mc_generate_lhe(ctypes.byref(c), pdf.handle if pdf else None, ntrain, niter, nevents, nbins, seed,
                                 prec, alpha, os.fsencode(path), threads, _stream(stream), ctypes.byref(out),
                                 ctypes.byref(st)))
    return out, st


def events_from_bytes(buf):
    """View raw mc_event bytes (e.g. a uint8 tensor copied to the host) as records."""
    return np.frombuffer(memoryview(buf), dtype=EVENT_DTYPE)


def mc_vegas_set_channels(v, alpha):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    _check(lib().mc_vegas_set_channels(v.handle, a.ctypes.data_as(_dp)))


def mc_vegas_get_channels(v):
    """(alpha[3], W[3]) of the three-channel process."""
    a, w = np.zeros(3), np.zeros(3)
    _check(lib().mc_vegas_get_channels(v.handle, a.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
    return a, w


def mc_channel_update(alpha, w, beta=0.5, amin=0.02):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(len(a))
    _check(lib().mc_channel_update(len(a), a.ctypes.data_as(_dp), ww.ctypes.data_as(_dp), beta, amin,
                                   out.ctypes.data_as(_dp)))
    return out


def mc_vegas_refine(v, alpha=1.5, stream=None):
    _check(lib().mc_vegas_refine(v.handle, alpha, _stream(stream)))


def mc_integrate(itg, pdf, niter, nevents, nbins=50, seed=0, gid=0, prec=MC_FP64, alpha=1.5, target_rel_err=0.0,
                 stream=None):
    c = _integrand(itg)
    out = Result()
    per = (IterResult * niter)()
    _check(lib().mc_integrate(ctypes.byref(c), pdf.handle if pdf else None, niter, nevents, nbins, seed, gid, prec,
                              alpha, target_rel_err, _stream(stream), ctypes.byref(out), per))
    return out, [per[i] for i in range(out.n_iter)]


def mc_debug_events(v, itg, pdf, first, k, out_dev, stream=None):
    c = _integrand(itg)
    _check(lib().mc_debug_events(v.handle, ctypes.byref(c), pdf.handle if pdf else None, first, k, _ptr(out_dev),
                                 _stream(stream)))


def mc_vegas_kernel_ms(v):
    ms = ctypes.c_float()
    _check(lib().mc_vegas_kernel_ms(v.handle, ctypes.byref(ms)))
    return ms.value


class Batch:
    """Owns an mc_batch handle (many integrands, one persistent launch per iteration)."""

    def __init__(self, handle, ndims, nbins):
        self.handle, self.ndims, self.nbins = handle, ndims, nbins

    def free(self):
        if self.handle:
            _check(lib().mc_batch_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_batch_create(itgs, nevents, pdf, nbins=50, seed=0, prec=MC_FP32_KAHAN):
    n = len(itgs)
    arr = (Integrand * n)(*[_integrand(t) for t in itgs])
    ev = (ctypes.c_int64 * n)(*[int(x) for x in nevents])
    h = _vp()
    _check(lib().mc_batch_create(n, arr, ev, pdf.handle if pdf else None, nbins, seed, prec, ctypes.byref(h)))
    return Batch(h, [t.ndim() for t in itgs], nbins)


def mc_batch_iterate(b, alpha=1.5, stream=None):
    out = (IterResult * len(b.ndims))()
    _check(lib().mc_batch_iterate(b.handle, alpha, _stream(stream), out))
    return [out[i] for i in range(len(b.ndims))]


def mc_batch_get_grid(b, i):
    e = np.zeros((b.ndims[i], b.nbins + 1))
    _check(lib().mc_batch_get_grid(b.handle, i, e.ctypes.data_as(_dp)))
    return e


def mc_batch_shape(b):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().mc_batch_shape(b.handle, *[ctypes.byref(x) for x in v]))
    return dict(block=v[0].value, events_per_thread=v[1].value, grid=v[2].value, ntiles=v[3].value)


def mc_batch_kernel_ms(b):
    ms = ctypes.c_float()
    _check(lib().mc_batch_kernel_ms(b.handle, ctypes.byref(ms)))
    return ms.value


def mc_batch_free(b):
    b.free()


EPI_BIAS_RELU_BF16, EPI_BIAS_F32, EPI_RELU_MASK_BF16, EPI_ATOMIC_F32, EPI_PARTIAL_F32 = 0, 1, 2, 3, 4


def mc_gemm_bf16(M, N, K, bn, epilogue, a, b, c, bias=None, mask=None, splits=1, err=None, stream=None):
    """C[M x N] (+)= A[M x K] . B[N x K]^T on the tcgen05 tensor cores (torch tensors on the device)."""
    null = ctypes.c_void_p(0)
    _check(lib().mc_gemm_bf16(M, N, K, bn, epilogue, _ptr(a), a.stride(0), _ptr(b), b.stride(0),
                              _ptr(bias) if bias is not None else null, _ptr(c), c.stride(-2),
                              _ptr(mask) if mask is not None else null, mask.stride(0) if mask is not None else 0,
                              splits, _ptr(err), _stream(stream)))


def mc_gemm_bf16_tn(M, N, K, bn, epilogue, x, y, c, splits=1, err=None, stream=None):
    """C[M x N] (+)= X^T Y, X [K x M], Y [K x N] row-major BF16 (torch tensors on the device)."""
    _check(lib().mc_gemm_bf16_tn(M, N, K, bn, epilogue, _ptr(x), x.stride(0), _ptr(y), y.stride(0), _ptr(c),
                                 c.stride(-2), splits, _ptr(err), _stream(stream)))


def mc_gemm_bf16_xn(M, N, K, bn, epilogue, x, b, c, splits=1, err=None, stream=None):
    """C[M x N] (+)= X^T B^T, X [K x M], B [N x K] row-major BF16 (torch tensors on the device)."""
    _check(lib().mc_gemm_bf16_xn(M, N, K, bn, epilogue, _ptr(x), x.stride(0), _ptr(b), b.stride(0), _ptr(c),
                                 c.stride(-2), splits, _ptr(err), _stream(stream)))


def mc_gemm_bf16_rs(M, N, K, bn, epilogue, a, b, c=None, c_t=None, bias=None, mask=None, err=None, stream=None):
    """Persistent B-resident variant; c row-major and/or c_t transposed (torch tensors on the device)."""
    null = ctypes.c_void_p(0)
    _check(lib().mc_gemm_bf16_rs(M, N, K, bn, epilogue, _ptr(a), a.stride(0), _ptr(b), b.stride(0),
                                 _ptr(bias) if bias is not None else null, _ptr(c) if c is not None else null,
                                 c.stride(0) if c is not None else 0, _ptr(c_t) if c_t is not None else null,
                                 c_t.stride(0) if c_t is not None else 0, _ptr(mask) if mask is not None else null,
                                 mask.stride(0) if mask is not None else 0, _ptr(err), _stream(stream)))


MC_NOALLOC_MAX_BLOCKS = 4096


def mc_vegas_iterate_noalloc(itg, pdf, ndim, nbins, edges64_dev, edges32_dev, prec, seed, iteration, gid, nevents,
                             blocks, hist_w2_dev, hist_n_dev, sums_dev, stream=None):
    """Allocation-free iteration: every buffer is the caller's (device
    pointers); sums_dev receives mc_device_sums (8 x 8 bytes: sum_hi, sum_lo,
    sum2_hi, sum2_lo, wmax as FP64, then n_nonzero, n_bad, n_noconv as int64)."""
    c = _integrand(itg)
    e32 = _ptr(edges32_dev) if edges32_dev is not None else None
    _check(lib().mc_vegas_iterate_noalloc(ctypes.byref(c), pdf.handle if pdf else None, ndim, nbins,
                                          _ptr(edges64_dev), e32, prec, seed, iteration, gid, nevents, blocks,
                                          _ptr(hist_w2_dev), _ptr(hist_n_dev), _ptr(sums_dev), _stream(stream)))


def mc_fma_peak(kind, iters, out_dev, stream=None):
    """Launch the FMA-throughput kernel (kind 0 f32, 1 f32x2, 2 f64) on
    `stream`; returns the launch's FLOP.  out_dev: device float32, one per
    thread of the grid (SMs x 2048)."""
    flop = ctypes.c_double()
    _check(lib().mc_fma_peak(kind, iters, _ptr(out_dev), out_dev.numel(), ctypes.byref(flop), _stream(stream)))
    return flop.value


def mc_launch_shape(itg, prec, nevents):
    b, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().mc_launch_shape(ctypes.byref(_integrand(itg)), prec, nevents, ctypes.byref(b), ctypes.byref(t)))
    return b.value, t.value


FLOW_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def pack_flow_params(layers):
    """Packed FP32 parameter vector (the mc_flow layout) from per-layer dicts of arrays."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).ravel() for p in layers for k in FLOW_KEYS])


def unpack_flow_params(flat, ndim, nlayers, bins, hidden=256):
    """Per-layer dicts of arrays from a packed parameter vector."""
    out, o = [], 0
    for l in range(nlayers):
        nb = (ndim + 1 - (l % 2)) // 2
        na, nout = ndim - nb, nb * (2 * bins + 1)
        shapes = dict(W1=(hidden, na), b1=(hidden,), W2=(hidden, hidden), b2=(hidden,), W3=(hidden, hidden),
                      b3=(hidden,), W4=(nout, hidden), b4=(nout,))
        d = {}
        for k in FLOW_KEYS:
            n = int(np.prod(shapes[k]))
            d[k] = np.asarray(flat[o:o + n]).reshape(shapes[k])
            o += n
        out.append(d)
    assert o == len(flat)
    return out


class Flow:
    """Owns an mc_flow handle (normalizing-flow sampler on the device)."""

    def __init__(self, handle, cfg, nparam, max_batch):
        self.handle, self.cfg, self.nparam, self.max_batch = handle, cfg, nparam, max_batch

    def free(self):
        if self.handle:
            _check(lib().mc_flow_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mc_flow_param_count(ndim, layers, bins, hidden=256):
    n = ctypes.c_int64()
    _check(lib().mc_flow_param_count(ctypes.byref(FlowCfg(ndim, layers, bins, hidden)), ctypes.byref(n)))
    return n.value


def mc_flow_create(ndim, layers, bins, init_layers, max_batch, seed=0, hidden=256):
    cfg = FlowCfg(ndim, layers, bins, hidden)
    flat = np.ascontiguousarray(pack_flow_params(init_layers), dtype=np.float32)
    n = mc_flow_param_count(ndim, layers, bins, hidden)
    if flat.size != n:
        raise McError(MC_EINVAL, f"flow needs {n} parameters, got {flat.size}")
    h = _vp()
    _check(lib().mc_flow_create(ctypes.byref(cfg), flat.ctypes.data_as(_fp), max_batch, seed, ctypes.byref(h)))
    return Flow(h, cfg, n, max_batch)


def mc_flow_free(f):
    f.free()


def mc_flow_set_params(f, layers):
    flat = np.ascontiguousarray(pack_flow_params(layers), dtype=np.float32)
    _check(lib().mc_flow_set_params(f.handle, flat.ctypes.data_as(_fp)))


def mc_flow_get_params(f):
    flat = np.zeros(f.nparam, dtype=np.float32)
    _check(lib().mc_flow_get_params(f.handle, flat.ctypes.data_as(_fp)))
    return unpack_flow_params(flat, f.cfg.ndim, f.cfg.layers, f.cfg.bins, f.cfg.hidden)


def mc_flow_set_fused(f, enable):
    """enable: bool (both directions) or a mask (bit 0 forward, bit 1 backward)."""
    mask = (3 if enable else 0) if isinstance(enable, bool) else int(enable)
    _check(lib().mc_flow_set_fused(f.handle, mask))


def mc_flow_forward(f, z_dev, x_dev, logq_dev, stream=None):
    """z [n x ndim] -> x, log q (float32 device tensors)."""
    _check(lib().mc_flow_forward(f.handle, z_dev.shape[0], _ptr(z_dev), _ptr(x_dev), _ptr(logq_dev),
                                 _stream(stream)))


def mc_flow_loss_grad(f, x_dev, w_dev, grads=True, stream=None):
    """Loss at fixed points and weights; returns (loss, per-layer gradient dicts or None)."""
    loss = ctypes.c_double()
    g = np.zeros(f.nparam, dtype=np.float32) if grads else None
    _check(lib().mc_flow_loss_grad(f.handle, x_dev.shape[0], _ptr(x_dev), _ptr(w_dev), ctypes.byref(loss),
                                   g.ctypes.data_as(_fp) if grads else None, _stream(stream)))
    return loss.value, (unpack_flow_params(g, f.cfg.ndim, f.cfg.layers, f.cfg.bins, f.cfg.hidden) if grads else None)


def mc_flow_adam_step(f, lr=1e-3, stream=None):
    _check(lib().mc_flow_adam_step(f.handle, lr, _stream(stream)))


def mc_flow_train(f, itg, pdf, steps, batch, lr=1e-3, stream=None, losses=True):
    out = (ctypes.c_double * max(steps, 1))() if losses else None
    _check(lib().mc_flow_train(f.handle, ctypes.byref(_integrand(itg)), pdf.handle if pdf else None, steps, batch, lr,
                               _stream(stream), out))
    return list(out)[:steps] if losses else None


def mc_flow_grad_count(f):
    n = ctypes.c_int64()
    _check(lib().mc_flow_grad_count(f.handle, ctypes.byref(n)))
    return n.value


def mc_flow_step_sample(f, itg, pdf, first, count, stream=None):
    """This rank's share of a training step's batch; returns its sum of w."""
    w = ctypes.c_double()
    _check(lib().mc_flow_step_sample(f.handle, ctypes.byref(_integrand(itg)), pdf.handle if pdf else None, first,
                                     count, _stream(stream), ctypes.byref(w)))
    return w.value


def mc_flow_step_grads(f, wsum_total, grads_dev=None, stream=None):
    """Gradient of this share with the loss normalised by wsum_total, into
    grads_dev (device float32 [mc_flow_grad_count]) or kept in place."""
    _check(lib().mc_flow_step_grads(f.handle, wsum_total, _ptr(grads_dev) if grads_dev is not None else None,
                                    _stream(stream)))


def mc_flow_step_apply(f, grads_dev=None, lr=1e-3, stream=None):
    _check(lib().mc_flow_step_apply(f.handle, _ptr(grads_dev) if grads_dev is not None else None, lr,
                                    _stream(stream)))


def mc_flow_iterate(f, itg, pdf, nevents, iteration=0, stream=None):
    r = IterResult()
    _check(lib().mc_flow_iterate(f.handle, ctypes.byref(_integrand(itg)), pdf.handle if pdf else None, nevents,
                                 iteration, _stream(stream), ctypes.byref(r)))
    return r


def mc_integrate_flow(itg, pdf, ndim, layers, bins, init_layers, train_steps, train_batch, lr=1e-3, niter=15,
                      nevents=10_000_000, nbins=50, seed=0, target_rel_err=0.0, stream=None, hidden=256):
    """Flow importance sampling with plain VEGAS as judge and fallback; returns (Result, used_flow)."""
    cfg = FlowCfg(ndim, layers, bins, hidden)
    flat = np.ascontiguousarray(pack_flow_params(init_layers), dtype=np.float32)
    out = Result()
    used = ctypes.c_int()
    _check(lib().mc_integrate_flow(ctypes.byref(_integrand(itg)), pdf.handle if pdf else None, ctypes.byref(cfg),
                                   flat.ctypes.data_as(_fp), train_steps, train_batch, lr, niter, nevents, nbins, seed,
                                   target_rel_err, _stream(stream), ctypes.byref(out), ctypes.byref(used)))
    return out, bool(used.value)


__all__ = ["McError", "Integrand", "IterResult", "Result", "GenStats", "Lhe", "EVENT_DTYPE", "Pdf", "Vegas", "Flow",
           "FlowCfg", "workloads", "events_from_bytes",
           "pack_flow_params", "unpack_flow_params", *SYMBOLS]
