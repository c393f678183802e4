"""Host-side checks of the C ABI: the library loads, exports every function
declared in include/mcint.h, the ctypes structs match the declared layout, and
argument validation rejects bad input before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2302_03343_b300 import build as B
from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mcint.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return M.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(mc_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(M.SYMBOLS) == names


def test_struct_layouts():
    assert ctypes.sizeof(M.Integrand) == 8 + 12 * 8
    assert ctypes.sizeof(M.IterResult) == 8 * 6 + 8
    assert ctypes.sizeof(M.Result) == 3 * 8 + 8 + 8
    text = open(HEADER).read()
    for k, v in M.REC.items():
        assert re.search(rf"#define MC_REC_{k} {v}\b", text), k
    assert re.search(rf"#define MC_REC_STRIDE {M.REC_STRIDE}\b", text)


def test_validation_without_device_work(L):
    with pytest.raises(M.McError) as e:
        M.mc_vegas_init(0, 50, 0, M.MC_FP64)
    assert e.value.code == M.MC_EINVAL
    # MC_MAX_DIM (17) is the three-channel grid; one more is rejected
    for args in ((M.MC_MAX_DIM + 1, 50, 0, M.MC_FP64), (4, 1, 0, M.MC_FP64), (4, 257, 0, M.MC_FP64),
                 (4, 50, 0, 7)):
        with pytest.raises(M.McError) as e:
            M.mc_vegas_init(*args)
        assert e.value.code == M.MC_EINVAL, args
    g = W.synthetic_pdf_grid(0)
    bad = W.PdfGrid(x=g.x[::-1].copy(), q=g.q, pids=g.pids, xf=g.xf, params=g.params)
    with pytest.raises(M.McError) as e:
        M.mc_pdf_load(bad)
    assert "increasing" in str(e.value)
    xf = g.xf.copy()
    xf[3, 4, 5] = np.nan
    with pytest.raises(M.McError) as e:
        M.mc_pdf_load(W.PdfGrid(x=g.x, q=g.q, pids=g.pids, xf=xf, params=g.params))
    assert "non-finite" in str(e.value)


def test_gauss_dim_is_bounded_before_device_work(L):
    """The Gaussian kernels loop over at most 16 dimensions: gauss_dim 0 and 17
    are rejected as invalid input by every entry point that reads it, before
    any device call (so the answer is the same with or without a GPU)."""
    for d in (0, 17):
        with pytest.raises(M.McError) as e:
            M.mc_integrate(W.gauss(d), None, 2, 1000)
        assert e.value.code == M.MC_EINVAL, d
        with pytest.raises(M.McError) as e:
            M.mc_launch_shape(W.gauss(d), M.MC_FP64, 1000)
        assert e.value.code == M.MC_EINVAL, d
