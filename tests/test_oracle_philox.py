"""Pins of the oracle's Philox4x32-10 and integer uniforms.

External pin: the Philox4_32_10 generator of the cuRAND host library, run on
the CPU, emits block j of four words as Philox4x32-10 of counter (0, 0, j, 0)
under key (seed low, seed high).
"""
import ctypes
import os

import numpy as np
import pytest

import oracle as O

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_host(seed, n):
    lib = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(n, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.skipif(not os.path.exists(CURAND), reason="cuRAND host library not present")
@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF])
def test_philox_matches_curand_host(seed):
    ref = _curand_host(seed, 4 * 64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(64):
        got = O.philox4x32_10([0, 0, j, 0], key)
        np.testing.assert_array_equal(got, ref[4 * j:4 * j + 4])


def test_uniform_int_layout_fp32_and_fp64():
    seed, it, gid = 0x1234, 3, 5
    k32 = O.uniform_ints(seed, it, gid, 1, 6, 10, 1)[0]
    k64 = O.uniform_ints(seed, it, gid, 0, 6, 10, 1)[0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w0 = O.philox4x32_10([10, 0, it, gid | (0 << 8)], key)
    w1 = O.philox4x32_10([10, 0, it, gid | (1 << 8)], key)
    w2 = O.philox4x32_10([10, 0, it, gid | (2 << 8)], key)
    assert list(k32[:4]) == [int(w) >> 9 for w in w0]
    assert list(k32[4:6]) == [int(w) >> 9 for w in w1[:2]]
    for d, (w, s) in enumerate([(w0, 0), (w0, 1), (w1, 0), (w1, 1), (w2, 0), (w2, 1)]):
        assert int(k64[d]) == ((int(w[2 * s]) << 32) | int(w[2 * s + 1])) >> 12


def test_uniform_moments():
    for prec, bits in ((0, 52), (1, 23)):
        k = O.uniform_ints(7, 0, 0, prec, 4, 0, 50000).astype(np.float64)
        u = (2 * k + 1) / 2.0 ** (bits + 1)
        assert np.all((u > 0) & (u < 1))
        assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
        assert abs(u.var() - 1 / 12) < 0.002
        c = np.corrcoef(u[:, 0], u[:, 1])[0, 1]
        assert abs(c) < 0.02
