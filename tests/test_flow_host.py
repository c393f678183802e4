"""Host-side pieces of the flow sampler's C ABI that need no GPU: the
parameter count against the shapes of the initial parameters, the packed
layout round trip, and argument validation before any device work."""
import numpy as np
import pytest

from paper_2302_03343_b300 import mcint as M
from paper_2302_03343_b300 import workloads as W


@pytest.mark.parametrize("D,L,K", [(7, 6, 32), (4, 2, 8), (14, 6, 32), (2, 1, 2), (16, 16, 32)])
def test_param_count_matches_initial_parameters(D, L, K):
    arrays = W.flow_init_params(D, L=L, K=K, hidden=256, seed=0)
    n = sum(v.size for layer in arrays for v in layer.values())
    assert M.mc_flow_param_count(D, L, K) == n


def test_pack_unpack_round_trip():
    arrays = W.flow_init_params(7, L=6, K=32, seed=3, last_scale=1.0)
    flat = M.pack_flow_params(arrays)
    back = M.unpack_flow_params(flat, 7, 6, 32)
    for a, b in zip(arrays, back):
        for k in M.FLOW_KEYS:
            assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("cfg", [(1, 6, 32), (17, 6, 32), (7, 0, 32), (7, 17, 32), (7, 6, 1), (7, 6, 33)])
def test_create_rejects_bad_configurations(cfg):
    D, L, K = cfg
    arrays = W.flow_init_params(max(D, 2), L=max(L, 1), K=max(min(K, 32), 2), hidden=256, seed=0)
    with pytest.raises(M.McError) as e:
        h = M._vp()
        flat = M.pack_flow_params(arrays)
        M._check(M.lib().mc_flow_create(M.ctypes.byref(M.FlowCfg(D, L, K, 256)),
                                        flat.ctypes.data_as(M._fp), 128, 0, M.ctypes.byref(h)))
    assert e.value.code == M.MC_EINVAL
