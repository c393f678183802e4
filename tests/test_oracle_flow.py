"""Pins of the flow oracle (oracle/flow.py): invertibility, the log-Jacobian
against a finite-difference Jacobian determinant, normalisation of the
density, the identity at zero last-layer weights, gradients against central
finite differences, and one Adam step against the update equations."""
import math

import numpy as np
import pytest
import torch

from oracle import flow as F
from paper_2302_03343_b300 import workloads as W

K = 32
D = 7


def rand_params(seed=1, scale=0.5, L=6):
    arrays = W.flow_init_params(D, L=L, K=K, hidden=32, seed=seed, last_scale=scale)
    return F.params_from_arrays(arrays)


def test_masks_cover_every_dimension_three_times():
    counts = np.zeros(D, int)
    for a, b in W.flow_layer_masks(D, 6):
        assert sorted(a + b) == list(range(D)) and not set(a) & set(b)
        counts[b] += 1
    assert (counts == 3).all()


def test_identity_at_zero_last_layer():
    params = rand_params(scale=0.0)
    z = torch.rand(200, D, dtype=F.DT, generator=torch.Generator().manual_seed(0))
    x, logq = F.flow_forward(params, z, K)
    assert torch.allclose(x, z, atol=1e-14) and torch.allclose(logq, torch.zeros_like(logq), atol=1e-13)


def test_forward_inverse_round_trip():
    params = rand_params()
    z = torch.rand(500, D, dtype=F.DT, generator=torch.Generator().manual_seed(1))
    x, lq_f = F.flow_forward(params, z, K)
    assert (x > 0).all() and (x < 1).all()
    z2, lq_i = F.flow_inverse(params, x, K)
    assert torch.max(torch.abs(z2 - z)) < 1e-12
    assert torch.max(torch.abs(lq_f - lq_i)) < 1e-10


def test_log_jacobian_against_finite_differences():
    params = rand_params(seed=3)
    z = torch.rand(4, D, dtype=F.DT, generator=torch.Generator().manual_seed(2)) * 0.9 + 0.05
    _, logq = F.flow_forward(params, z, K)
    h = 1e-6
    for n in range(z.shape[0]):
        J = np.zeros((D, D))
        for j in range(D):
            zp, zm = z[n:n + 1].clone(), z[n:n + 1].clone()
            zp[0, j] += h
            zm[0, j] -= h
            J[:, j] = ((F.flow_forward(params, zp, K)[0] - F.flow_forward(params, zm, K)[0]) / (2 * h)).numpy()[0]
        assert abs(math.log(abs(np.linalg.det(J))) + logq[n].item()) < 1e-6


def test_density_integrates_to_one():
    params = rand_params(seed=4, scale=0.3)
    x = torch.rand(200000, D, dtype=F.DT, generator=torch.Generator().manual_seed(3))
    _, logq = F.flow_inverse(params, x, K)
    q = torch.exp(logq)
    assert abs(q.mean().item() - 1.0) < 4 * q.std().item() / math.sqrt(x.shape[0])


def test_gradients_against_finite_differences():
    params = rand_params(seed=5, L=2)
    g = torch.Generator().manual_seed(4)
    x = torch.rand(64, D, dtype=F.DT, generator=g)
    w = torch.rand(64, dtype=F.DT, generator=g)
    L0, grads = F.loss_and_grads(params, x, w, K)
    rng = np.random.default_rng(0)
    for layer in range(2):
        for name in ("W1", "W2", "W3", "W4", "b4"):
            t = params[layer][name]
            for _ in range(2):
                idx = tuple(int(rng.integers(s)) for s in t.shape)
                h = 1e-6
                old = t[idx].item()
                t[idx] = old + h
                lp = F.loss(params, x, w, K).item()
                t[idx] = old - h
                lm = F.loss(params, x, w, K).item()
                t[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[layer][name][idx].item()
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (layer, name, idx, fd, an)


def test_adam_first_steps_by_hand():
    p = [{"a": torch.tensor([1.0, -2.0], dtype=F.DT)}]
    g = [{"a": torch.tensor([0.5, -0.25], dtype=F.DT)}]
    st = F.adam_state(p)
    p1 = F.adam_step(p, g, st, 1, lr=1e-3)
    # m_hat = g, v_hat = g^2 after one step: update -lr g/(|g| + eps)
    exp1 = torch.tensor([1.0 - 1e-3 * 0.5 / (0.5 + 1e-8), -2.0 + 1e-3 * 0.25 / (0.25 + 1e-8)], dtype=F.DT)
    assert torch.allclose(p1[0]["a"], exp1, rtol=0, atol=1e-15)
    g2 = [{"a": torch.tensor([0.1, 0.3], dtype=F.DT)}]
    p2 = F.adam_step(p1, g2, st, 2, lr=1e-3)
    m = 0.9 * (0.1 * torch.tensor([0.5, -0.25], dtype=F.DT)) + 0.1 * torch.tensor([0.1, 0.3], dtype=F.DT)
    v = 0.999 * (0.001 * torch.tensor([0.25, 0.0625], dtype=F.DT)) + 0.001 * torch.tensor([0.01, 0.09], dtype=F.DT)
    mh, vh = m / (1 - 0.9 ** 2), v / (1 - 0.999 ** 2)
    assert torch.allclose(p2[0]["a"], p1[0]["a"] - 1e-3 * mh / (torch.sqrt(vh) + 1e-8), rtol=0, atol=1e-15)
