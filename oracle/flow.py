"""Oracle of the normalizing-flow importance sampler (FP64, PyTorch on the CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the plain reference the
CUDA flow kernels are checked against; shares no code with them.

The thesis uses importance sampling with an adaptive density (Sec. "Importance
sampling": E_N = (1/N) sum f(x_n)/p(x_n); the optimal p is |f| / int |f|) and
trains networks made of dense layers y = phi(W x + b) (Sec. "Deep learning")
with Adam (Sec. "Optimizers": m_t, v_t, bias-corrected m_hat, v_hat, update
theta -= eta m_hat / (sqrt(v_hat) + eps)).  It prints no flow; the sampler is
the piecewise-quadratic coupling flow of Mueller et al. ("Neural Importance
Sampling", 2019), with these readings of what the thesis leaves open:

* D dimensions, L coupling layers; layer l transforms the dimensions with
  d % 2 == l % 2 and conditions on the others.
* Conditioner: u = 2 x_A - 1 -> dense 256 -> ReLU -> dense 256 -> ReLU ->
  dense 256 -> ReLU -> dense d_B (2K + 1); per transformed dimension K width
  logits and K + 1 height logits.
* Spline: widths W = softmax(width logits); heights V = exp(height logits)
  normalised so that sum_k (V_k + V_{k+1}) / 2 W_k = 1; the density in bin b is
  linear between V_b and V_{b+1}, the CDF quadratic; the forward map is the
  CDF, the inverse solves the quadratic in the stable root form.
* Base density uniform on the unit cube; log q(x) = -sum over layers and
  transformed dimensions of log c, c the spline density at the layer input.
* Loss (forward KL with importance weights, x sampled from the flow and held
  fixed): L = -sum_i w_i log q(x_i) / sum_i w_i, w_i = |f(x_i)| / q(x_i).

`bf16=True` rounds to BF16 (round to nearest even) every operand the CUDA
path feeds its tensor cores: the conditioner input u, the weights W1..W4, the
first layer's bias b1 (a weight on a constant input of one there), and the
hidden activations after each ReLU.  b2..b4 are added in FP32 and every
product accumulates in FP32, so the GPU can be compared with the same
roundings.
"""
import math

import torch

DT = torch.float64


def layer_masks(D, L):
    """(conditioning indices, transformed indices) per layer."""
    out = []
    for l in range(L):
        b = [d for d in range(D) if d % 2 == l % 2]
        a = [d for d in range(D) if d % 2 != l % 2]
        out.append((a, b))
    return out


def _r16(t):
    return t.to(torch.bfloat16).to(DT)


def _r32(t):
    return t.to(torch.float32).to(DT)


def spline_params(logits, K):
    """Widths [.., K] and normalised vertex heights [.., K+1]."""
    W = torch.softmax(logits[..., :K], dim=-1)
    Vt = torch.exp(logits[..., K:])
    area = ((Vt[..., :-1] + Vt[..., 1:]) / 2 * W).sum(-1, keepdim=True)
    return W, Vt / area


def _edges(W, V):
    zero = torch.zeros_like(W[..., :1])
    X = torch.cat([zero, torch.cumsum(W, -1)[..., :-1]], -1)
    seg = (V[..., :-1] + V[..., 1:]) / 2 * W
    C = torch.cat([zero, torch.cumsum(seg, -1)[..., :-1]], -1)
    return X, C


def _pick(t, b):
    return torch.gather(t, -1, b.unsqueeze(-1)).squeeze(-1)


def spline_forward(x, logits, K):
    """y = C(x) and log c(x) per transformed coordinate."""
    W, V = spline_params(logits, K)
    X, C = _edges(W, V)
    b = ((x.unsqueeze(-1) >= X).sum(-1) - 1).clamp(0, K - 1)
    Wb, Xb, Cb, Vb, Vb1 = _pick(W, b), _pick(X, b), _pick(C, b), _pick(V, b), _pick(V, b + 1)
    d = x - Xb
    y = Cb + d * Vb + d * d / (2 * Wb) * (Vb1 - Vb)
    c = Vb + d / Wb * (Vb1 - Vb)
    return y, torch.log(c)


def spline_inverse(y, logits, K):
    """x = C^-1(y) and log c(x)."""
    W, V = spline_params(logits, K)
    X, C = _edges(W, V)
    b = ((y.unsqueeze(-1) >= C).sum(-1) - 1).clamp(0, K - 1)
    Wb, Xb, Cb, Vb, Vb1 = _pick(W, b), _pick(X, b), _pick(C, b), _pick(V, b), _pick(V, b + 1)
    r = (y - Cb) / Wb
    dv = Vb1 - Vb
    alpha = 2 * r / (Vb + torch.sqrt(Vb * Vb + 2 * dv * r))
    x = Xb + alpha * Wb
    c = Vb + alpha * dv
    return x, torch.log(c)


def conditioner(p, xa, K, nb, bf16=False):
    """Logits [B, nb, 2K+1] of one layer from its conditioning coordinates."""
    u = 2 * xa - 1
    if bf16:
        # every dense layer on BF16 operands (the first layer's bias enters
        # as a BF16 weight on a constant input 1), FP32 accumulation
        u = _r16(_r32(u))
        h = _r16(torch.relu(u @ _r16(p["W1"]).T + _r16(p["b1"])))
        h = _r16(torch.relu(h @ _r16(p["W2"]).T + _r32(p["b2"])))
        h = _r16(torch.relu(h @ _r16(p["W3"]).T + _r32(p["b3"])))
        out = h @ _r16(p["W4"]).T + _r32(p["b4"])
    else:
        h = torch.relu(u @ p["W1"].T + p["b1"])
        h = torch.relu(h @ p["W2"].T + p["b2"])
        h = torch.relu(h @ p["W3"].T + p["b3"])
        out = h @ p["W4"].T + p["b4"]
    return out.reshape(xa.shape[0], nb, 2 * K + 1)


def flow_forward(params, z, K, bf16=False):
    """Sampling direction: z (uniform) -> x, and log q(x)."""
    D = z.shape[1]
    masks = layer_masks(D, len(params))
    x = z.clone()
    logdet = torch.zeros(z.shape[0], dtype=DT)
    for p, (a, b) in zip(params, masks):
        logits = conditioner(p, x[:, a], K, len(b), bf16)
        y, lc = spline_forward(x[:, b], logits, K)
        x = x.clone()
        x[:, b] = y
        logdet = logdet + lc.sum(-1)
    return x, -logdet


def flow_inverse(params, x, K, bf16=False):
    """Density direction: x -> z, and log q(x)."""
    D = x.shape[1]
    masks = layer_masks(D, len(params))
    z = x.clone()
    logq = torch.zeros(x.shape[0], dtype=DT)
    for p, (a, b) in reversed(list(zip(params, masks))):
        logits = conditioner(p, z[:, a], K, len(b), bf16)
        xb, lc = spline_inverse(z[:, b], logits, K)
        z = z.clone()
        z[:, b] = xb
        logq = logq - lc.sum(-1)
    return z, logq


def loss(params, x, w, K, bf16=False):
    """-sum w log q(x) / sum w with x and w held fixed."""
    _, logq = flow_inverse(params, x, K, bf16)
    return -(w * logq).sum() / w.sum()


def loss_and_grads(params, x, w, K, bf16=False):
    ps = [{k: v.detach().clone().requires_grad_(True) for k, v in p.items()} for p in params]
    L = loss(ps, x, w, K, bf16)
    L.backward()
    return L.item(), [{k: v.grad.detach().clone() for k, v in p.items()} for p in ps]


def adam_step(params, grads, state, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (thesis Sec. "Optimizers"); state holds m and v per tensor."""
    out = []
    for p, g, st in zip(params, grads, state):
        q = {}
        for k in p:
            m = b1 * st["m"][k] + (1 - b1) * g[k]
            v = b2 * st["v"][k] + (1 - b2) * g[k] * g[k]
            st["m"][k], st["v"][k] = m, v
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            q[k] = p[k] - lr * mh / (torch.sqrt(vh) + eps)
        out.append(q)
    return out


def adam_state(params):
    return [{"m": {k: torch.zeros_like(v) for k, v in p.items()},
             "v": {k: torch.zeros_like(v) for k, v in p.items()}} for p in params]


def params_from_arrays(arrays):
    """Tensors (FP64) from the per-layer numpy arrays of workloads.flow_init_params."""
    return [{k: torch.tensor(v, dtype=DT) for k, v in layer.items()} for layer in arrays]
