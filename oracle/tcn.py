"""Oracle for the lambda network (test infrastructure; CPU, FP64).

The network of the learned-lambda path, written as plainly as possible with PyTorch's CPU
conv1d in float64: per series, input channels (x_t [w_t > 0], w_t), then
conv(2->64, kernel 9) -> ReLU -> conv(64->64) -> ReLU -> conv(64->64) -> ReLU -> conv(64->1) = o,
"same" zero padding (4 days each side), and log lambda = Lmin + sigmoid(o) (Lmax - Lmin)
(Section 4.2 gives the sigmoid output range; the architecture is the one the GPU path uses).

With emulate_bf16 the inputs, the weights and each layer's output activations are rounded
to BF16 (round to nearest even) where the GPU path stores them in BF16; arithmetic stays
FP64. Gradients come from torch.autograd in float64; the BF16 roundings are treated as the
identity in the backward pass (as the GPU path does: it differentiates the layers it ran).

Only the tests may import this module; it shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

# parameter vector: PyTorch conv1d layouts [out][in][k], concatenated in this order
LAYOUT = [("W1", (64, 2, 9)), ("b1", (64,)), ("W2", (64, 64, 9)), ("b2", (64,)),
          ("W3", (64, 64, 9)), ("b3", (64,)), ("W4", (1, 64, 9)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in LAYOUT)


def bf16_round(a):
    """Round float values to the nearest BF16 (ties to even), returned as float64.
    BF16 keeps the top 16 bits of the FP32 encoding; rounding adds half an ulp of that
    truncation plus the parity bit before truncating."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, off = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = theta[off:off + n].reshape(shape)
        off += n
    return out


def _round_st(a, on):
    """BF16 rounding in the forward pass, identity in the backward pass."""
    if not on:
        return a
    r = torch.from_numpy(bf16_round(a.detach().numpy()))
    return a + (r - a).detach()


def _forward_t(p, x, w, lmin, lmax, emulate_bf16):
    """Differentiable forward for one series (torch float64 tensors); returns (o, loglam)."""
    xin = torch.where(w > 0, x, torch.zeros_like(x))
    a = torch.stack([xin, w])[None]                              # [1, 2, T]
    a = _round_st(a, emulate_bf16)
    W = {k: (_round_st(v, emulate_bf16) if k.startswith("W") else v) for k, v in p.items()}
    for i in (1, 2, 3):
        a = torch.relu(F.conv1d(a, W[f"W{i}"], p[f"b{i}"], padding=4))
        a = _round_st(a, emulate_bf16)
    o = F.conv1d(a, W["W4"], p["b4"], padding=4)[0, 0]
    return o, lmin + torch.sigmoid(o) * (lmax - lmin)


def forward(theta, x, w, lmin, lmax, emulate_bf16=True):
    """x, w: [T] or [T, P] (tile layout). Returns (o, loglam) of the same shape."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    x2, w2 = x.reshape(x.shape[0], -1), w.reshape(w.shape[0], -1)
    p = {k: torch.from_numpy(v.copy()) for k, v in unpack(theta).items()}
    o = np.zeros_like(x2)
    ll = np.zeros_like(x2)
    with torch.no_grad():
        for s in range(x2.shape[1]):
            os_, ls = _forward_t(p, torch.from_numpy(x2[:, s].copy()), torch.from_numpy(w2[:, s].copy()),
                                 lmin, lmax, emulate_bf16)
            o[:, s], ll[:, s] = os_.numpy(), ls.numpy()
    return o.reshape(x.shape), ll.reshape(x.shape)


def vjp(theta, x, w, g_loglam, lmin, lmax, emulate_bf16=True):
    """dL/dtheta for L = sum g_loglam * loglam(theta), summed over the series."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g_loglam, dtype=np.float64)
    x2, w2, g2 = (a.reshape(a.shape[0], -1) for a in (x, w, g))
    th = torch.tensor(np.asarray(theta, dtype=np.float64), requires_grad=True)
    p, off = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        p[name] = th[off:off + n].reshape(shape)
        off += n
    total = 0.0
    for s in range(x2.shape[1]):
        _, ls = _forward_t(p, torch.from_numpy(x2[:, s].copy()), torch.from_numpy(w2[:, s].copy()),
                           lmin, lmax, emulate_bf16)
        total = total + torch.sum(torch.from_numpy(g2[:, s].copy()) * ls)
    total.backward()
    return th.grad.numpy().copy()


def adam_step(p, m, v, g, step, lr, b1, b2, eps):
    """One Adam update (Kingma and Ba, Algorithm 1) in FP64; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
