"""Pins for the lambda-network oracle (oracle/tcn.py): the convolution against brute force,
the gradient against central finite differences, the receptive field, the sigmoid range,
BF16 rounding against its definition, and Adam against a hand-computed step."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import tcn


def _theta(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    th = np.zeros(tcn.N_PARAMS)
    off = 0
    for name, shape in tcn.LAYOUT:
        n = int(np.prod(shape))
        fan = shape[1] * shape[2] if name.startswith("W") else 1
        th[off:off + n] = rng.normal(size=n) * (np.sqrt(2.0 / fan) if name.startswith("W") else 0.1) * scale
        off += n
    return th


def test_conv_same_brute_force():
    """conv1d with padding 4 is out[co][t] = b[co] + sum_{ci,k} W[co][ci][k] a[ci][t + k - 4],
    zero outside the series."""
    rng = np.random.default_rng(1)
    a = rng.normal(size=(2, 7))
    W = rng.normal(size=(3, 2, 9))
    b = rng.normal(size=3)
    ref = np.zeros((3, 7))
    for co in range(3):
        for t in range(7):
            s = b[co]
            for ci in range(2):
                for k in range(9):
                    if 0 <= t + k - 4 < 7:
                        s += W[co, ci, k] * a[ci, t + k - 4]
            ref[co, t] = s
    got = F.conv1d(torch.from_numpy(a)[None], torch.from_numpy(W), torch.from_numpy(b), padding=4)[0].numpy()
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_bf16_round_definition():
    """Values exactly representable stay; halfway cases go to the even neighbour; the result
    keeps 8 significant bits."""
    assert tcn.bf16_round(np.array([1.0, -2.5, 0.0]))[0] == 1.0
    one_ulp = 2.0 ** -7                       # BF16 spacing at 1
    half = 1.0 + one_ulp / 2                  # tie: to even (1.0)
    assert tcn.bf16_round(np.array([half]))[0] == 1.0
    tie_up = 1.0 + 3 * one_ulp / 2            # tie between 1+ulp (odd) and 1+2ulp (even)
    assert tcn.bf16_round(np.array([tie_up]))[0] == 1.0 + 2 * one_ulp
    x = np.random.default_rng(2).normal(size=1000)
    r = tcn.bf16_round(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8 * 1.0001


def test_sigmoid_range():
    th = _theta(3)
    T = 30
    x = np.random.default_rng(4).random(T)
    w = np.ones(T)
    o, ll = tcn.forward(th, x, w, -2.0, 5.0, emulate_bf16=False)
    assert np.all(ll > -2.0) and np.all(ll < 5.0)
    sig = 1 / (1 + np.exp(-o))
    assert np.allclose(ll, -2.0 + 7.0 * sig, atol=1e-12)


def test_receptive_field_is_16_days():
    """Four kernel-9 layers: changing day t0 moves log lambda only on days t0-16 .. t0+16."""
    th = _theta(5)
    T, t0 = 80, 40
    rng = np.random.default_rng(6)
    x = rng.random(T)
    w = np.ones(T)
    _, l1 = tcn.forward(th, x, w, -2.0, 5.0, emulate_bf16=False)
    x2 = x.copy()
    x2[t0] += 0.5
    _, l2 = tcn.forward(th, x2, w, -2.0, 5.0, emulate_bf16=False)
    changed = np.nonzero(np.abs(l2 - l1) > 0)[0]
    assert changed.min() >= t0 - 16 and changed.max() <= t0 + 16
    assert changed.size > 0


def test_vjp_central_differences():
    th = _theta(7, scale=0.7)
    T = 24
    rng = np.random.default_rng(8)
    x = rng.random(T)
    w = (rng.random(T) < 0.6).astype(float)
    g = rng.normal(size=T)
    grad = tcn.vjp(th, x, w, g, -2.0, 5.0, emulate_bf16=False)
    idx = rng.choice(tcn.N_PARAMS, 24, replace=False)
    idx = np.concatenate([idx, [tcn.N_PARAMS - 1, 1152, 1216 + 5, 75072 + 3]])  # biases and W4
    h = 1e-5
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fp = np.sum(g * tcn.forward(tp, x, w, -2.0, 5.0, emulate_bf16=False)[1])
        fm = np.sum(g * tcn.forward(tm, x, w, -2.0, 5.0, emulate_bf16=False)[1])
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_adam_first_step_is_signed_lr():
    """With zero moments, Adam's first bias-corrected step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = tcn.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01, 0.9, 0.999, 1e-8)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
