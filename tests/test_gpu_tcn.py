"""Lambda network kernels against the FP64 oracle: the tensor-core 64 -> 64 layer alone (both
modes), the whole forward, the backward, Adam, the MSE gradient, and a short training run
through the smoother."""
import numpy as np
import pytest
import torch

from oracle import tcn as otcn
from paper_2604_00048_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


def _bf16_np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _theta_full(ws, seed):
    """He-normal weights in every layer (so o spans several units) and nonzero biases."""
    th = ws.tcn_init(seed, device="cpu")
    g = torch.Generator().manual_seed(seed + 100)
    off, (n, shape) = ws.TCN_OFFSETS["W4"][0], (576, (1, 64, 9))
    th[off:off + n] = torch.randn(n, generator=g) * (2.0 / 576) ** 0.5
    for b in ("b1", "b2", "b3", "b4"):
        o, shp = ws.TCN_OFFSETS[b]
        th[o:o + shp[0]] = torch.randn(shp[0], generator=g) * 0.05
    return th.cuda()


def _stream_input(n, T, seed):
    g = torch.Generator().manual_seed(seed)
    rows = n * (T + 4)
    a = torch.randn(rows, 64, generator=g).clamp_min(0)  # ReLU-like activations
    gap = (torch.arange(rows) % (T + 4)) >= T
    a[gap] = 0
    return a.to(torch.bfloat16).cuda(), gap.numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_conv64_layer(ws, mode):
    """7 series x 150 days = 1078 rows: three 384-row tiles, the last one ragged."""
    n, T = 7, 150
    th = _theta_full(ws, 1)
    packed = ws.tcn_pack(th)
    W = th[ws.TCN_OFFSETS["W2"][0]:ws.TCN_OFFSETS["W2"][0] + 36864].reshape(64, 64, 9).cpu().double().numpy()
    Wb = otcn.bf16_round(W)
    bias = th[ws.TCN_OFFSETS["b2"][0]:ws.TCN_OFFSETS["b2"][0] + 64].contiguous()
    inp, gap = _stream_input(n, T, 2)
    x = _bf16_np(inp)
    rows = x.shape[0]
    xp = np.zeros((rows + 8, 64))
    xp[4:4 + rows] = x
    if mode == 0:
        wpl = packed[1152:1152 + 36864]
        out, err = ws.tcn_conv64(inp, wpl, T, 0, bias=bias)
        ref = np.zeros((rows, 64))
        for k in range(9):
            ref += xp[k:k + rows] @ Wb[:, :, k].T
        ref = np.maximum(ref + bias.cpu().double().numpy(), 0)
        ref[gap] = 0
    else:
        wpl = packed[1152 + 36864:1152 + 2 * 36864]
        mask, _ = _stream_input(n, T, 3)
        out, err = ws.tcn_conv64(inp, wpl, T, 1, mask=mask)
        ref = np.zeros((rows, 64))
        for k in range(9):  # data gradient: sum_co W[co][ci][k] dh[r - k + 4][co]
            ref += xp[8 - k:8 - k + rows] @ Wb[:, :, k]
        ref = np.where(_bf16_np(mask) > 0, ref, 0)
    torch.cuda.synchronize()
    assert int(err.abs().sum()) == 0
    got = _bf16_np(out)
    scale = np.max(np.abs(ref))
    # FP32 accumulation of BF16 products, then one BF16 rounding of the result
    assert np.max(np.abs(got - ref) - 2.0 ** -8 * np.abs(ref)) <= 1e-4 * scale


def _tcn_inputs(T, P, seed):
    rc = synth.Recipe(**{**synth.RECIPES["learned"].__dict__, "T": T, "seed": synth.RECIPES["learned"].seed + seed})
    out = synth.generate_tile(rc, P, device="cuda", want_clean=True)
    return out["x"][:, 0, :].contiguous(), out["w"], out["clean"][:, 0, :].contiguous()


def test_forward_matches_oracle(ws):
    T, P = 130, 12
    x, w, _ = _tcn_inputs(T, P, 1)
    th = _theta_full(ws, 3)
    net = ws.Tcn(th)
    lam, ll = net.forward(x, w)
    torch.cuda.synchronize()
    lmin, lmax = ws.TCN_LOG_LAM
    o_ref, ll_ref = otcn.forward(th.cpu().double().numpy(), x.cpu().double().numpy(), w.cpu().double().numpy(),
                                 lmin, lmax, emulate_bf16=True)
    assert np.std(o_ref) > 0.1  # o spans a useful part of the sigmoid
    got = ll.cpu().double().numpy()
    assert np.max(np.abs(got - ll_ref)) <= 2e-3 * (lmax - lmin)
    assert torch.allclose(lam, torch.exp(ll), rtol=1e-6)


def test_backward_matches_oracle(ws):
    T, P = 90, 10
    x, w, _ = _tcn_inputs(T, P, 2)
    th = _theta_full(ws, 4)
    net = ws.Tcn(th)
    net.forward(x, w, training=True)
    g = torch.randn(T, P, generator=torch.Generator().manual_seed(5)).cuda()
    net.backward(g)
    torch.cuda.synchronize()
    lmin, lmax = ws.TCN_LOG_LAM
    ref = otcn.vjp(th.cpu().double().numpy(), x.cpu().double().numpy(), w.cpu().double().numpy(),
                   g.cpu().double().numpy(), lmin, lmax, emulate_bf16=True)
    got = net.grad.cpu().double().numpy()
    for name, (off, shape) in ws.TCN_OFFSETS.items():
        n = int(np.prod(shape))
        r, q = ref[off:off + n], got[off:off + n]
        # the data gradients between layers are stored in BF16 (2^-8 relative each)
        assert np.max(np.abs(q - r)) <= 3e-2 * np.max(np.abs(r)), name


def test_adam_matches_oracle(ws):
    n = ws.TCN_PARAMS
    g = torch.Generator().manual_seed(9)
    p0, gr = torch.randn(n, generator=g), torch.randn(n, generator=g)
    m0, v0 = torch.randn(n, generator=g) * 0.1, torch.rand(n, generator=g) * 0.1
    p, m, v, gd = (t.clone().cuda() for t in (p0, m0, v0, gr))
    import ctypes
    ws._check(ws._lib.ws_adam_step(ws._ptr(p), ws._ptr(m), ws._ptr(v), ws._ptr(gd), n, 3, 1e-3, 0.9, 0.999, 1e-8,
                                   None))
    pr, mr, vr = otcn.adam_step(p0.double().numpy(), m0.double().numpy(), v0.double().numpy(), gr.double().numpy(),
                                3, 1e-3, 0.9, 0.999, 1e-8)
    assert np.allclose(p.cpu().double().numpy(), pr, rtol=1e-5, atol=1e-7)
    # FP32 rounding of 0.9 m + 0.1 g: about 6e-8 times the magnitude of the terms (|g| <= ~5)
    assert np.allclose(m.cpu().double().numpy(), mr, rtol=1e-5, atol=5e-7)
    assert torch.all(gd == 0)


def test_mse_grad(ws):
    g = torch.Generator().manual_seed(1)
    z, t = torch.randn(10007, generator=g).cuda(), torch.randn(10007, generator=g).cuda()
    loss = torch.zeros(1, device="cuda")
    gz = ws.mse_grad(z, t, 2.0 / z.numel(), loss)
    d = (z - t).double()
    assert torch.allclose(gz.double(), 2 * d / z.numel(), rtol=1e-6)
    assert abs(loss.item() - float((d * d).mean())) <= 1e-5 * float((d * d).mean())


def test_training_reduces_loss(ws):
    """Twenty Adam steps through the smoother (z = Omega(lambda)^{-1} W x, loss = mean
    (z - clean)^2, gradient by the adjoint) on one batch of 256 two-year series."""
    T, P = 730, 256
    x, w, clean = _tcn_inputs(T, P, 3)
    net = ws.Tcn(ws.tcn_init(11))
    losses = []
    for it in range(20):
        lam, _ = net.forward(x, w, training=True)
        z, st = ws.smooth(x[:, None, :], w, lam, 2)
        loss = torch.zeros(1, device="cuda")
        gz = ws.mse_grad(z[:, 0, :].contiguous(), clean, 2.0 / clean.numel(), loss)
        _, glam, _ = ws.smooth_adjoint(w, lam, z, gz[:, None, :].contiguous(), 2, want_gx=False, log_lambda=True)
        net.backward(glam)
        net.step(3e-3)
        losses.append(loss.item())
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.9 * losses[0], losses


def test_checkpoint_round_trip(ws, tmp_path):
    """Weights, Adam moments and the step count survive save/load exactly; continuing from
    the loaded copy matches continuing from the original up to the order of the weight-
    gradient kernels' floating-point atomic sums (not bit-identical from run to run)."""
    from paper_2604_00048_b300 import train

    T, P = 120, 64
    x, w, clean = _tcn_inputs(T, P, 4)
    net = ws.Tcn(ws.tcn_init(21))
    for _ in range(2):
        train.train_step(net, x[:, None, :].contiguous(), w, clean, 1e-3)
    path = str(tmp_path / "net.ckpt")
    train.save_checkpoint(path, net, 2)
    net2, drawn = train.load_checkpoint(path)
    assert drawn == 2 and net2.step_count == net.step_count
    assert torch.equal(net2.theta, net.theta) and torch.equal(net2.m, net.m) and torch.equal(net2.v, net.v)
    before = net.theta.clone()
    train.train_step(net, x[:, None, :].contiguous(), w, clean, 1e-3)
    train.train_step(net2, x[:, None, :].contiguous(), w, clean, 1e-3)
    torch.cuda.synchronize()
    step = (net.theta - before).abs().max().item()
    assert step > 0
    assert (net.theta - net2.theta).abs().max().item() <= 1e-3 * step


def test_learned_lambda_beats_gcv_after_training(ws):
    """What the network gains over the method without it: after half an epoch of training
    (256 Adam steps on batches of 4096 two-year series with known clean signal, through the
    smoother's adjoint), smoothing at the network's per-day lambda is closer to the clean
    signal than smoothing at the per-series GCV choice (16-value grid), on 32,768 new series
    of the same generator (both final smooths with their refinement step)."""
    from paper_2604_00048_b300 import train

    net, batches, hist = train.train(2097152, 4096, 0.5, 2e-3, seed=0, log_every=10 ** 9)
    assert batches == 256 and np.isfinite(hist[-1][1])
    rmse_learned, rmse_gcv = train.evaluate(net, n=32768, chunk=32768)
    assert rmse_learned < rmse_gcv, (rmse_learned, rmse_gcv)
