"""Lambda network kernels at sizes where every persistent CTA takes many tiles.

The kernels loop over tiles (tile = blockIdx.x, blockIdx.x + gridDim.x, ...) and prefetch the
next tile's input while the current one computes; the small-batch tests elsewhere never give a
CTA a second tile. Here:
  - forward (k_tcn_fused): 4096 series x 730 days = 3.0M stream rows = 8,541 tiles of 352
    final rows on at most 148 CTAs (57+ tiles each); log lambda compared element-wise with the
    FP64 oracle (Section 4.2's network with BF16 rounding emulated) on 128 sampled series,
    including the first and last series of the batch (first and last tile);
  - backward: 400 series x 730 days = 293,600 rows (about 765 conv tiles of 384 rows, 834
    fused tiles, several per CTA); the whole weight gradient compared with the oracle's,
    which sums the per-series vector-Jacobian products;
  - the 64 -> 64 tensor-core layer alone (k_conv64, both modes) on 297 tiles.
Tolerances are those of the small-batch tests (BF16 storage of activations)."""
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


def _theta_full(ws, seed):
    """He-normal weights in every layer (o spans several units) and nonzero biases."""
    th = ws.tcn_init(seed, device="cpu")
    g = torch.Generator().manual_seed(seed + 100)
    off = ws.TCN_OFFSETS["W4"][0]
    th[off:off + 576] = torch.randn(576, generator=g) * (2.0 / 576) ** 0.5
    for b in ("b1", "b2", "b3", "b4"):
        o, shp = ws.TCN_OFFSETS[b]
        th[o:o + shp[0]] = torch.randn(shp[0], generator=g) * 0.05
    return th.cuda()


def _tcn_inputs(T, P, seed):
    rc = synth.Recipe(**{**synth.RECIPES["learned"].__dict__, "T": T, "seed": synth.RECIPES["learned"].seed + seed})
    out = synth.generate_tile(rc, P, device="cuda", want_clean=True)
    return out["x"][:, 0, :].contiguous(), out["w"]


def _sample(P, n, seed):
    idx = np.random.default_rng(seed).choice(np.arange(1, P - 1), size=n - 2, replace=False)
    return np.sort(np.concatenate([[0, P - 1], idx]))


@pytest.mark.parametrize("training", [False, True])
def test_forward_many_tiles_per_cta(ws, training):
    T, P = 730, 4096
    rows = P * (T + ws.TCN_GAP)
    n_tiles = -(-rows // 352)
    assert n_tiles > 50 * torch.cuda.get_device_properties(0).multi_processor_count
    x, w = _tcn_inputs(T, P, 11)
    th = _theta_full(ws, 13)
    net = ws.Tcn(th)
    lam, ll = net.forward(x, w, training=training)
    torch.cuda.synchronize()
    lmin, lmax = ws.TCN_LOG_LAM
    idx = _sample(P, 128, 3)
    _, ll_ref = otcn.forward(th.cpu().double().numpy(), x[:, idx].cpu().double().numpy(),
                             w[:, idx].cpu().double().numpy(), lmin, lmax, emulate_bf16=True)
    got = ll[:, idx].cpu().double().numpy()
    assert np.std(ll_ref) > 0.02 * (lmax - lmin)  # the outputs are far from constant
    assert np.max(np.abs(got - ll_ref)) <= 2e-3 * (lmax - lmin)
    assert torch.isfinite(ll).all()
    assert torch.allclose(lam, torch.exp(ll), rtol=1e-6)


def test_backward_many_tiles_per_cta(ws):
    T, P = 730, 400
    x, w = _tcn_inputs(T, P, 12)
    th = _theta_full(ws, 14)
    net = ws.Tcn(th)
    net.forward(x, w, training=True)
    g = torch.randn(T, P, generator=torch.Generator().manual_seed(15)).cuda()
    net.backward(g)
    torch.cuda.synchronize()
    lmin, lmax = ws.TCN_LOG_LAM
    thn, xn, wn, gn = (t.cpu().double().numpy() for t in (th, x, w, g))
    # the gradient of a sum over series is the sum of the per-series gradients
    ref = np.zeros_like(thn)
    for s0 in range(0, P, 100):
        ref += otcn.vjp(thn, xn[:, s0:s0 + 100], wn[:, s0:s0 + 100], gn[:, s0:s0 + 100], lmin, lmax,
                        emulate_bf16=True)
    got = net.grad.cpu().double().numpy()
    for name, (off, shape) in ws.TCN_OFFSETS.items():
        n = int(np.prod(shape))
        r, q = ref[off:off + n], got[off:off + n]
        # the data gradients between layers are stored in BF16 (2^-8 relative each)
        assert np.max(np.abs(q - r)) <= 3e-2 * np.max(np.abs(r)), name


def _stream_input(n, T, seed):
    g = torch.Generator().manual_seed(seed)
    rows = n * (T + 4)
    a = torch.randn(rows, 64, generator=g).clamp_min(0)
    gap = (torch.arange(rows) % (T + 4)) >= T
    a[gap] = 0
    return a.to(torch.bfloat16).cuda(), gap.numpy()


@pytest.mark.parametrize("mode", [0, 1])
def test_conv64_many_tiles(ws, mode):
    """120 series x 950 days = 114,480 rows: 299 tiles of 384 rows, the last one ragged."""
    n, T = 120, 950
    th = _theta_full(ws, 21)
    packed = ws.tcn_pack(th)
    o2 = ws.TCN_OFFSETS["W2"][0]
    Wb = otcn.bf16_round(th[o2:o2 + 36864].reshape(64, 64, 9).cpu().double().numpy())
    bias = th[ws.TCN_OFFSETS["b2"][0]:ws.TCN_OFFSETS["b2"][0] + 64].contiguous()
    inp, gap = _stream_input(n, T, 22)
    xs = inp.float().cpu().numpy().astype(np.float64)
    rows = xs.shape[0]
    assert -(-rows // 384) > 2 * torch.cuda.get_device_properties(0).multi_processor_count
    xp = np.zeros((rows + 8, 64))
    xp[4:4 + rows] = xs
    ref = np.zeros((rows, 64))
    if mode == 0:
        out, err = ws.tcn_conv64(inp, packed[1152:1152 + 36864], T, 0, bias=bias)
        for k in range(9):
            ref += xp[k:k + rows] @ Wb[:, :, k].T
        ref = np.maximum(ref + bias.cpu().double().numpy(), 0)
        ref[gap] = 0
    else:
        mask, _ = _stream_input(n, T, 23)
        out, err = ws.tcn_conv64(inp, packed[1152 + 36864:1152 + 2 * 36864], T, 1, mask=mask)
        for k in range(9):
            ref += xp[8 - k:8 - k + rows] @ Wb[:, :, k]
        ref = np.where(mask.float().cpu().numpy() > 0, ref, 0)
    torch.cuda.synchronize()
    assert int(err.abs().sum()) == 0
    got = out.float().cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref) - 2.0 ** -8 * np.abs(ref)) <= 1e-4 * scale
