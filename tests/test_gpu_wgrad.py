"""Gradient with respect to the observation weights (soft weights of Eq. 1): the adjoint
with WS_ADJ_RAW_G followed by ws_weight_grad, against the FP64 oracle (dL/dw_t = sum_b g_tb
(x_tb - z_tb), gaps taking x = 0), at a forward output z shared by both sides (the
oracle's own z, rounded to the GPU dtype); recompute, stored-factor and refined adjoints;
the layer's gradient in w; an FP64 finite-difference check through the GPU forward.
Tolerances: 1e-3 per series for FP32 (a gradient), 1e-7 for FP64."""
import numpy as np
import pytest
import torch

from oracle import dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import autograd, ws
    ws.tune_set(0, 0)
    return ws, autograd


def _rel_tp(a, b):
    """[T, P] arrays: per series ||a - b||_inf / max(||b||_inf, 1e-12), max over series."""
    num = np.max(np.abs(a - b), axis=0)
    den = np.maximum(np.max(np.abs(b), axis=0), 1e-12)
    return float(np.max(num / den)) if num.size else 0.0


def _case(ws, recipe, P, T, B, d, dtype, mode, **over):
    rc, g, c = tile_inputs(recipe, P, T=T, B=B, dtype=dtype, **over)
    zr, okr = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    z = torch.as_tensor(zr, dtype=dtype, device="cuda")
    gz = torch.randn(g["x"].shape, dtype=dtype, generator=torch.Generator().manual_seed(6)).to("cuda")
    fac = None
    if mode == "store":
        fac, _ = ws.factor(g["w"], g["lam"], d)
    gx, glam, gw, st = ws.smooth_adjoint_weights(g["x"], g["w"], g["lam"], z, gz, d, log_lambda=True,
                                                 factor=fac, refine=mode == "refine")
    ws.sync_status()
    gzc = gz.cpu().double().numpy()
    gwr = dense.vjp_w_tile(c["x"], c["w"], c["lam"], d, zr, gzc)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], d, zr, gzc, log_lambda=True)
    ok = okr if mode == "store" else st.cpu().numpy() == 0
    if mode != "store":
        assert np.array_equal(ok, okr)
    return (gx.cpu().double().numpy(), glam.cpu().double().numpy(), gw.cpu().double().numpy()), (gxr, glr, gwr), ok


@pytest.mark.parametrize("mode", ["recompute", "store", "refine"])
@pytest.mark.parametrize("d", [1, 2])
def test_weight_grad_fp32(mods, mode, d):
    """Heteroscedastic inputs (5-day revisits, lambda up to 1e5), 300 series x 200 days x 3
    bands: gw, and gx = W g from the same pass, within 1e-3 of the oracle."""
    ws, _ = mods
    (gx, glam, gw), (gxr, glr, gwr), ok = _case(ws, "hetero_tile", 300, 200, 3, d, torch.float32, mode)
    e_w, e_x = _rel_tp(gw[:, ok], gwr[:, ok]), rel_err_per_series(gx[:, :, ok], gxr[:, :, ok])
    assert e_w <= 1e-3 and e_x <= 1e-3, (e_w, e_x)
    assert np.all(gw[:, ~ok] == 0)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_weight_grad_fp64(mods, d):
    """FP64, daily acquisitions valid with p = 0.5, 130 series x 120 days x 2 bands."""
    ws, _ = mods
    (gx, glam, gw), (gxr, glr, gwr), ok = _case(ws, "layer", 130, 120, 2, d, torch.float64, "recompute",
                                               revisit=1, p_valid=0.5)
    # at d = 4 cond(Omega) reaches ~1e8 on these inputs: two FP64 solves agree to ~2e-8
    assert _rel_tp(gw[:, ok], gwr[:, ok]) <= 1e-7
    assert rel_err_per_series(gx[:, :, ok], gxr[:, :, ok]) <= 1e-7


def test_weight_grad_outputs(mods):
    """gx written in place over g, into a separate array or not at all: same gw and gx; the
    gradient in lambda is unchanged by the raw-g flag."""
    ws, _ = mods
    rc, g, c = tile_inputs("layer", 200, T=90, B=2)
    z, _ = ws.smooth(g["x"], g["w"], g["lam"], 2)
    gz = torch.randn_like(z)
    gx_a, gl_a, gw_a, _ = ws.smooth_adjoint_weights(g["x"], g["w"], g["lam"], z, gz, 2)
    gx_b, gl_b, gw_b, _ = ws.smooth_adjoint_weights(g["x"], g["w"], g["lam"], z, gz, 2, want_gx=False)
    gx_c, gl_c, _ = ws.smooth_adjoint(g["w"], g["lam"], z, gz, 2)
    ws.sync_status()
    assert gx_b is None and torch.equal(gw_a, gw_b)
    assert torch.equal(gx_a, gx_c) and torch.equal(gl_a, gl_c) and torch.equal(gl_b, gl_c)


def test_layer_weight_gradient(mods):
    """The autograd layer returns dL/dw when w requires grad: equal to the direct C-ABI calls
    at the layer's z (FP32), and within 1e-8 of the oracle in FP64 (oracle at its own z)."""
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 150, T=100, B=2)
    w = g["w"].clone().requires_grad_(True)
    x = g["x"].clone().requires_grad_(True)
    z, st = ag.whittaker_smooth(x, w, g["lam"], 2, refine=True)
    G = torch.randn(z.shape, generator=torch.Generator().manual_seed(3)).to("cuda")
    (z * G).sum().backward()
    gx_d, _, gw_d, _ = ws.smooth_adjoint_weights(g["x"], g["w"], g["lam"], z.detach(), G, 2, want_glam=False)
    ws.sync_status()
    assert torch.equal(w.grad, gw_d) and torch.equal(x.grad, gx_d)

    rc, g, c = tile_inputs("layer", 96, T=80, B=2, dtype=torch.float64, revisit=1, p_valid=0.5)
    w = g["w"].clone().requires_grad_(True)
    z, st = ag.whittaker_smooth(g["x"], w, g["lam"], 2, refine=False)
    G = torch.randn(z.shape, dtype=torch.float64, generator=torch.Generator().manual_seed(4)).to("cuda")
    (z * G).sum().backward()
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], 2)
    gwr = dense.vjp_w_tile(c["x"], c["w"], c["lam"], 2, zr, G.cpu().numpy())
    assert _rel_tp(w.grad.cpu().numpy()[:, ok], gwr[:, ok]) <= 1e-8


def test_weight_grad_finite_differences_fp64(mods):
    """FP64 finite differences of L = <G, z(w)> through the GPU forward along random
    directions of w: central differences on the valid days, one-sided second-order ones on
    the gaps (w = 0 cannot step below 0; x = 0 there), against <dL/dw, v> from the GPU
    adjoint."""
    ws, _ = mods
    rc, g, c = tile_inputs("layer", 64, T=60, B=3, dtype=torch.float64)
    x, w, lam = g["x"], g["w"], g["lam"]
    x = torch.where(w[:, None, :] > 0, x, torch.zeros_like(x))
    G = torch.randn(x.shape, dtype=torch.float64, generator=torch.Generator().manual_seed(8)).to("cuda")
    z, st = ws.smooth(x, w, lam, 2)
    _, _, gw, _ = ws.smooth_adjoint_weights(x, w, lam, z, G, 2, want_gx=False, want_glam=False)
    ws.sync_status()
    ok = st == 0

    def L(ww):
        zz, _ = ws.smooth(x, ww, lam, 2)
        return float((G * zz)[:, :, ok].sum())

    gen = torch.Generator().manual_seed(10)
    for on in (True, False):
        h = 1e-5 if on else 1e-6  # the one-sided formula's error is O(h^2 L''')
        for _ in range(3):
            v = torch.rand(w.shape, dtype=torch.float64, generator=gen).to("cuda") * 0.5
            v = torch.where((w > 0) == on, v, torch.zeros_like(v))
            if on:
                fd = (L(w + h * v) - L(w - h * v)) / (2 * h)
            else:
                fd = (-3 * L(w) + 4 * L(w + h * v) - L(w + 2 * h * v)) / (2 * h)
            an = float((gw * v)[:, ok].sum())
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (on, fd, an)
