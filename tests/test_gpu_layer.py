"""The differentiable layer: autograd through the CUDA smooth and adjoint, stored-factor
and recompute modes, and the three-year 4-band workload with a held-out loss."""
import numpy as np
import pytest
import torch

from oracle import banded, dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import autograd, ws
    ws.tune_set(0, 0)
    return ws, autograd


@pytest.mark.parametrize("store", [False, True])
@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-3), (torch.float64, 1e-7)])
def test_autograd_grads_match_oracle_vjp(mods, store, dtype, tol):
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 200, T=150, B=3, dtype=dtype, revisit=1, p_valid=0.5)
    x = g["x"].clone().requires_grad_(True)
    lam = g["lam"].clone().requires_grad_(True)
    z, st = ag.whittaker_smooth(x, g["w"], lam, 2, refine=dtype == torch.float32, store_factor=store)
    G = torch.randn(z.shape, dtype=dtype, generator=torch.Generator().manual_seed(2)).to("cuda")
    (z * G).sum().backward()
    ws.sync_status()
    ok = st.cpu().numpy() == 0
    # the layer's backward is the C-ABI adjoint at the layer's own z ...
    gx_d, gl_d, _ = ws.smooth_adjoint(g["w"], g["lam"], z.detach(), G, 2)
    assert torch.equal(x.grad, gx_d) if not store else torch.allclose(x.grad, gx_d, rtol=tol, atol=1e-12)
    # ... and matches the oracle's gradients, which the oracle computes at its own z (the
    # adjoint's parity at a shared z is tested in test_gpu_adjoint.py)
    zr, okr = dense.smooth_tile(c["x"], c["w"], c["lam"], 2)
    assert np.array_equal(ok, okr)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], 2, zr, G.cpu().double().numpy())
    e_x = rel_err_per_series(x.grad.cpu().numpy()[:, :, ok], gxr[:, :, ok])
    gl = lam.grad.cpu().double().numpy()[:, ok]
    e_l = np.max(np.max(np.abs(gl - glr[:, ok]), 0) / np.maximum(np.max(np.abs(glr[:, ok]), 0), 1e-6))
    assert e_x <= tol and e_l <= tol, (e_x, e_l)


def test_gradcheck_fp64(mods):
    """Backward against finite differences of the forward, both on the GPU in FP64."""
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 4, T=14, B=2, dtype=torch.float64, revisit=1, p_valid=0.7)
    w = torch.ones_like(g["w"])
    x = g["x"].clone().requires_grad_(True)
    lam = (g["lam"] * 1e-3).clone().requires_grad_(True)
    fn = lambda xx, ll: ag.whittaker_smooth(xx, w, ll, 2, refine=False)[0]
    assert torch.autograd.gradcheck(fn, (x, lam), eps=1e-6, atol=1e-7, rtol=1e-6)


def test_store_and_recompute_agree_and_factored_api(mods):
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 257, T=200, B=2, dtype=torch.float64)
    x, w, lam = g["x"], g["w"], g["lam"]
    fac, st = ws.factor(w, lam, 2)
    fac2 = torch.empty_like(fac)
    z, st2 = ws.smooth(x, w, lam, 2, factor=fac2)
    assert torch.equal(st, st2)
    ok = st == 0
    assert torch.allclose(fac[:, :, ok], fac2[:, :, ok], rtol=1e-12, atol=1e-14)
    z2 = ws.solve(fac, w, x, 2)
    assert torch.allclose(z2[:, :, ok], z[:, :, ok], rtol=1e-10, atol=1e-12)
    G = torch.randn_like(z)
    gx1, gl1, _ = ws.smooth_adjoint(w, lam, z, G, 2, log_lambda=True)
    gx2, gl2, _ = ws.smooth_adjoint(w, lam, z, G, 2, log_lambda=True, factor=fac)
    ws.sync_status()
    assert torch.allclose(gx1[:, :, ok], gx2[:, :, ok], rtol=1e-9, atol=1e-12)
    assert torch.allclose(gl1[:, ok], gl2[:, ok], rtol=1e-8, atol=1e-14)


def test_fd_check_fp64_64px_T60(mods):
    """FP64 central finite differences on 64 pixels, T = 60: dL/dx and dL/dlog(lambda) of a
    held-out loss through the GPU forward, against the GPU adjoint."""
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 64, T=60, B=4, dtype=torch.float64)
    x, w, lam, hold = g["x"], g["w"], g["lam"], g["holdout"]
    hb = hold.unsqueeze(1).expand_as(x).to(torch.float64)

    def loss(xx, ll):
        z, _ = ws.smooth(xx, w, ll, 2)
        return float((((z - x) ** 2) * hb).sum() / max(1.0, float(hb.sum())))

    z, st = ws.smooth(x, w, lam, 2)
    gz = 2 * (z - x) * hb / max(1.0, float(hb.sum()))
    gx, gll, _ = ws.smooth_adjoint(w, lam, z, gz, 2, log_lambda=True)
    ws.sync_status()
    gen = torch.Generator().manual_seed(9)
    for _ in range(6):
        v = torch.randn(x.shape, dtype=torch.float64, generator=gen).to("cuda")
        h = 1e-4
        fd = (loss(x + h * v, lam) - loss(x - h * v, lam)) / (2 * h)
        an = float((gx * v).sum())
        assert abs(fd - an) <= 1e-6 * max(1e-8, abs(an)) + 1e-12
        u = torch.randn(lam.shape, dtype=torch.float64, generator=gen).to("cuda")
        fd = (loss(x, lam * torch.exp(h * u)) - loss(x, lam * torch.exp(-h * u))) / (2 * h)
        an = float((gll * u).sum())
        assert abs(fd - an) <= 1e-6 * max(1e-8, abs(an)) + 1e-12


def test_layer_workload_sampled(mods):
    """The 65,536-pixel, T = 1095, 4-band workload: held-out MSE loss through the layer
    (FP32, refined forward); gradients with respect to x and log lambda, store and
    recompute, checked on 1024 sampled pixels against the FP64 banded oracle."""
    ws, ag = mods
    rc, g, c = tile_inputs("layer", 65536, B=4)
    x = g["x"].clone().requires_grad_(True)
    loglam = g["lam"].log().clone().requires_grad_(True)
    hold = g["holdout"]
    hb = hold.unsqueeze(1).expand_as(x).to(torch.float32)
    n = float(hb.sum())
    grads = {}
    for store in (False, True):
        x.grad = None
        loglam.grad = None
        z, st = ag.whittaker_smooth(x, g["w"], loglam.exp(), 2, refine=True, store_factor=store)
        loss = (((z - g["x"]) ** 2) * hb).sum() / n
        loss.backward()
        grads[store] = (x.grad.clone(), loglam.grad.clone(), z.detach().clone(), st.clone())
    ws.sync_status()
    gx0, gl0, z0, st0 = grads[False]
    gx1, gl1, _, _ = grads[True]
    assert torch.allclose(gx0, gx1, rtol=1e-3, atol=1e-9) and torch.allclose(gl0, gl1, rtol=1e-3, atol=1e-9)
    idx = np.random.default_rng(4).choice(65536, 1024, replace=False)
    ok = st0.cpu().numpy()[idx] == 0
    idx = idx[ok]
    zs = z0[:, :, idx].cpu().double().numpy()
    # the oracle runs the whole pipeline itself: its z, the held-out loss gradient at its z,
    # then the vector-Jacobian products
    zr, _ = banded.smooth_tile(c["x"][:, :, idx], c["w"][:, idx], c["lam"][:, idx], 2)
    assert rel_err_per_series(zs, zr) <= 1e-4
    hbn = hold.cpu().numpy()[:, None, idx].astype(np.float64)
    gz = 2 * (zr - c["x"][:, :, idx]) * hbn / n
    gxr, glr, _ = banded.vjp_tile(c["w"][:, idx], c["lam"][:, idx], 2, zr, gz, log_lambda=True)
    e_x = rel_err_per_series(gx0[:, :, idx].cpu().numpy(), gxr)
    gl = gl0[:, idx].cpu().double().numpy()
    e_l = np.max(np.max(np.abs(gl - glr), 0) / np.maximum(np.max(np.abs(glr), 0), 1e-12))
    assert e_x <= 1e-3 and e_l <= 1e-3, (e_x, e_l)
