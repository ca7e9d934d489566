"""The adjoint with Section 4.3's masked-MSE loss fused into its sweeps (ws_solve_adjoint_mse)
against the FP64 oracle: the loss per series and its gradient dL/dz = scale m (z - target)
from oracle/dense.masked_mse, then the oracle's VJP (Eqs. 4-5) of that gradient. Inputs as
the differentiable-layer workload: 20% of the valid days held out (weight 0, observation
kept as the target); the loss is their mean squared error (scale = 2 / n_held). z is the
oracle's smooth rounded to FP32 (both sides differentiate at the same z). Tolerances: 1e-3
on gx and dL/dlog lambda (per series, as the other adjoint tests), 1e-5 on the loss."""
import numpy as np
import pytest
import torch

from oracle import dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    yield mod
    mod.tune_set(0, 0, 0)


def _glam_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    if a.ndim == 1:
        return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-6)))
    return float(np.max(np.max(np.abs(a - b), axis=0) / np.maximum(np.max(np.abs(b), axis=0), 1e-6)))


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("B", [1, 4, 10])
@pytest.mark.parametrize("P", [260, 261])   # 260: TMA staging; 261: plain loads
def test_adjoint_mse_matches_oracle(ws, d, B, P):
    ws.tune_set(0, 8)
    rc, g, c = tile_inputs("layer", P, T=120, B=B, revisit=1, p_valid=0.5)
    hold = c["holdout"].astype(np.float64)
    n_held = int(hold.sum()) * B
    scale = 2.0 / n_held
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    zr = zr.astype(np.float32).astype(np.float64)
    z = torch.as_tensor(zr, dtype=torch.float32, device="cuda")
    mask = g["holdout"].to(torch.float32)
    gx, glam, loss, st = ws.smooth_adjoint_mse(g["w"], g["lam"], z, g["x"], d, mask=mask, scale=scale,
                                               log_lambda=True)
    ws.sync_status()
    okg = st.cpu().numpy() == 0
    assert np.array_equal(okg, ok)
    lr, gzr = dense.masked_mse(zr, c["x"], hold, scale)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], d, zr, gzr, log_lambda=True)
    assert rel_err_per_series(gx.cpu().numpy()[:, :, ok], gxr[:, :, ok]) <= 1e-3
    assert _glam_err(glam.cpu().numpy()[:, ok], glr[:, ok]) <= 1e-3
    assert np.max(np.abs(loss.cpu().numpy() - lr)) <= 1e-5 * max(np.max(np.abs(lr)), 1e-12)
    assert np.all(glam.cpu().numpy()[-d:, :] == 0)


def test_adjoint_mse_unmasked_scalar_lambda_and_band_groups(ws):
    """mask = NULL (every day weighs 1, the training loss against the clean signal), scalar
    lambda (Eq. 2: glam per series), 13 bands in two band groups (the loss and glam summed
    over both)."""
    ws.tune_set(0, 0)
    rc, g, c = tile_inputs("homo_fp64", 200, T=150, B=13)
    tgt = torch.sin(torch.arange(150, device="cuda", dtype=torch.float32) / 9.0)[:, None, None].expand(150, 13, 200)
    tgt = tgt.contiguous()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], 2)
    zr = zr.astype(np.float32).astype(np.float64)
    z = torch.as_tensor(zr, dtype=torch.float32, device="cuda")
    scale = 2.0 / tgt.numel()
    gx, glam, loss, st = ws.smooth_adjoint_mse(g["w"], g["lam"], z, tgt, 2, scale=scale, log_lambda=True)
    ws.sync_status()
    lr, gzr = dense.masked_mse(zr, tgt.cpu().double().numpy(), None, scale)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], 2, zr, gzr, log_lambda=True)
    assert rel_err_per_series(gx.cpu().numpy()[:, :, ok], gxr[:, :, ok]) <= 1e-3
    assert _glam_err(glam.cpu().numpy()[ok], glr[ok]) <= 1e-3
    assert np.max(np.abs(loss.cpu().numpy() - lr)) <= 1e-5 * np.max(np.abs(lr))


def test_adjoint_mse_equals_unfused_path(ws):
    """The fused call and ws_mse_grad + ws_solve_adjoint (the gradient written to memory and
    read back) agree to FP32 rounding on the three-year layer workload."""
    ws.tune_set(0, 0)
    rc, g, c = tile_inputs("layer", 512, B=4)
    z, _ = ws.smooth(g["x"], g["w"], g["lam"], 2)
    mask = g["holdout"].to(torch.float32)
    scale = 2.0 / float(mask.sum() * 4)
    gx, glam, loss, st = ws.smooth_adjoint_mse(g["w"], g["lam"], z, g["x"], 2, mask=mask, scale=scale,
                                               log_lambda=True)
    gz = (scale * mask[:, None, :] * (z - g["x"])).contiguous()
    gx2, glam2, _ = ws.smooth_adjoint(g["w"], g["lam"], z, gz, 2, log_lambda=True)
    ws.sync_status()
    ok = st.cpu().numpy() == 0
    assert rel_err_per_series(gx.cpu().numpy()[:, :, ok], gx2.cpu().numpy()[:, :, ok]) <= 1e-5
    assert _glam_err(glam.cpu().numpy()[:, ok], glam2.cpu().numpy()[:, ok]) <= 1e-5
    ref = 0.5 * scale * (mask[:, None, :] * (z - g["x"]) ** 2).sum(dim=(0, 1))
    assert torch.allclose(loss, ref, rtol=1e-5, atol=1e-12)


def test_adjoint_mse_layer_workload_full_size_sampled(ws):
    """The differentiable-layer workload at full size (65,536 series x 1095 days x 4 bands,
    20% of the valid days held out) in the launch configuration of a training step: the GPU
    smooth's z, the fused adjoint on all series, and 64 sampled series (first and last
    included) against the oracle's masked_mse + VJP at that z (1e-3)."""
    ws.tune_set(0, 0, 0)
    from paper_2604_00048_b300 import synth
    rc = synth.RECIPES["layer"]
    P = 65536
    out = synth.generate_tile(rc, P, device="cuda")
    x, w, lam, hold = out["x"], out["w"], out["lam"], out["holdout"]
    z, _ = ws.smooth(x, w, lam, rc.d, refine=True)
    mask = hold.to(torch.float32)
    scale = 2.0 / float(mask.sum() * rc.n_bands)
    gx, glam, loss, st = ws.smooth_adjoint_mse(w, lam, z, x, rc.d, mask=mask, scale=scale, log_lambda=True)
    ws.sync_status()
    idx = np.sort(np.concatenate([[0, P - 1], np.random.default_rng(9).choice(np.arange(1, P - 1), 62, replace=False)]))
    zs = z[:, :, idx].cpu().double().numpy()
    xs, ws_, ls = x[:, :, idx].cpu().double().numpy(), w[:, idx].cpu().double().numpy(), lam[:, idx].cpu().double().numpy()
    ms = mask[:, idx].cpu().double().numpy()
    lr, gzr = dense.masked_mse(zs, xs, ms, scale)
    gxr, glr = dense.vjp_tile(ws_, ls, rc.d, zs, gzr, log_lambda=True)
    ok = st[idx].cpu().numpy() == 0
    assert ok.all()
    assert rel_err_per_series(gx[:, :, idx].cpu().numpy(), gxr) <= 1e-3
    assert _glam_err(glam[:, idx].cpu().numpy(), glr) <= 1e-3
    assert np.max(np.abs(loss[idx].cpu().numpy() - lr) / np.maximum(np.abs(lr), 1e-30)) <= 1e-5
