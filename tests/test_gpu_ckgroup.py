"""Checkpoint groups of the tile kernels: one checkpoint per chunk against one per two chunks.

With two chunks per checkpoint the backward sweep recomputes both chunks resident in the
two-stage ring from one checkpoint and refills the ring in a different order (the next
group's earlier chunk first). Each mode of the kernel (smooth, the refinement's correction
solve with accumulation, the adjoint plain, refined and with the masked-MSE loss) runs at
chunk counts 1, 2, 3, 5 and 8 (odd counts leave a last chunk alone; ragged last chunks;
chunks shorter than d), with TMA staging (300 series) and per-thread copies (301 series,
row pitch not a multiple of 16 bytes). Both settings are compared with the FP64 oracle at
the tolerances of the other parity tests, and with each other: the arithmetic is the same,
so they agree to the last bits of FP32 rounding."""
import numpy as np
import pytest
import torch

from oracle import dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu

# (T, chunk cap): chunks per series 1, 2, 3 (last chunk of one day), 5 (chunks of 2 days,
# shorter than d = 3) and 8
SHAPES = [(5, 8), (16, 8), (17, 8), (9, 2), (61, 8)]


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    yield mod
    mod.tune_set(0, 0)


def _both(ws, chunk, fn):
    out = []
    for grp in (1, 2):
        ws.tune_set(0, chunk, checkpoint_group=grp)
        r = fn()
        ws.sync_status()
        out.append([t.clone() if isinstance(t, torch.Tensor) else t for t in r])
    ws.tune_set(0, 0)
    return out


def _close(a, b, rtol):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    scale = max(float(np.max(np.abs(b))), 1e-30)
    assert float(np.max(np.abs(a - b))) <= rtol * scale


@pytest.mark.parametrize("T,chunk", SHAPES)
@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("B", [3, 10])  # 10 bands: two threads per pixel
def test_smooth_refined_checkpoint_groups(ws, T, chunk, P, d, B):
    """Smooth + refinement step (MODE_SMOOTH, then MODE_RAW accumulating onto z0)."""
    rc, g, c = tile_inputs("layer", P, T=T, B=B, revisit=1, p_valid=0.7)
    (z1, s1), (z2, s2) = _both(ws, chunk, lambda: ws.smooth(g["x"], g["w"], g["lam"], d, refine=True))
    assert torch.equal(s1, s2)
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert np.array_equal(s2.cpu().numpy() == 0, ok)
    for z in (z1, z2):
        assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-4
    _close(z2, z1, 1e-6)


@pytest.mark.parametrize("T,chunk", SHAPES)
@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_smooth_fp64_checkpoint_groups(ws, T, chunk, P, d):
    rc, g, c = tile_inputs("layer", P, T=T, B=2, dtype=torch.float64, revisit=1, p_valid=0.7)
    (z1, s1), (z2, s2) = _both(ws, chunk, lambda: ws.smooth(g["x"], g["w"], g["lam"], d))
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert np.array_equal(s2.cpu().numpy() == 0, ok)
    # eps64 * cond(Omega): a few valid days under lambda up to 1e5 (the FP64 smooth tests' bound)
    assert rel_err_per_series(z2.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-6
    _close(z2, z1, 1e-12)


@pytest.mark.parametrize("T,chunk", SHAPES)
@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("refine", [False, True])
def test_adjoint_checkpoint_groups(ws, T, chunk, P, d, refine):
    """The adjoint (MODE_ADJ; with the refinement step also MODE_RAW and the accumulating
    MODE_ADJ) at the oracle's z rounded to FP32, 10 bands."""
    rc, g, c = tile_inputs("layer", P, T=T, B=10, revisit=1, p_valid=0.7)
    gz = torch.randn(g["x"].shape, generator=torch.Generator().manual_seed(T + P + d)).to("cuda")
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    zr = zr.astype(np.float32).astype(np.float64)
    z = torch.as_tensor(zr, dtype=torch.float32, device="cuda")
    (gx1, gl1, s1), (gx2, gl2, s2) = _both(
        ws, chunk, lambda: ws.smooth_adjoint(g["w"], g["lam"], z, gz, d, refine=refine))
    assert np.array_equal(s2.cpu().numpy() == 0, ok)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], d, zr, gz.cpu().double().numpy())
    assert rel_err_per_series(gx2.cpu().numpy()[:, :, ok], gxr[:, :, ok]) <= 1e-3
    num = np.max(np.abs(gl2.cpu().double().numpy() - glr)[:, ok], axis=0)
    den = np.maximum(np.max(np.abs(glr[:, ok]), axis=0), 1e-6)
    assert float(np.max(num / den)) <= 1e-3
    _close(gx2, gx1, 1e-5)
    _close(gl2, gl1, 1e-5)


@pytest.mark.parametrize("T,chunk", SHAPES)
@pytest.mark.parametrize("P", [300, 301])
def test_adjoint_mse_checkpoint_groups(ws, T, chunk, P):
    """The adjoint with the masked-MSE loss formed in the kernel (d = 2, 10 bands)."""
    d = 2
    rc, g, c = tile_inputs("layer", P, T=T, B=10, revisit=1, p_valid=0.7)
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    zr = zr.astype(np.float32).astype(np.float64)
    z = torch.as_tensor(zr, dtype=torch.float32, device="cuda")
    gen = torch.Generator().manual_seed(7 + T)
    target = (torch.as_tensor(zr, dtype=torch.float32) + 0.1 * torch.randn(zr.shape, generator=gen)).to("cuda")
    mask = (torch.rand((T, P), generator=gen) < 0.3).float().to("cuda")
    scale = 2.0 / (10 * T * P)
    (gx1, gl1, l1, s1), (gx2, gl2, l2, s2) = _both(
        ws, chunk, lambda: ws.smooth_adjoint_mse(g["w"], g["lam"], z, target, d, mask=mask, scale=scale))
    lr, gzr = dense.masked_mse(zr, target.cpu().double().numpy(), mask.cpu().double().numpy(), scale)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], d, zr, gzr)
    assert rel_err_per_series(gx2.cpu().numpy()[:, :, ok], gxr[:, :, ok]) <= 1e-3
    assert np.allclose(l2.cpu().double().numpy(), lr, rtol=1e-4, atol=1e-12)
    _close(gx2, gx1, 1e-5)
    _close(gl2, gl1, 1e-5)
    _close(l2, l1, 1e-6)
