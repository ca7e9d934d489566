"""The tile kernels at 64 and 128 pixel series per CTA (ws_tune_pixels_per_cta, FP32) against
the FP64 oracle: smooth with its refinement step (z0 staged with the correction solve's
chunks), and the adjoint (z staged with its chunks). Several 64-pixel tiles plus a ragged
one, chunks of 8 days with a ragged last chunk, TMA (P = 300) and plain-load (P = 301)
staging, one and two threads per pixel. Tolerances as the 128-pixel tests: 1e-4 on z,
1e-3 on the gradients (Eqs. 4-5)."""
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


@pytest.mark.parametrize("npc", [64, 128])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("B", [3, 10])
def test_smooth_refined_np(ws, d, P, B, npc):
    ws.tune_set(0, 8, npc)
    rc, g, c = tile_inputs("layer", P, T=61, B=B, revisit=1, p_valid=0.5)
    z, st = ws.smooth(g["x"], g["w"], g["lam"], d, refine=True)
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert np.array_equal(st.cpu().numpy() == 0, ok)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-4
    assert np.all(z.cpu().numpy()[:, :, ~ok] == 0)


@pytest.mark.parametrize("npc", [64, 128])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("B", [4, 10])
def test_adjoint_np(ws, d, P, B, npc):
    ws.tune_set(0, 8, npc)
    rc, g, c = tile_inputs("layer", P, T=120, B=B, revisit=1, p_valid=0.5)
    gz = torch.randn(g["x"].shape, generator=torch.Generator().manual_seed(5)).to("cuda")
    zr, okr = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    zr = zr.astype(np.float32).astype(np.float64)
    z = torch.as_tensor(zr, dtype=torch.float32, device="cuda")
    gx, glam, st = ws.smooth_adjoint(g["w"], g["lam"], z, gz, d, log_lambda=True, refine=True)
    ws.sync_status()
    ok = st.cpu().numpy() == 0
    assert np.array_equal(ok, okr)
    gxr, glr = dense.vjp_tile(c["w"], c["lam"], d, zr, gz.cpu().double().numpy(), log_lambda=True)
    assert rel_err_per_series(gx.cpu().numpy()[:, :, ok], gxr[:, :, ok]) <= 1e-3
    num = np.max(np.abs(glam.cpu().numpy()[:, ok] - glr[:, ok]), axis=0)
    assert np.max(num / np.maximum(np.max(np.abs(glr[:, ok]), axis=0), 1e-6)) <= 1e-3


def test_np64_matches_np128_bitwise_on_one_chunk_layout(ws):
    """Same chunk length, 64 or 128 pixels per CTA: every series runs the same arithmetic,
    so z is bit-identical."""
    rc, g, c = tile_inputs("hetero_tile", 1000, T=200)
    ws.tune_set(0, 6, 128)
    z1, s1 = ws.smooth(g["x"], g["w"], g["lam"], 2)
    ws.tune_set(0, 6, 64)
    z2, s2 = ws.smooth(g["x"], g["w"], g["lam"], 2)
    ws.sync_status()
    assert torch.equal(z1, z2) and torch.equal(s1, s2)
