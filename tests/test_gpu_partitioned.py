"""Partitioned parallel-in-time solve (ws_smooth_partitioned) against the FP64 oracles.

The three-year and nine-year workloads with few series: the 10-band heteroscedastic tile
(5-day revisits valid with p = 0.35, per-day lambda 10^U[1,5] smoothed) at T = 3288, 1 to 64
series, against the dense oracle (Eq. 3 by dense Cholesky) on sampled series and the banded
FP64 oracle on all; every order d = 1..4 on daily-valid inputs at lengths that put domain
edges and a short last domain in different places; FP64 data; scalar lambda; status codes.
Tolerance: max relative error per series and band 1e-4 for FP32 outputs (no refinement
step: the solve runs in double-float), 1e-6 for FP64 (eps64 * cond(Omega) on these inputs)."""
import numpy as np
import pytest
import torch

from oracle import banded, dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


@pytest.mark.parametrize("P", [1, 5, 64])
def test_partitioned_long_series_against_dense_oracle(ws, P):
    rc, g, c = tile_inputs("hetero_tile", P, B=10)
    assert rc.T == 3288
    z, st = ws.smooth_partitioned(g["x"], g["w"], g["lam"], 2)
    ws.sync_status()
    ok = st.cpu().numpy() == 0
    zb, stb = banded.smooth_tile(c["x"], c["w"], c["lam"], 2)
    assert np.array_equal(ok, stb == 0)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zb[:, :, ok]) <= 1e-4
    for p in np.random.default_rng(P).choice(P, size=min(P, 3), replace=False):
        zd = dense.smooth_one(c["x"][:, :, p], c["w"][:, p], c["lam"][:, p], 2)
        assert rel_err_per_series(z.cpu().numpy()[:, :, p:p + 1], zd[:, :, None]) <= 1e-4


@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("T", [7, 64, 65, 700, 1025])
def test_partitioned_orders_and_domain_edges(ws, d, T):
    if T <= d:
        pytest.skip("needs T > d")
    P = 7
    rc, g, c = tile_inputs("layer", P, T=T, B=3, revisit=1, p_valid=0.5)
    z, st = ws.smooth_partitioned(g["x"], g["w"], g["lam"], d)
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert np.array_equal(st.cpu().numpy() == 0, ok)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-4
    assert np.all(z.cpu().numpy()[:, :, ~ok] == 0)


@pytest.mark.parametrize("d", [2, 3])
def test_partitioned_fp64_and_scalar_lambda(ws, d):
    rc, g, c = tile_inputs("homo_fp64", 9, T=900, B=2, dtype=torch.float64)
    z, st = ws.smooth_partitioned(g["x"], g["w"], g["lam"], d)
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert np.array_equal(st.cpu().numpy() == 0, ok)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-6
    rc, g, c = tile_inputs("homo_fp64", 9, T=900, B=2)
    z, st = ws.smooth_partitioned(g["x"], g["w"], g["lam"], d)
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], d)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-4


def test_partitioned_status_codes(ws):
    """A series with one valid day (d = 2: not positive definite), one with a negative
    weight and one with a zero lambda row (invalid arguments), among regular ones: their
    codes match the tile path's and their outputs are zero."""
    rc, g, c = tile_inputs("layer", 6, T=300, B=2, revisit=1, p_valid=0.5)
    w = g["w"].clone()
    lam = g["lam"].clone()
    w[:, 1] = 0
    w[10, 1] = 1
    w[50, 2] = -1
    lam[20, 3] = 0
    z, st = ws.smooth_partitioned(g["x"], w, lam, 2)
    zt, stt = ws.smooth(g["x"], w, lam, 2)
    ws.sync_status()
    assert torch.equal(st, stt)
    assert st[1].item() == ws.SERIES_NOT_PD and st[2].item() == ws.SERIES_BADARG and st[3].item() == ws.SERIES_BADARG
    bad = (st != 0).cpu().numpy()
    assert np.all(z.cpu().numpy()[:, :, bad] == 0)
    zr, ok = dense.smooth_tile(c["x"][:, :, [0, 4, 5]], c["w"][:, [0, 4, 5]], c["lam"][:, [0, 4, 5]], 2)
    assert rel_err_per_series(z.cpu().numpy()[:, :, [0, 4, 5]], zr) <= 1e-4


def test_partitioned_1024_series_sampled(ws):
    """1,024 series of the 10-band tile at T = 3288 (the top of the few-series regime): 32
    sampled series against the banded FP64 oracle (1e-4) and agreement with the tile path
    with its refinement step on all series."""
    from paper_2604_00048_b300 import synth
    rc = synth.RECIPES["hetero_tile"]
    P = 1024
    out = synth.generate_tile(rc, P, device="cuda")
    z, st = ws.smooth_partitioned(out["x"], out["w"], out["lam"], 2)
    zt, stt = ws.smooth(out["x"], out["w"], out["lam"], 2, refine=True)
    ws.sync_status()
    assert torch.equal(st, stt) and int((st != 0).sum()) == 0
    rel = ((z - zt).abs().amax(dim=0) / zt.abs().amax(dim=0).clamp_min(1e-6)).max().item()
    assert rel <= 1e-4
    idx = np.random.default_rng(4).choice(P, 32, replace=False)
    c = {k: out[k][..., idx].cpu().double().numpy() for k in ("x", "w", "lam")}
    zb, stb = banded.smooth_tile(c["x"], c["w"], c["lam"], 2)
    assert np.all(stb == 0)
    assert rel_err_per_series(z[:, :, idx].cpu().numpy(), zb) <= 1e-4
