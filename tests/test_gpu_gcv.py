"""GCV grid search (ws_gcv_smooth) against the dense FP64 oracle: per-value scores, the
choice, and the final smoothing at the chosen lambda."""
import numpy as np
import pytest
import torch

from oracle import dense
from paper_2604_00048_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


def _inputs(T, P, seed_shift=0, p_valid=None):
    base = synth.RECIPES["learned"].__dict__
    kw = {**base, "T": T, "seed": base["seed"] + seed_shift}
    if p_valid is not None:
        kw["p_valid"] = p_valid
    out = synth.generate_tile(synth.Recipe(**kw), P, device="cuda")
    return out["x"], out["w"]


def _check(ws, x, w, d, grid, ids, score_tol=5e-3, near_tol=1e-3):
    z, lam_best, scores, st = ws.gcv_smooth(x, w, grid, d, refine=True)
    torch.cuda.synchronize()
    xs, wc = x.cpu().double().numpy()[:, 0, :], w.cpu().double().numpy()
    zc, lb, sc, stc = z.cpu().double().numpy()[:, 0, :], lam_best.cpu().numpy(), scores.cpu().numpy(), st.cpu().numpy()
    for p in ids:
        if not dense.is_pd(wc[:, p], float(grid[0]), d):
            assert stc[p] == ws.SERIES_NOT_PD and np.all(np.isnan(sc[:, p]))
            continue
        best, ref_scores, _ = dense.gcv_one(xs[:, p], wc[:, p], grid, d)
        assert stc[p] == 0
        # scores: relative agreement with the FP64 oracle (FP32 solves, double-word
        # selected inverse). Where the smoother nearly interpolates (lambda = 1, d = 3) the
        # residuals x - z are small and carry FP32's error of z relative to x: ~2e-3 there,
        # ~3e-4 elsewhere; near the minimum, where the choice is made, 1e-3 is kept.
        # V = n RSS / (n - tr H)^2 amplifies an error of tr H by 2 tr H / (n - tr H): on a
        # series with a handful of valid days that factor passes 100 and FP32 cannot fix V,
        # so those grid values are left out of the score comparison (status, choice kept).
        n = wc[:, p].sum()
        trh = np.array([dense.hat_trace(wc[:, p], float(lv), d) for lv in grid])
        determined = 2 * trh / (n - trh) <= 100
        rel = np.abs(sc[:, p] - ref_scores) / ref_scores
        assert np.max(rel[determined], initial=0) <= score_tol, (p, sc[:, p], ref_scores)
        near = (ref_scores <= 1.1 * ref_scores.min()) & determined
        assert np.max(rel[near], initial=0) <= near_tol, (p, sc[:, p], ref_scores)
        if not determined.all():
            continue
        # the choice is the argmin of the kernel's own scores (ties to the smaller lambda) ...
        g = int(np.argmin(sc[:, p]))
        assert lb[p] == np.float32(grid[g])
        # ... and optimal under the oracle's scores within that tolerance
        assert ref_scores[g] <= ref_scores.min() * (1 + 2 * near_tol)
        # final smoothing at the chosen lambda
        zr = dense.smooth_one(xs[:, p], wc[:, p], float(np.float32(grid[g])), d)
        assert np.max(np.abs(zc[:, p] - zr)) / max(np.max(np.abs(zr)), 1e-6) <= 1e-4


@pytest.mark.parametrize("d", [1, 2, 3])
def test_gcv_parity_small(ws, d):
    """T = 200 (12 chunks and a ragged tail), 300 series (not a multiple of 16). At d = 3
    the FP32 solves inside the search carry ~1e-2 of the score at the grid's ends (near
    interpolation at lambda = 1, cond(Omega) ~ 4^d lambda at 1e5); the choice is still held
    to 1e-3 near the minimum."""
    x, w = _inputs(200, 300, d)
    _check(ws, x, w, d, ws.GCV_GRID, range(0, 300, 7), score_tol=2e-2 if d == 3 else 5e-3)


def test_gcv_short_grid_and_degenerate_series(ws):
    """Five grid values; one series without any valid day (NOT_PD, NaN scores) and one
    with a single valid day (NOT_PD at d = 2)."""
    x, w = _inputs(120, 40, 9)
    w[:, 3] = 0
    w[:, 5] = 0
    w[10, 5] = 1
    grid = [1.0, 10.0, 100.0, 1e3, 1e4]
    _check(ws, x, w, 2, grid, range(40))


def test_gcv_single_value_grid(ws):
    x, w = _inputs(90, 33, 4)
    z, lam_best, scores, st = ws.gcv_smooth(x, w, [50.0], 2)
    assert torch.all(lam_best == 50.0)
    zr, _ = ws.smooth(x, w, torch.full((33,), 50.0, device="cuda"), 2)
    assert torch.equal(z, zr)


def test_gcv_full_length_sampled(ws):
    """The learned-lambda evaluation shape at T = 730 (2 years): 4096 series, 12 sampled."""
    x, w = _inputs(730, 4096, 1)
    ids = np.random.default_rng(5).choice(4096, 12, replace=False)
    _check(ws, x, w, 2, ws.GCV_GRID, ids)


@pytest.mark.parametrize("d", [1, 2])
def test_gcv_on_acquisition_dates(ws, d):
    """ws_gcv_smooth_dates: the learned-lambda workload kept on each series' acquisition dates
    (5-day revisit from a random phase; 146 dates of 730 days), 200 series, log10 lambda in
    {2, 2 1/3, ..., 7}: scores against the dense GCV with the uneven-spacing operator, the choice optimal within 1e-3 of the oracle's
    scores, the final (refined) smooth at the chosen lambda within 1e-4."""
    base = synth.RECIPES["learned"].__dict__
    out = synth.generate_dates_tile(synth.Recipe(**base), 200, device="cpu")
    c = {k: v.double().numpy() for k, v in out.items()}
    g = {k: v.to("cuda") for k, v in out.items()}
    # on 5-day spacing a divided-difference row weighs (1/5)^(2d) of a daily one: the grid is
    # shifted two decades up so that its small end does not interpolate the observations
    grid = [10.0 ** (2 + i / 3.0) for i in range(16)]
    z, lam_best, scores, st = ws.gcv_smooth(g["x"], g["w"], grid, d, refine=True, t=g["t"])
    torch.cuda.synchronize()
    sc, lb, stc = scores.cpu().numpy(), lam_best.cpu().numpy(), st.cpu().numpy()
    zc = z.cpu().double().numpy()[:, 0, :]
    checked = 0
    for p in range(0, 200, 3):
        wp, xp, tp = c["w"][:, p], c["x"][:, 0, p], c["t"][:, p]
        if not dense.is_pd(wp, float(grid[0]), d):
            assert stc[p] == ws.SERIES_NOT_PD
            continue
        best, ref, _ = dense.gcv_one(xp, wp, grid, d, t=tp)
        n = wp.sum()
        trh = np.array([dense.hat_trace(wp, float(lv), d, tp) for lv in grid])
        determined = 2 * trh / (n - trh) <= 100
        rel = np.abs(sc[:, p] - ref) / ref
        assert np.max(rel[determined], initial=0) <= 5e-3, (p, sc[:, p], ref)
        if not determined.all():
            continue
        gi = int(np.argmin(sc[:, p]))
        assert lb[p] == np.float32(grid[gi]) and ref[gi] <= ref.min() * (1 + 2e-3)
        if gi == best:  # the oracle's own smooth at its own choice
            zr = dense.smooth_one_dates(xp, wp, float(np.float32(grid[best])), d, tp)
            assert np.max(np.abs(zc[:, p] - zr)) / max(np.max(np.abs(zr)), 1e-6) <= 1e-4
            checked += 1
    assert checked >= 20
