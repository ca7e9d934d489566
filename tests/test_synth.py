"""Synthetic-input recipes: moments, structure, determinism (CPU only)."""
import numpy as np
import torch

from paper_2604_00048_b300 import synth


def test_hash_deterministic_and_uniform():
    idx = torch.arange(200000, dtype=torch.int64)
    a = synth.uniform(7, 3, idx)
    b = synth.uniform(7, 3, idx)
    assert torch.equal(a, b)
    assert 0.0 <= float(a.min()) and float(a.max()) < 1.0
    assert abs(float(a.mean()) - 0.5) < 0.005
    c = synth.uniform(7, 4, idx)
    assert abs(float(torch.corrcoef(torch.stack([a, c]))[0, 1])) < 0.01
    big = torch.tensor([2 ** 40 + 5, 2 ** 40 + 6], dtype=torch.int64)
    assert synth.hash_u32(1, 1, big)[0] != synth.hash_u32(1, 1, big)[1]


def test_tile_recipe_moments():
    rc = synth.RECIPES["hetero_tile"]
    rc = synth.Recipe(**{**rc.__dict__, "T": 730})
    out = synth.generate_tile(rc, 512, want_clean=True)
    x, w, lam, clean = out["x"], out["w"], out["lam"], out["clean"]
    T, B, P = x.shape
    assert (T, B, P) == (730, 10, 512) and w.shape == (730, 512) and lam.shape == (730, 512)
    frac = float(w.mean())
    assert abs(frac - rc.p_valid / rc.revisit) < 0.01            # valid fraction ~ p/5
    # acquisitions fall on one phase of the 5-day grid per series
    days = [torch.nonzero(w[:, p]).view(-1) for p in range(8)]
    for d in days:
        assert torch.all((d - d[0]) % 5 == 0)
    assert torch.all(x.permute(1, 0, 2)[:, w == 0] == 0)
    lo, hi = rc.lam_log10
    assert float(lam.min()) >= 10 ** lo and float(lam.max()) <= 10 ** hi
    # 15-day moving average of 10^U[1,5]: mean (1e5 - 10) / (4 ln 10)
    assert abs(float(lam.double().mean()) / ((1e5 - 10) / (4 * np.log(10))) - 1) < 0.05
    resid = (x - clean)[w.view(T, 1, P).expand(T, B, P) > 0]
    spikes = float((resid < -0.08).double().mean())
    assert 0.07 < spikes < 0.13                                  # ~10% of valid days
    core = resid[resid.abs() < 0.08]
    assert abs(float(core.std()) - 0.02) < 0.002                 # noise sd 0.02


def test_tile_series_offsets_are_consistent():
    rc = synth.RECIPES["layer"]
    a = synth.generate_tile(rc, 64, series0=0)
    b = synth.generate_tile(rc, 16, series0=32)
    for k in ("x", "w", "lam"):
        assert torch.equal(a[k][..., 32:48], b[k])
    assert "holdout" in a and torch.all(a["w"][a["holdout"]] == 0)
    hf = float(a["holdout"].double().sum() / (a["holdout"].double().sum() + a["w"].double().sum()))
    assert abs(hf - 0.2) < 0.04


def test_scalar_lambda_recipe():
    rc = synth.RECIPES["homo_fp64"]
    out = synth.generate_tile(rc, 300, dtype=torch.float64)
    assert out["lam"].shape == (300,) and out["x"].dtype == torch.float64
    assert float(out["lam"].min()) >= 1.0 and float(out["lam"].max()) <= 1e4


def test_ragged_layout_thirds_and_offsets():
    rc = synth.RECIPES["ragged"]
    n = 3000
    lengths, order, offsets = synth.ragged_layout(rc, n)
    assert int(lengths.min()) >= 120 and int(lengths.max()) <= 3288
    assert [int((order == k).sum()) for k in (1, 2, 3)] == [1000, 1000, 1000]
    assert torch.all(offsets[1:] - offsets[:-1] == lengths)
    out = synth.generate_ragged(rc, 50)
    assert out["x"].shape[0] == int(out["offsets"][-1])
    assert torch.all(out["x"][out["w"] == 0] == 0)


def test_piecewise_noise_variance_recipe():
    rc = synth.RECIPES["learned"]
    out = synth.generate_tile(rc, 256, want_clean=True)
    assert out["x"].shape == (730, 1, 256)


def test_dates_tile_is_the_daily_tile_on_acquisition_days():
    """generate_dates_tile keeps each series on its revisit days: strictly increasing dates 5
    days apart from the series' phase, every valid day of the daily tile among them with the
    same observation, no valid day dropped, lambda the daily field there times the revisit."""
    import torch

    from paper_2604_00048_b300 import synth

    rc = synth.Recipe(**{**synth.RECIPES["hetero_tile"].__dict__, "T": 200, "n_bands": 3})
    out = synth.generate_dates_tile(rc, 70, device="cpu", block=32)
    daily = synth.generate_tile(rc, 70, device="cpu")
    t = out["t"].long()
    Ta = (rc.T - rc.revisit) // rc.revisit + 1
    assert out["x"].shape == (Ta, 3, 70) and t.shape == (Ta, 70)
    assert torch.all(t[1:] - t[:-1] == rc.revisit) and torch.all(t[0] < rc.revisit) and torch.all(t[-1] < rc.T)
    assert torch.equal(out["w"], torch.gather(daily["w"], 0, t))
    assert torch.equal(out["x"], torch.gather(daily["x"], 0, t.view(Ta, 1, 70).expand(Ta, 3, 70)))
    assert torch.equal(out["w"].sum(0), daily["w"].sum(0))
    assert torch.allclose(out["lam"], torch.gather(daily["lam"], 0, t) * rc.revisit)
