"""Seeded synthetic pixel time series shaped like multi-year Sentinel-2 tiles.

This module holds none of the smoother's arithmetic. It only draws counter-based
random numbers and turns them into inputs: a double-logistic seasonal signal per
band, a 5-day revisit with random validity (weights 0/1), Gaussian noise, negative
spikes that stand in for undetected clouds, and per-series or per-day smoothing
weights lambda. The paper's own data (Sentinel-2 / MAJA tiles over France, Section 4.1)
is not available; these recipes stand in for it with its shapes (daily grid over
2016-2024, 10 spectral bands, ragged lengths).

Every value is a pure function of (seed, stream, index), computed with integer
torch ops that give identical results on CPU and GPU. Transcendental steps
(exp, log, cos, pow) may differ in the last bit between devices, so a consumer
that compares two implementations generates once and copies the bytes.

Layouts produced:
  tile   : x[t, b, p], w[t, p], lam[t, p] (per day) or lam[p] (scalar), p fastest
  ragged : series i occupies [off[i], off[i+1]) of each flat array
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import Optional

import torch

_M32 = 0xFFFFFFFF

# stream ids (each names one independent family of random numbers)
S_PHASE, S_VALID, S_SPIKE_DAY, S_SPIKE_MAG, S_NOISE_A, S_NOISE_B = 1, 2, 3, 4, 5, 6
S_OFF, S_AMP, S_SOS, S_EOS, S_R1, S_R2 = 7, 8, 9, 10, 11, 12
S_LAM, S_HOLD, S_LEN, S_ORDER, S_CHANGE, S_VAR = 13, 14, 15, 16, 17, 18


def _mix(h: torch.Tensor) -> torch.Tensor:
    """32-bit avalanche on int64 lanes; every product stays below 2**63."""
    h = h ^ (h >> 16)
    h = (h * 0x7FEB352D) & _M32
    h = h ^ (h >> 15)
    h = (h * 0x5BD1E995) & _M32
    h = h ^ (h >> 16)
    return h


def _mix_int(v: int) -> int:
    v &= _M32
    v ^= v >> 16
    v = (v * 0x7FEB352D) & _M32
    v ^= v >> 15
    v = (v * 0x5BD1E995) & _M32
    v ^= v >> 16
    return v


def hash_u32(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Counter-based 32-bit hash of a non-negative int64 index (< 2**62)."""
    base = _mix_int(_mix_int(seed * 0x9E3779B1 + 0x632BE5AB) ^ (stream * 0x27D4EB2D))
    idx = idx.to(torch.int64)
    h = _mix((idx & _M32) ^ base)
    h = _mix(h ^ (idx >> 32) ^ 0x165667B1)
    return h


def uniform(seed: int, stream: int, idx: torch.Tensor, dtype=torch.float32) -> torch.Tensor:
    """U[0, 1) with 24 random bits (exact in float32 and float64)."""
    return (hash_u32(seed, stream, idx) >> 8).to(dtype) * (1.0 / 16777216.0)


def uniform_open(seed: int, stream: int, idx: torch.Tensor, dtype=torch.float32) -> torch.Tensor:
    """U(0, 1): never exactly 0, safe under log."""
    return ((hash_u32(seed, stream, idx) >> 8).to(dtype) + 0.5) * (1.0 / 16777216.0)


def normal(seed: int, stream_a: int, stream_b: int, idx: torch.Tensor, dtype=torch.float32):
    """Standard normal by the Box-Muller transform of two independent uniforms."""
    u1 = uniform_open(seed, stream_a, idx, dtype)
    u2 = uniform(seed, stream_b, idx, dtype)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos((2.0 * math.pi) * u2)


@dataclass(frozen=True)
class Recipe:
    """One synthetic workload. Units: days on a daily grid starting 2016-01-01."""
    seed: int
    T: int
    n_bands: int = 1
    d: int = 2
    p_valid: float = 0.35          # probability that an acquisition is valid
    revisit: int = 5               # days between acquisitions
    noise_sd: float = 0.02         # homoscedastic noise (used when noise_var is None)
    noise_var: Optional[tuple] = None   # (lo, hi): piecewise-constant variance U[lo, hi]
    change_rate: float = 3.0       # mean number of variance change points per series
    spike_frac: float = 0.10       # fraction of valid days hit by a negative spike
    spike_mag: tuple = (0.1, 0.5)
    lam_kind: str = "per_day"      # "per_day" | "scalar"
    lam_log10: tuple = (1.0, 5.0)  # lambda = 10 ** U[lo, hi]
    lam_window: int = 0            # centred moving average of the per-day lambda (0 = none)
    holdout_frac: float = 0.0      # fraction of valid days held out (weight set to 0)


# The five workloads: shapes, distributions and seeds.
RECIPES = {
    # plain homoscedastic smoother in FP64: 4096 series, one year, scalar lambda
    "homo_fp64": Recipe(seed=20260001, T=365, n_bands=1, d=2, p_valid=0.4,
                        lam_kind="scalar", lam_log10=(0.0, 4.0)),
    # heteroscedastic 10-band tile: 512x512 pixels, 2016-01-01..2024-12-31
    "hetero_tile": Recipe(seed=20260002, T=3288, n_bands=10, d=2, p_valid=0.35,
                          lam_kind="per_day", lam_log10=(1.0, 5.0), lam_window=15),
    # ragged batch: lengths U{120..3288}, orders {1,2,3}
    "ragged": Recipe(seed=20260003, T=3288, n_bands=1, d=0, p_valid=0.4,
                     lam_kind="per_day", lam_log10=(0.0, 5.0)),
    # differentiable layer: 3 years, 4 bands, 20% of valid days held out
    "layer": Recipe(seed=20260004, T=1095, n_bands=4, d=2, p_valid=0.35,
                    lam_kind="per_day", lam_log10=(1.0, 5.0), lam_window=15,
                    holdout_frac=0.2),
    # learned lambda: two years, noise variance switching at random change points
    "learned": Recipe(seed=20260005, T=730, n_bands=1, d=2, p_valid=0.4,
                      noise_var=(0.01, 0.1), lam_kind="per_day", lam_log10=(1.0, 5.0)),
}

RAGGED_T_RANGE = (120, 3288)


def _signal(rc: Recipe, t: torch.Tensor, p: torch.Tensor, b: torch.Tensor, dtype):
    """Clean double-logistic seasonal curve, repeated yearly.

    t: [C,1,1] day, p: [1,1,P] global series id, b: [1,B,1] band.
    Phenology dates are drawn per (series, year) and shared by all bands;
    offset and amplitude are drawn per (series, band)."""
    nb = rc.n_bands
    year = torch.div(t, 365, rounding_mode="floor")
    tau = (t - 365 * year).to(dtype)
    ny = (rc.T + 364) // 365 + 1
    py = p * ny + year                               # [C,1,P]
    sos = 80.0 + 60.0 * uniform(rc.seed, S_SOS, py, dtype)
    eos = 230.0 + 70.0 * uniform(rc.seed, S_EOS, py, dtype)
    r1 = 5.0 + 10.0 * uniform(rc.seed, S_R1, py, dtype)
    r2 = 5.0 + 10.0 * uniform(rc.seed, S_R2, py, dtype)
    pb = p * nb + b                                  # [1,B,P]
    off = 0.2 * uniform(rc.seed, S_OFF, pb, dtype)
    amp = 0.2 + 0.6 * uniform(rc.seed, S_AMP, pb, dtype)
    shape = torch.sigmoid((tau - sos) / r1) - torch.sigmoid((tau - eos) / r2)
    return off + amp * shape                         # [C,B,P]


def _weights(rc: Recipe, t: torch.Tensor, p: torch.Tensor, dtype):
    """0/1 acquisition validity on a revisit grid with a random phase per series."""
    phase = hash_u32(rc.seed, S_PHASE, p) % rc.revisit
    acq = torch.remainder(t - phase, rc.revisit) == 0
    key = p * rc.T + t
    valid = acq & (uniform(rc.seed, S_VALID, key, torch.float32) < rc.p_valid)
    return valid


def _noise_sd(rc: Recipe, t: torch.Tensor, p: torch.Tensor, dtype):
    """Noise standard deviation per (day, series)."""
    if rc.noise_var is None:
        return torch.full((1, 1, 1), rc.noise_sd, dtype=dtype, device=t.device)
    raise RuntimeError("piecewise variance needs the whole series: use generate_tile")


def _lam_raw(rc: Recipe, t: torch.Tensor, p: torch.Tensor, dtype):
    lo, hi = rc.lam_log10
    key = p * (rc.T + 64) + (t + 32)
    u = uniform(rc.seed, S_LAM, key, torch.float64)
    return torch.pow(10.0, lo + (hi - lo) * u).to(dtype)


def _piecewise_sd(rc: Recipe, p: torch.Tensor, T: int, device, dtype):
    """Piecewise-constant noise sd per (day, series): change points arrive as a
    Bernoulli process with mean rate change_rate per series; each segment draws a
    variance U[lo, hi]. Returns [T, 1, P]."""
    t = torch.arange(T, device=device, dtype=torch.int64).view(T, 1)
    key = p.view(1, -1) * T + t
    flip = uniform(rc.seed, S_CHANGE, key, torch.float32) < (rc.change_rate / T)
    flip[0] = False
    seg = torch.cumsum(flip.to(torch.int64), dim=0)          # [T, P]
    lo, hi = rc.noise_var
    var = lo + (hi - lo) * uniform(rc.seed, S_VAR, p.view(1, -1) * 4096 + seg, torch.float64)
    return torch.sqrt(var).to(dtype).view(T, 1, -1)


def generate_tile(rc: Recipe, n_series: int, series0: int = 0, device="cpu",
                  dtype=torch.float32, want_clean: bool = False, chunk_days: int = 128):
    """Dense time-major tile for global series ids series0 .. series0+n_series-1.

    Returns a dict with x [T,B,P], w [T,P], lam [T,P] or [P], and optionally
    clean [T,B,P] (noise-free signal) and holdout [T,P] (bool, held-out valid days
    whose weight was set to 0; x keeps the observation there as the target)."""
    T, B, P = rc.T, rc.n_bands, n_series
    dev = torch.device(device)
    x = torch.empty((T, B, P), dtype=dtype, device=dev)
    w = torch.empty((T, P), dtype=dtype, device=dev)
    clean = torch.empty((T, B, P), dtype=dtype, device=dev) if want_clean else None
    hold = torch.zeros((T, P), dtype=torch.bool, device=dev) if rc.holdout_frac > 0 else None
    p = torch.arange(series0, series0 + P, device=dev, dtype=torch.int64)
    pv = p.view(1, 1, P)
    bv = torch.arange(B, device=dev, dtype=torch.int64).view(1, B, 1)
    sd_full = _piecewise_sd(rc, p, T, dev, dtype) if rc.noise_var is not None else None
    for t0 in range(0, T, chunk_days):
        t1 = min(T, t0 + chunk_days)
        C = t1 - t0
        t = torch.arange(t0, t1, device=dev, dtype=torch.int64).view(C, 1, 1)
        sig = _signal(rc, t, pv, bv, dtype)
        valid = _weights(rc, t, pv, dtype)                        # [C,1,P]
        key_b = ((pv * B + bv) * T + t)                           # [C,B,P]
        sd = sd_full[t0:t1] if sd_full is not None else rc.noise_sd
        obs = sig + sd * normal(rc.seed, S_NOISE_A, S_NOISE_B, key_b, dtype)
        key = pv * T + t
        spike = valid & (uniform(rc.seed, S_SPIKE_DAY, key, torch.float32) < rc.spike_frac)
        lo, hi = rc.spike_mag
        mag = lo + (hi - lo) * uniform(rc.seed, S_SPIKE_MAG, key_b, dtype)
        obs = obs - torch.where(spike, mag, torch.zeros((), dtype=dtype, device=dev))
        wt = valid.to(dtype)
        if hold is not None:
            h = valid & (uniform(rc.seed, S_HOLD, key, torch.float32) < rc.holdout_frac)
            hold[t0:t1] = h.view(C, P)
            wt = torch.where(h, torch.zeros((), dtype=dtype, device=dev), wt)
            keep = valid
        else:
            keep = valid
        x[t0:t1] = torch.where(keep, obs, torch.zeros((), dtype=dtype, device=dev))
        w[t0:t1] = wt.view(C, P)
        if clean is not None:
            clean[t0:t1] = sig
    lam = generate_lambda(rc, n_series, series0, device=dev, dtype=dtype, chunk_days=chunk_days)
    out = {"x": x, "w": w, "lam": lam}
    if clean is not None:
        out["clean"] = clean
    if hold is not None:
        out["holdout"] = hold
    return out


def generate_dates_tile(rc: Recipe, n_series: int, series0: int = 0, device="cpu", dtype=torch.float32,
                        block: int = 16384):
    """The tile of generate_tile kept on each series' acquisition days only (the revisit grid
    from its random phase) instead of the padded daily grid: Ta = (T - revisit) // revisit + 1
    acquisitions per series (every phase has that many inside T days). Returns t [Ta,P]
    (day numbers), x [Ta,B,P], w [Ta,P] (1 on valid acquisitions), lam [Ta,P] (the daily
    field at those days times the revisit: rows 5 days apart stand for 5 daily rows, so the
    smoothing is comparable to the daily grid's) or [P] for scalar recipes. Generated a block
    of series at a time from the daily tile."""
    T, B, P, r = rc.T, rc.n_bands, n_series, rc.revisit
    Ta = (T - r) // r + 1
    dev = torch.device(device)
    t = torch.empty((Ta, P), dtype=dtype, device=dev)
    x = torch.empty((Ta, B, P), dtype=dtype, device=dev)
    w = torch.empty((Ta, P), dtype=dtype, device=dev)
    scalar = rc.lam_kind == "scalar"
    lam = torch.empty((P,) if scalar else (Ta, P), dtype=dtype, device=dev)
    k = torch.arange(Ta, device=dev, dtype=torch.int64).view(Ta, 1)
    for s0 in range(0, P, block):
        n = min(block, P - s0)
        daily = generate_tile(rc, n, series0=series0 + s0, device=dev, dtype=dtype)
        p = torch.arange(series0 + s0, series0 + s0 + n, device=dev, dtype=torch.int64).view(1, n)
        phase = hash_u32(rc.seed, S_PHASE, p) % r
        days = phase + r * k                                   # [Ta, n]
        t[:, s0:s0 + n] = days.to(dtype)
        w[:, s0:s0 + n] = torch.gather(daily["w"], 0, days)
        x[:, :, s0:s0 + n] = torch.gather(daily["x"], 0, days.view(Ta, 1, n).expand(Ta, B, n))
        if scalar:
            lam[s0:s0 + n] = daily["lam"] * r
        else:
            lam[:, s0:s0 + n] = torch.gather(daily["lam"], 0, days) * r
        del daily
    return {"t": t, "x": x, "w": w, "lam": lam}


def generate_lambda(rc: Recipe, n_series: int, series0: int = 0, device="cpu",
                    dtype=torch.float32, chunk_days: int = 128):
    """Per-day lambda [T,P] (entry k weights difference row k) or scalar [P]."""
    dev = torch.device(device)
    P, T = n_series, rc.T
    p = torch.arange(series0, series0 + P, device=dev, dtype=torch.int64)
    if rc.lam_kind == "scalar":
        lo, hi = rc.lam_log10
        u = uniform(rc.seed, S_LAM, p, torch.float64)
        return torch.pow(10.0, lo + (hi - lo) * u).to(dtype)
    lam = torch.empty((T, P), dtype=dtype, device=dev)
    h = rc.lam_window // 2
    for t0 in range(0, T, chunk_days):
        t1 = min(T, t0 + chunk_days)
        a0, a1 = max(0, t0 - h), min(T, t1 + h)
        t = torch.arange(a0, a1, device=dev, dtype=torch.int64).view(-1, 1)
        raw = _lam_raw(rc, t, p.view(1, P), torch.float64)        # [a1-a0, P]
        if h == 0:
            lam[t0:t1] = raw[t0 - a0:t1 - a0].to(dtype)
            continue
        cs = torch.cat([torch.zeros((1, P), dtype=torch.float64, device=dev),
                        torch.cumsum(raw, dim=0)], dim=0)
        tt = torch.arange(t0, t1, device=dev, dtype=torch.int64)
        lo_i = torch.clamp(tt - h, min=0) - a0
        hi_i = torch.clamp(tt + h + 1, max=T) - a0
        s = cs[hi_i] - cs[lo_i]
        cnt = (hi_i - lo_i).to(torch.float64).view(-1, 1)
        lam[t0:t1] = (s / cnt).to(dtype)
    return lam


def ragged_layout(rc: Recipe, n_series: int, device="cpu", t_range=RAGGED_T_RANGE, orders=(1, 2, 3)):
    """Lengths T_i ~ U{t_range}, orders d_i from `orders` in equal shares assigned through
    a shuffled index, and int64 offsets (n_series + 1)."""
    dev = torch.device(device)
    i = torch.arange(n_series, device=dev, dtype=torch.int64)
    lo, hi = t_range
    lengths = lo + (hash_u32(rc.seed, S_LEN, i) % (hi - lo + 1))
    perm_key = hash_u32(rc.seed, S_ORDER, i)
    rank = torch.empty_like(i)
    rank[torch.argsort(perm_key * n_series + i)] = i
    ords = torch.tensor(list(orders), device=dev, dtype=torch.int8)
    order = ords[rank % len(orders)]
    offsets = torch.zeros(n_series + 1, device=dev, dtype=torch.int64)
    offsets[1:] = torch.cumsum(lengths, 0)
    return lengths, order, offsets


def generate_ragged(rc: Recipe, n_series: int, device="cpu", dtype=torch.float32,
                    chunk_elems: int = 1 << 26, t_range=RAGGED_T_RANGE, orders=(1, 2, 3)):
    """Packed ragged batch: series i occupies [off[i], off[i+1]) of x, w, lam."""
    dev = torch.device(device)
    lengths, order, offsets = ragged_layout(rc, n_series, dev, t_range, orders)
    N = int(offsets[-1].item())
    x = torch.empty(N, dtype=dtype, device=dev)
    w = torch.empty(N, dtype=dtype, device=dev)
    lam = torch.empty(N, dtype=dtype, device=dev)
    sid_all = torch.repeat_interleave(torch.arange(n_series, device=dev, dtype=torch.int64), lengths)
    one = replace(rc, n_bands=1)
    for e0 in range(0, N, chunk_elems):
        e1 = min(N, e0 + chunk_elems)
        sid = sid_all[e0:e1]
        t = torch.arange(e0, e1, device=dev, dtype=torch.int64) - offsets[sid]
        tv, pv = t.view(-1, 1, 1), sid.view(-1, 1, 1)
        zero = torch.zeros((1, 1, 1), dtype=torch.int64, device=dev)
        # element-wise: broadcast over a [E,1,1] grid, one band
        sig = _signal(one, tv, pv, zero, dtype).view(-1)
        valid = _weights(one, tv, pv, dtype).view(-1)
        key = (sid * rc.T + t)
        obs = sig + rc.noise_sd * normal(rc.seed, S_NOISE_A, S_NOISE_B, key, dtype)
        spike = valid & (uniform(rc.seed, S_SPIKE_DAY, key, torch.float32) < rc.spike_frac)
        lo, hi = rc.spike_mag
        mag = lo + (hi - lo) * uniform(rc.seed, S_SPIKE_MAG, key, dtype)
        obs = obs - torch.where(spike, mag, torch.zeros((), dtype=dtype, device=dev))
        x[e0:e1] = torch.where(valid, obs, torch.zeros((), dtype=dtype, device=dev))
        w[e0:e1] = valid.to(dtype)
        lam[e0:e1] = _lam_raw(one, t, sid, torch.float64).to(dtype)
    return {"x": x, "w": w, "lam": lam, "offsets": offsets, "order": order, "lengths": lengths}
