#!/usr/bin/env python
"""Throughput of the Whittaker-Henderson hot path on one 512x512-pixel tile.

Workload (synthetic, seeded, generated on the device): 262,144 pixel series, T = 3288
daily steps (2016-01-01 .. 2024-12-31), d = 2, 10 spectral bands sharing the weights
and a per-day lambda = 10^U[1,5] smoothed over 15 days, FP32. One step is the smooth
(Eq. 3, forward and backward sweeps) plus the adjoint (Eqs. 4-5: gradients with
respect to x and log lambda) over the whole tile. Inputs (34.5 GB of x alone) are far
larger than the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank processes its own tile
(different series ids, no collective on the data path): weak scaling, value = the
series of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "series/s fwd and fwd+bwd at T=3288,d=2; HBM roofline %; learned-λ vs GCV time"
FALLBACK_HBM_GBS = 6400.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pixels", type=int, default=262144, help="series per rank (262144 = the full tile)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-sub", type=int, default=16, help="sub-blocks of the end-to-end block")
    ap.add_argument("--e2e-streams", type=int, default=3, help="streams the end-to-end sub-blocks rotate over")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ragged-no-autotune", action="store_true",
                    help="ragged: keep the default configuration with the length-class tiles (profiling)")
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-gcv", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-posterior", action="store_true")
    ap.add_argument("--no-wgrad", action="store_true")
    ap.add_argument("--no-dates", action="store_true")
    ap.add_argument("--no-partitioned", action="store_true")
    ap.add_argument("--no-layer", action="store_true")
    ap.add_argument("--no-homo", action="store_true")
    ap.add_argument("--tcn-ckpt", default=None, help="trained lambda network (else one epoch is trained first)")
    ap.add_argument("--train-epochs", type=float, default=1.0, help="epochs of lambda-network training before timing")
    ap.add_argument("--only", choices=["gcv", "learned", "ragged", "posterior", "dates", "partitioned", "layer", "homo"],
                    default=None,
                    help="run one secondary measurement alone (profiling) and print it")
    ap.add_argument("--series", type=int, default=None, help="series of the --only measurement")
    ap.add_argument("--days", type=int, default=None, help="days of the --only posterior measurement (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle baseline")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# sources the tile kernels (smooth, refine, adjoint) are built from
TILE_SOURCES = ["ws_df.cuh", "ws_internal.h", "ws_ptx.cuh", "ws_sweep.cuh", "ws_tile.cu", "ws_tile_d1.cu",
                "ws_tile_d2.cu", "ws_tile_d3.cu", "ws_tile_d4.cu", "ws_tile_impl.cuh"]


def kernel_sources_sha(names=TILE_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_00048_b300", "csrc")
    for name in sorted(names):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str):
    """DRAM bytes per launch recorded by an ncu capture summary under profiles/, or None
    when the summary is missing or was taken on different kernel sources."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    want = kernel_sources_sha()
    for name in sorted(os.listdir(pdir)):
        if not name.endswith(".md") or not name.startswith(kernel):
            continue
        txt = open(os.path.join(pdir, name)).read()
        m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
        s = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
        if m and s and s.group(1) == want:
            return float(m.group(1))
    return None


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4) if r[4 + i] == "Active"})
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": reasons, "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def tile_config(P, T, B, d, world, has_bwd=True):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": f"hetero_tile: {P} px x {T} d x {B} bands, d={d}, per-day lambda, "
                        + ("smooth + refinement step + adjoint" if has_bwd else "smooth + refinement step"),
            "pixels_per_rank": P, "T": T, "bands": B, "d": d,
            "parallelism": f"replicas x{world} (pixel shards, no collective)",
            "l2": "inputs larger than L2 (34.5 GB of x per rank), no flush"}


def rank_series0(rank: int, per_rank: int) -> int:
    """First series id of a rank's shard: ranks process disjoint, consecutive id ranges."""
    return rank * per_rank


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time (all ranks take part; identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def pinned_copy_gbs(dev, nbytes=1 << 30, reps=5):
    """Plain pinned host <-> device copy bandwidth (GB/s): host-to-device alone,
    device-to-host alone, and both directions at once on two streams (the link's
    full-duplex rate), best of `reps`: the denominator of the end-to-end copies."""
    import torch

    h1 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d1 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def best(fn):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    def h2d():
        with torch.cuda.stream(s1):
            d1.copy_(h1, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    def both():
        h2d()
        d2h()

    t_h, t_d, t_b = best(h2d), best(d2h), best(both)
    del h1, h2, d1, d2
    return {"h2d_gbs": nbytes / t_h / 1e9, "d2h_gbs": nbytes / t_d / 1e9, "bidirectional_gbs": 2 * nbytes / t_b / 1e9,
            "bytes": nbytes}


def aggregate_rate(per_rank: int, world: int, steps: int, ms: float) -> float:
    """Whole-job throughput: the series of all ranks over the slowest rank's time."""
    return per_rank * world * steps / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e nominal bandwidth (context beside the measured peak)
CPU_SAMPLE = 512  # series of the oracle's timed sample, the same in both arms


def cpu_oracle_runs(x, w, lam, gz, d, runs, warmup=1, with_bwd=True):
    """Banded FP64 oracle (Algorithm 1, OpenMP over pixels) on one contiguous sample of
    series (tile layout [T][B][n], the same arrays in both arms of the bench): `warmup`
    untimed runs, then `runs` timed runs of smooth (+ adjoint). Returns the run times (s)."""
    from oracle import banded

    times = []
    for i in range(warmup + runs):
        t0 = time.perf_counter()
        z, _ = banded.smooth_tile(x, w, lam, d)
        if with_bwd:
            banded.vjp_tile(w, lam, d, z, gz, log_lambda=True)
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    return times


def cpu_oracle_rate(x, w, lam, gz, d, target_s, with_bwd=True):
    """The oracle's rate on the first CPU_SAMPLE series (contiguous copies), repeated until
    about target_s seconds of timed work: returns (series/s, cores, sample description)."""
    import numpy as np

    from oracle import banded

    cores = banded.max_threads()
    n = min(x.shape[2], CPU_SAMPLE)
    xs, wsn, ls, gs = (np.ascontiguousarray(a[..., :n]) for a in (x, w, lam, gz))
    t1 = cpu_oracle_runs(xs, wsn, ls, gs, d, 1, warmup=1, with_bwd=with_bwd)[0]
    runs = int(max(1, min(20, target_s / max(t1, 1e-3))))
    times = cpu_oracle_runs(xs, wsn, ls, gs, d, runs, warmup=0, with_bwd=with_bwd)
    return n * len(times) / sum(times), cores, (
        f"{n} of the tile's series (all {x.shape[0]} days, {x.shape[1]} bands, contiguous), FP64, "
        f"{len(times)} timed runs after one warm-up")


def ragged_measure(dev, steps, n=1 << 20, autotune=True):
    """The ragged batch: 1,048,576 series, T ~ U{120..3288}, d in {1,2,3}, one band, FP32,
    one persistent launch replayed from a CUDA graph with the autotuned configuration."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, n, device=dev)
    x, w, lam = out["x"], out["w"], out["lam"]
    N = x.numel()
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z = torch.empty_like(x)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    plan.execute(x, w, lam, z=z, status=st, autotune=autotune, graph=True, tiles=True)  # tiles kept only if faster

    def timed(refine, tiles=True):
        for _ in range(2):
            plan.execute(x, w, lam, z=z, status=st, graph=True, refine=refine, tiles=tiles)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.execute(x, w, lam, z=z, status=st, graph=True, refine=refine, tiles=tiles)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_lanes = timed(False, tiles=False)  # every series on the per-lane kernel
    ms_solve = timed(False)  # length-class tiles (+ short series per lane)
    ms = timed(True)  # the accuracy-gated result: refinement + double-float re-solve of unsettled series
    hbm, _ = peaks()
    alg = 16.0 * N  # read x, w, lambda; write z (FP32), once
    info = plan.info()
    res = {"workload": f"ragged: {n} series, T~U{{120..3288}}, d in {{1,2,3}}, 1 band, FP32 + refinement",
           "series_per_s": n / (ms / 1e3), "ms": ms, "pixel_days": N,
           "solve_only_ms": ms_solve, "solve_only_series_per_s": n / (ms_solve / 1e3),
           "solve_per_lane_kernel_ms": ms_lanes,
           "solve_only_alg_gbs": alg / (ms_solve / 1e3) / 1e9,
           "frac_of_measured_hbm_solve_only": alg / (ms_solve / 1e3) / 1e9 / hbm,
           "hp_resolved_series": info["hp_series"],
           "plan": {k: info[k] for k in ("n_items", "chunk_days", "warps_per_cta", "grid", "graph", "tiles")},
           "series_with_status": int((st != 0).sum().item())}
    del out, x, w, lam, z, plan
    torch.cuda.empty_cache()
    return res


def gcv_measure(dev, steps, P=262144):
    """GCV grid search (16 lambda values, log10 in {0, 1/3, ..., 5}) then the smoothing at the
    chosen lambda, on the learned-lambda evaluation set: 262,144 series x 730 days, d = 2,
    one band, FP32."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    T = 730
    out = synth.generate_tile(synth.RECIPES["learned"], P, device=dev)
    x, w = out["x"], out["w"]
    ws.gcv_smooth(x, w, None, 2, refine=True, want_scores=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        z, lam_best, _, st = ws.gcv_smooth(x, w, None, 2, refine=True, want_scores=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    hbm, _ = peaks()
    res = {"workload": f"gcv: {P} series x {T} days, d=2, 1 band, FP32, 16-value grid, then the smooth "
                       "with its refinement step",
           "series_per_s": P / (ms / 1e3), "ms": ms,
           "lambda_evals_per_s": 16 * P / (ms / 1e3),
           "series_with_status": int((st != 0).sum().item())}
    del out, x, w, z, lam_best, st
    torch.cuda.empty_cache()
    return res


def wgrad_measure(dev, steps, x, w, lam, z, gz, gx, glam):
    """Gradient with respect to the weights on the heteroscedastic tile: the adjoint with the
    raw-g flag, then ws_weight_grad (dL/dw and gx = W g in one streaming pass). Times the
    two C-ABI calls separately; algorithmic bytes of the weight-gradient pass per pixel-day:
    read g, x, z (B each) and w, write gx (B) and gw: 4 (4B + 2)."""
    import ctypes

    import torch

    from paper_2604_00048_b300 import ws

    T, B, P = x.shape
    gw = torch.empty_like(w)
    pb = ws.make_problem(T, B, P, 2, ws.F32, ws.LAM_PER_DAY)
    stream = torch.cuda.Stream(device=dev)

    def run(ev=None):
        if ev is not None:
            ev[0].record(stream)
        ws.smooth_adjoint(w, lam, z, gz, 2, gx=gx, glam=glam, log_lambda=True, stream=stream, _raw_g=True)
        if ev is not None:
            ev[1].record(stream)
        ws._check(ws.lib().ws_weight_grad(ctypes.byref(pb), ws._ptr(x), ws._ptr(w), ws._ptr(z), ws._ptr(gx),
                                          ws._ptr(gx), ws._ptr(gw), ws._stream_ptr(stream)))
        if ev is not None:
            ev[2].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(2):
            run()
    torch.cuda.synchronize()
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            run(e)
            evs.append(e)
    torch.cuda.synchronize()
    adj = statistics.median([e[0].elapsed_time(e[1]) for e in evs])
    wg = statistics.median([e[1].elapsed_time(e[2]) for e in evs])
    hbm, _ = peaks()
    byts = 4.0 * (4 * B + 2) * float(P) * T
    del gw
    return {"workload": f"weight gradient: {P} series x {T} days x {B} bands, d=2, FP32 (adjoint with raw g, "
                        "then dL/dw and gx = W g)",
            "adjoint_raw_g_ms": adj, "weight_grad_ms": wg, "series_per_s": P / ((adj + wg) / 1e3),
            "weight_grad_achieved_gbs": byts / (wg / 1e3) / 1e9,
            "weight_grad_frac_of_measured_hbm": byts / (wg / 1e3) / 1e9 / hbm}


def dates_measure(dev, steps, P=262144):
    """Smoothing on acquisition dates (ws_smooth_dates): the heteroscedastic tile kept on each
    series' 657 acquisition days of 3288 (5-day revisit) instead of the daily grid, 10 bands,
    d = 2, FP32. Algorithmic bytes per series-acquisition: read x (B), w, lambda, t; write z
    (B): 4 (2B + 3)."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["hetero_tile"]
    out = synth.generate_dates_tile(rc, P, device=dev)
    t, x, w, lam = out["t"], out["x"], out["w"], out["lam"]
    del out
    z = torch.empty_like(x)
    st = torch.empty(P, dtype=torch.uint8, device=dev)
    for _ in range(3):
        ws.smooth_dates(t, x, w, lam, rc.d, z=z, status=st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ws.smooth_dates(t, x, w, lam, rc.d, z=z, status=st)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    e0.record()
    for _ in range(steps):
        ws.smooth_dates(t, x, w, lam, rc.d, z=z, status=st, refine=True)
    e1.record()
    torch.cuda.synchronize()
    ms_ref = e0.elapsed_time(e1) / steps
    # the adjoint on the same dates (gx and dL/dlog lambda)
    gz = torch.randn(x.shape, generator=torch.Generator(device=dev).manual_seed(5), device=dev)
    gx, glam = torch.empty_like(x), torch.empty_like(lam)
    for _ in range(2):
        ws.smooth_dates_adjoint(t, w, lam, z, gz, rc.d, gx=gx, glam=glam, log_lambda=True, status=st)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        ws.smooth_dates_adjoint(t, w, lam, z, gz, rc.d, gx=gx, glam=glam, log_lambda=True, status=st)
    e1.record()
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / steps
    # the posterior spread and the GCV search (band 0) on the same dates
    outs = (torch.empty(x.shape[0], P, device=dev), torch.empty(x.shape[1], P, device=dev), torch.empty_like(x),
            torch.empty(P, dtype=torch.uint8, device=dev))
    x0 = x[:, :1, :].contiguous()
    ws.posterior(x, w, lam, z, rc.d, out=outs, t=t)
    ws.gcv_smooth(x0, w, None, rc.d, refine=True, want_scores=False, t=t)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        ws.posterior(x, w, lam, z, rc.d, out=outs, t=t)
    e1.record()
    torch.cuda.synchronize()
    ms_post = e0.elapsed_time(e1) / steps
    e0.record()
    for _ in range(steps):
        ws.gcv_smooth(x0, w, None, rc.d, refine=True, want_scores=False, t=t)
    e1.record()
    torch.cuda.synchronize()
    ms_gcv = e0.elapsed_time(e1) / steps
    del outs, x0
    Ta, B, _ = x.shape
    hbm, _ = peaks()
    byts = 4.0 * (2 * B + 3) * float(P) * Ta
    byts_adj = 4.0 * (3 * B + 4) * float(P) * Ta  # read gz, z, w, lambda, t; write gx, glam
    res = {"workload": f"dates: {P} series x {Ta} acquisition dates (5-day revisit over {rc.T} days) x {B} bands, "
                       f"d={rc.d}, FP32",
           "ms": ms, "series_per_s": P / (ms / 1e3), "achieved_gbs": byts / (ms / 1e3) / 1e9,
           "frac_of_measured_hbm": byts / (ms / 1e3) / 1e9 / hbm,
           "refined_ms": ms_ref, "adjoint_ms": ms_adj, "adjoint_achieved_gbs": byts_adj / (ms_adj / 1e3) / 1e9,
           "posterior_ms": ms_post, "gcv_band0_ms": ms_gcv,
           "series_with_status": int((st != 0).sum().item())}
    del t, x, w, lam, z, st, gz, gx, glam
    torch.cuda.empty_cache()
    return res


def posterior_measure(dev, steps, x=None, w=None, lam=None, z=None, P=262144, T=None):
    """Posterior spread (ws_posterior: diag(Omega^{-1}), sigma2 per band, sd) on the
    heteroscedastic tile (the smooth z given; generated and smoothed here when absent).
    Algorithmic bytes per pixel-day: read x, z (B bands each), w, lambda; write diag and sd
    (B): 4 (3B + 3)."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["hetero_tile"]
    if T is not None:
        rc = synth.Recipe(**{**rc.__dict__, "T": T})
    if x is None:
        out = synth.generate_tile(rc, P, device=dev)
        x, w, lam = out["x"], out["w"], out["lam"]
        del out
        z, _ = ws.smooth(x, w, lam, rc.d, refine=True)
    T, B, P = x.shape
    outs = (torch.empty(T, P, device=dev), torch.empty(B, P, device=dev), torch.empty_like(x),
            torch.empty(P, dtype=torch.uint8, device=dev))
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for _ in range(3):
            ws.posterior(x, w, lam, z, rc.d, out=outs, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            ws.posterior(x, w, lam, z, rc.d, out=outs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    hbm, _ = peaks()
    byts = 4.0 * (3 * B + 3) * float(P) * T
    res = {"workload": f"posterior: {P} series x {T} days x {B} bands, d={rc.d}, FP32 (diag of Omega^-1, "
                       "sigma2 per band, sd)",
           "ms": ms, "series_per_s": P / (ms / 1e3), "algorithmic_bytes": byts,
           "achieved_gbs": byts / (ms / 1e3) / 1e9, "frac_of_measured_hbm": byts / (ms / 1e3) / 1e9 / hbm,
           "series_with_status": int((outs[3] != 0).sum().item()), "launches_per_call": 2}
    del outs
    return res


def homo_measure(dev, steps, P=4096):
    """The plain homoscedastic smoother in FP64 (4,096 series x 365 days, one band, scalar
    lambda): a launch-bound size, timed as replays of a CUDA graph holding the C-ABI call."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["homo_fp64"]
    out = synth.generate_tile(rc, P, device=dev, dtype=torch.float64)
    x, w, lam = out["x"], out["w"], out["lam"]
    z = torch.empty_like(x)
    st = torch.empty(P, dtype=torch.uint8, device=dev)
    pb = ws.make_problem(rc.T, 1, P, rc.d, ws.F64, ws.LAM_SCALAR)
    wsb = torch.zeros(ws.workspace_size(pb, 0), dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        for _ in range(3):
            ws.smooth(x, w, lam, rc.d, z=z, status=st, workspace_buf=wsb, stream=s)
    torch.cuda.synchronize()
    reps = max(50, 10 * steps)

    def graph_ms(call):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
                call()
        for _ in range(5):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = graph_ms(lambda: ws.smooth(x, w, lam, rc.d, z=z, status=st, workspace_buf=wsb, stream=s))
    bad = int((st != 0).sum().item())
    wsp = torch.zeros(ws.workspace_size(pb, ws.PARTITIONED), dtype=torch.uint8, device=dev)
    zp = torch.empty_like(x)
    with torch.cuda.stream(s):
        ws.smooth_partitioned(x, w, lam, rc.d, z=zp, status=st, workspace_buf=wsp, stream=s)
    torch.cuda.synchronize()
    ms_p = graph_ms(lambda: ws.smooth_partitioned(x, w, lam, rc.d, z=zp, status=st, workspace_buf=wsp, stream=s))
    rel = float(((zp - z).abs().amax(dim=0) / z.abs().amax(dim=0).clamp_min(1e-12)).max())
    return {"workload": f"homo_fp64: {P} series x {rc.T} days, d={rc.d}, 1 band, FP64, scalar lambda",
            "ms": ms, "series_per_s": P / (ms / 1e3), "replays": reps, "series_with_status": bad,
            "partitioned_ms": ms_p, "partitioned_series_per_s": P / (ms_p / 1e3),
            "partitioned_max_rel_diff": rel,
            "note": "CUDA-graph replays of one C-ABI call (tile path: one series per thread, 32 CTAs)"}


def layer_measure(dev, steps, P=65536):
    """The differentiable layer (65,536 series x 1095 days x 4 bands, d = 2, FP32; loss = the
    mean squared error of z against the 20% held-out valid observations): forward + backward
    through the autograd layer in recompute and store-factor modes (gradients to x and
    log lambda; the loss in PyTorch), and the C-ABI path with the loss fused into the adjoint
    (ws_smooth_batch with refinement + ws_solve_adjoint_mse)."""
    import torch

    from paper_2604_00048_b300 import autograd, synth, ws

    rc = synth.RECIPES["layer"]
    out = synth.generate_tile(rc, P, device=dev)
    x, w, lam, mask = out["x"], out["w"], out["lam"], out["holdout"].to(torch.float32)
    del out
    scale = 2.0 / float(mask.sum() * rc.n_bands)
    loglam = lam.log()

    def autograd_step(store):
        xg = x.clone().requires_grad_(True)
        ll = loglam.clone().requires_grad_(True)
        z, _ = autograd.whittaker_smooth(xg, w, ll.exp(), rc.d, refine=True, store_factor=store)
        loss = 0.5 * scale * (mask[:, None, :] * (z - x) ** 2).sum()
        loss.backward()
        return xg.grad, ll.grad

    z = torch.empty_like(x)
    st = torch.empty(P, dtype=torch.uint8, device=dev)
    gx, glam, lossp = torch.empty_like(x), torch.empty_like(lam), torch.empty(P, device=dev)

    def fused_step():
        ws.smooth(x, w, lam, rc.d, z=z, status=st, refine=True)
        ws.smooth_adjoint_mse(w, lam, z, x, rc.d, mask=mask, scale=scale, gx=gx, glam=glam, loss=lossp,
                              log_lambda=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    ms_re = timed(lambda: autograd_step(False))
    ms_st = timed(lambda: autograd_step(True))
    ms_fu = timed(fused_step)
    ws.sync_status(dev)
    return {"workload": f"layer: {P} series x {rc.T} days x {rc.n_bands} bands, d={rc.d}, FP32, held-out MSE loss, "
                        "gradients to x and log lambda",
            "autograd_recompute_ms": ms_re, "autograd_store_factor_ms": ms_st,
            "fused_loss_cabi_ms": ms_fu, "series_per_s_fused": P / (ms_fu / 1e3),
            "stored_factor_bytes": (rc.d + 1) * rc.T * P * 4,
            "note": "autograd rows include PyTorch's loss and exp ops; the fused row is two C-ABI calls"}


def partitioned_measure(dev, steps, P=64):
    """Few long series: P series of the heteroscedastic tile (3288 days, 10 bands, d = 2)
    smoothed by the partitioned parallel-in-time solve (double-float, no refinement step
    needed) against the one-series-per-thread tile path with its refinement step (the
    FP32 path's accuracy contract at lambda up to 1e5); both timed with CUDA events."""
    import torch

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["hetero_tile"]
    out = synth.generate_tile(rc, P, device=dev)
    x, w, lam = out["x"], out["w"], out["lam"]
    z = torch.empty_like(x)
    st = torch.empty(P, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(5, steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), min(ts)

    ms_p, best_p = timed(lambda: ws.smooth_partitioned(x, w, lam, rc.d, z=z, status=st, stream=stream))
    zp = z.clone()
    ms_t, best_t = timed(lambda: ws.smooth(x, w, lam, rc.d, z=z, status=st, refine=True, stream=stream))
    ws.sync_status(dev, stream)
    rel = float(((zp - z).abs().amax(dim=0) / z.abs().amax(dim=0).clamp_min(1e-6)).max())
    return {"workload": f"partitioned: {P} series x {rc.T} days x {rc.n_bands} bands, d={rc.d}, FP32 in/out",
            "partitioned_ms": ms_p, "partitioned_best_ms": best_p, "tile_refined_ms": ms_t,
            "tile_refined_best_ms": best_t, "speedup_vs_tile": ms_t / ms_p,
            "max_rel_diff_vs_tile": rel, "series_with_status": int((st != 0).sum().item())}


def learned_measure(dev, steps, ckpt=None, train_epochs=1.0, P=262144):
    """Learned lambda vs the GCV grid on the evaluation set (262,144 new series x 730 days,
    d = 2, one band): the lambda network is trained first on the project's kernels (one
    epoch of 2,097,152 series in batches of 4096) unless a checkpoint is given. Timed: the
    network's forward plus the smoothing at its per-day lambda, against ws_gcv_smooth."""
    import math

    import torch

    from paper_2604_00048_b300 import synth, train, ws

    t0 = time.time()
    if ckpt:
        net, _ = train.load_checkpoint(ckpt, device=dev)
        trained = {"checkpoint": os.path.basename(ckpt)}
    else:
        net, nb, hist = train.train(2097152, 4096, train_epochs, 2e-3, seed=0, log_every=10 ** 9, device=dev)
        torch.cuda.synchronize()
        trained = {"batches": nb, "batch": 4096, "epochs": train_epochs, "train_s": time.time() - t0}
    T = 730
    base = synth.RECIPES["learned"]
    rc = synth.Recipe(**{**base.__dict__, "seed": base.seed + 1000, "T": T})
    out = synth.generate_tile(rc, P, device=dev, want_clean=True)
    x, w, clean = out["x"], out["w"], out["clean"][:, 0, :].contiguous()
    del out

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, r

    ms_l, (zl, lam, _) = timed(lambda: train.learned_smooth(net, x, w, refine=True))
    ms_tcn, _ = timed(lambda: net.forward(x[:, 0, :], w, want_loglam=False))
    ms_g, (zg, _, _, _) = timed(lambda: ws.gcv_smooth(x, w, None, 2, refine=True, want_scores=False))
    rl, rg = train.rmse(zl, clean), train.rmse(zg, clean)
    flop = 150912.0 * P * T  # network multiply-adds x 2 per position
    res = {"workload": f"learned lambda vs GCV: {P} new series x {T} days, d=2, 1 band (both smooths refined)",
           "learned_ms": ms_l, "tcn_forward_ms": ms_tcn, "gcv_ms": ms_g,
           "learned_series_per_s": P / (ms_l / 1e3), "gcv_series_per_s": P / (ms_g / 1e3),
           "learned_faster_than_gcv": ms_l < ms_g,
           "tcn_tflops": flop / (ms_tcn / 1e3) / 1e12,
           "rmse_learned": rl, "rmse_gcv": rg, "rmse_ratio": rl / rg, "training": trained}
    del x, w, clean, zl, zg, lam
    torch.cuda.empty_cache()
    return res


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, timed on this host's cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import torch

    from paper_2604_00048_b300 import synth

    rc = synth.RECIPES["hetero_tile"]
    n = CPU_SAMPLE
    inp = synth.generate_tile(rc, n, device="cpu", dtype=torch.float32)
    x, w, lam = (np.ascontiguousarray(inp[k].double().numpy()) for k in ("x", "w", "lam"))
    gz = np.random.default_rng(7).normal(size=x.shape)
    from oracle import banded

    times = cpu_oracle_runs(x, w, lam, gz, rc.d, args.steps, warmup=args.warmup)
    dt = sum(times)
    val = n * len(times) / dt
    cores = banded.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "series/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": tile_config(262144, 3288, 10, 2, 1),
            "sample": {"series_per_step": n, "parallelism": "host cores",
                       "note": "FP64 banded oracle: smooth + adjoint (FP64 needs no refinement step)"},
            "cpu_baseline": {"value": val, "unit": "series/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} series per step of the tile (3288 days, 10 bands), FP64 banded oracle"},
            "e2e": {"value": val, "unit": "series/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_only(args):
    """One secondary measurement alone (used by the profiling commands)."""
    import torch

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    steps = max(1, args.steps)
    if args.only == "gcv":
        res = gcv_measure(dev, steps, args.series or 262144)
    elif args.only == "dates":
        res = dates_measure(dev, steps, P=args.series or 262144)
    elif args.only == "posterior":
        res = posterior_measure(dev, steps, P=args.series or 262144, T=args.days)
    elif args.only == "learned":
        res = learned_measure(dev, steps, args.tcn_ckpt, args.train_epochs, args.series or 262144)
    elif args.only == "partitioned":
        res = partitioned_measure(dev, steps, args.series or 64)
    elif args.only == "layer":
        res = layer_measure(dev, steps, args.series or 65536)
    elif args.only == "homo":
        res = homo_measure(dev, steps, args.series or 4096)
    else:
        res = ragged_measure(dev, steps, args.series or (1 << 20), autotune=not args.ragged_no_autotune)
    print(json.dumps({"only": args.only, **res}), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    if args.only:
        return run_only(args)
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    from paper_2604_00048_b300 import synth, ws

    rc = synth.RECIPES["hetero_tile"]
    P, T, B, d = args.pixels, rc.T, rc.n_bands, rc.d
    series0 = rank_series0(rank, P)
    inp = synth.generate_tile(rc, P, series0=series0, device=dev, dtype=torch.float32)
    x, w, lam = inp["x"], inp["w"], inp["lam"]
    del inp
    gen = torch.Generator(device=dev)
    gen.manual_seed(20260102 + rank)
    z = torch.empty_like(x)
    status = torch.empty(P, dtype=torch.uint8, device=dev)
    has_bwd = hasattr(ws, "smooth_adjoint")
    if has_bwd:
        gz = torch.randn(x.shape, generator=gen, device=dev, dtype=torch.float32)
        gx = torch.empty_like(x)
        glam = torch.empty_like(lam)
    stream = torch.cuda.Stream(device=dev)
    ev = []

    def step(record):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        ws.smooth(x, w, lam, d, z=z, status=status, stream=stream)           # 1 tile kernel
        e[1].record(stream)
        ws.refine(x, w, lam, z, d, stream=stream)                            # residual + tile kernel
        e[2].record(stream)
        if has_bwd:
            ws.smooth_adjoint(w, lam, z, gz, d, gx=gx, glam=glam, log_lambda=True, stream=stream)  # 1 tile kernel
        e[3].record(stream)
        if record:
            ev.append(e)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False)
    torch.cuda.synchronize()
    ws.sync_status(dev, stream)
    bad = int((status != 0).sum().item())

    gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
    clocks = ClockSampler(gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}")
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    ws.sync_status(dev, stream)
    ms = max_over_ranks(ms, dev)
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    fwd_ms = statistics.median([e[0].elapsed_time(e[1]) for e in ev])
    ref_ms = statistics.median([e[1].elapsed_time(e[2]) for e in ev])
    bwd_ms = statistics.median([e[2].elapsed_time(e[3]) for e in ev]) if has_bwd else 0.0
    ms_step = ms / args.steps
    value = aggregate_rate(P, world, args.steps, ms)

    # roofline of the dominant kernel: algorithmic bytes per pixel-day, FP32
    pd = float(P) * T
    fwd_bytes = 4.0 * (2 * B + 2) * pd          # read x (B), w, lambda; write z (B)
    bwd_bytes = 4.0 * (3 * B + 3) * pd          # read gz, z (2B), w, lambda; write gx (B), glam
    hbm, peak_kind = peaks()
    if has_bwd and bwd_ms > fwd_ms:
        kname, kms, kbytes = "adjoint_tile", bwd_ms, bwd_bytes
    else:
        kname, kms, kbytes = "smooth_tile", fwd_ms, fwd_bytes
    achieved = kbytes / (kms / 1e3) / 1e9
    traffic = traffic_from_profile(kname)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback", "traffic": traffic,
            "algorithmic_bytes_per_launch": kbytes, "kernel_ms": kms,
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS}

    # end to end through the C-ABI with host buffers (pinned), on a block of the tile: the
    # block is streamed as sub-blocks of series over three streams (each with its own device
    # buffers and workspace), so host-to-device copies, the solves and device-to-host copies
    # of different sub-blocks overlap (PCIe is full duplex)
    e2e = None
    if not args.no_e2e:
        Pe, nsub, nstr = min(P, 32768), args.e2e_sub, args.e2e_streams
        Ps = Pe // nsub
        host = []
        for k in range(nsub):
            sl = slice(k * Ps, (k + 1) * Ps)
            hb = {"x": x[:, :, sl].contiguous().cpu().pin_memory(), "w": w[:, sl].contiguous().cpu().pin_memory(),
                  "l": lam[:, sl].contiguous().cpu().pin_memory()}
            hb["z"] = torch.empty_like(hb["x"]).pin_memory()
            if has_bwd:
                hb["g"] = gz[:, :, sl].contiguous().cpu().pin_memory()
                hb["gx"] = torch.empty_like(hb["x"]).pin_memory()
                hb["gl"] = torch.empty_like(hb["l"]).pin_memory()
            host.append(hb)
        streams = [torch.cuda.Stream(device=dev) for _ in range(nstr)]
        devb = []
        for k in range(nstr):
            db = {n: torch.empty_like(t, device=dev) for n, t in host[0].items()}
            db["st"] = torch.empty(Ps, dtype=torch.uint8, device=dev)
            pb = ws.make_problem(T, B, Ps, d, ws.F32, ws.LAM_PER_DAY)
            need = max(ws.workspace_size(pb, ws.REFINE), ws.workspace_size(pb, ws.GRAD_LOGLAM))
            db["ws"] = torch.zeros(need, dtype=torch.uint8, device=dev)
            devb.append(db)

        def e2e_step():
            for k in range(nsub):
                s_k, db, hb = streams[k % nstr], devb[k % nstr], host[k]
                with torch.cuda.stream(s_k):
                    for n in ("x", "w", "l") + (("g",) if has_bwd else ()):
                        db[n].copy_(hb[n], non_blocking=True)
                    ws.smooth(db["x"], db["w"], db["l"], d, z=db["z"], status=db["st"], refine=True, stream=s_k,
                              workspace_buf=db["ws"])
                    if has_bwd:
                        ws.smooth_adjoint(db["w"], db["l"], db["z"], db["g"], d, gx=db["gx"], glam=db["gl"],
                                          log_lambda=True, stream=s_k, workspace_buf=db["ws"])
                        hb["gx"].copy_(db["gx"], non_blocking=True)
                        hb["gl"].copy_(db["gl"], non_blocking=True)
                    hb["z"].copy_(db["z"], non_blocking=True)
            for s_k in streams:
                s_k.synchronize()

        e2e_step()
        ke = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        dt = time.perf_counter() - t0
        h2d = sum(hb[n].numel() * 4 for hb in host for n in ("x", "w", "l") + (("g",) if has_bwd else ()))
        d2h = sum(hb[n].numel() * 4 for hb in host for n in ("z",) + (("gx", "gl") if has_bwd else ()))
        link = pinned_copy_gbs(dev)
        moved = (h2d + d2h) * ke / dt / 1e9
        e2e = {"value": Pe * world * ke / dt, "unit": "series/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "series_per_step": Pe,
               "note": "pinned host buffers, copies + C-ABI calls + sync inside the timed region, "
                       f"{Pe}-series block of the tile in {nsub} sub-blocks over {nstr} streams",
               "host_link": {**link, "e2e_copy_gbs": moved,
                             "frac_of_bidirectional_copy": moved / link["bidirectional_gbs"]}}
        del host, devb

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ns = CPU_SAMPLE
        xs = x[:, :, :ns].double().cpu().numpy()
        wsn = w[:, :ns].double().cpu().numpy()
        ls = lam[:, :ns].double().cpu().numpy()
        gs = gz[:, :, :ns].double().cpu().numpy() if has_bwd else np.zeros_like(xs)
        rate, cores, sample = cpu_oracle_rate(xs, wsn, ls, gs, d, args.cpu_seconds, with_bwd=has_bwd)
        cpu = {"value": rate, "unit": "series/s", "cores": cores, "kind": "oracle", "sample": sample}

    launches_per_step = 3 + (1 if has_bwd else 0)
    wgrad = None
    if has_bwd and not args.no_wgrad:
        wgrad = wgrad_measure(dev, max(3, args.steps), x, w, lam, z, gz, gx, glam)
    if has_bwd:
        del gz, gx, glam
    ws._ws_cache.clear()
    torch.cuda.empty_cache()
    posterior = None if args.no_posterior else posterior_measure(dev, max(3, args.steps), x, w, lam, z)
    ragged = None
    if not args.no_ragged:
        del x, w, lam, z, status
        ws._ws_cache.clear()
        torch.cuda.empty_cache()
        ragged = ragged_measure(dev, max(3, args.steps))
    dates = None if args.no_dates else dates_measure(dev, max(3, args.steps))
    gcv = None if args.no_gcv else gcv_measure(dev, max(3, args.steps))
    learned = None if args.no_learned else learned_measure(dev, max(3, args.steps), args.tcn_ckpt, args.train_epochs)
    partitioned = None if args.no_partitioned else partitioned_measure(dev, max(5, args.steps))
    layer = None if args.no_layer else layer_measure(dev, max(5, args.steps))
    homo = None if args.no_homo else homo_measure(dev, max(5, args.steps))
    line = {"metric": METRIC, "value": value, "unit": "series/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": tile_config(P, T, B, d, world, has_bwd),
            "fwd_series_per_s": P * world / ((fwd_ms + ref_ms) / 1e3),
            "fwd_unrefined_series_per_s": P * world / (fwd_ms / 1e3),
            "smooth_ms": fwd_ms, "refine_ms": ref_ms, "adjoint_ms": bwd_ms,
            "step_ms_median": statistics.median(step_ms), "step_ms_best": min(step_ms),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "ragged": ragged, "gcv": gcv, "learned": learned,
            "posterior": posterior, "weight_grad": wgrad, "dates": dates, "partitioned": partitioned,
            "layer": layer, "homo_fp64": homo,
            "gpu_launches": launches_per_step * args.steps, "clocks": ck,
            "series_with_status": bad}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
