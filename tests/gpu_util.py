"""Helpers shared by the GPU tests: seeded inputs generated once and copied to both sides."""
import numpy as np
import torch

from paper_2604_00048_b300 import synth


def tile_inputs(recipe: str, P: int, T=None, B=None, dtype=torch.float32, series0=0, device="cuda", **over):
    rc = synth.RECIPES[recipe]
    kw = dict(rc.__dict__)
    kw.update(over)
    if T is not None:
        kw["T"] = T
    if B is not None:
        kw["n_bands"] = B
    rc = synth.Recipe(**kw)
    out = synth.generate_tile(rc, P, series0=series0, device="cpu", dtype=dtype)
    gpu = {k: v.to(device) for k, v in out.items()}
    cpu = {k: v.double().numpy() if v.is_floating_point() else v.numpy() for k, v in out.items()}
    return rc, gpu, cpu


def rel_err_per_series(a, b):
    """max over (series, band) of ||a - b||_inf(t) / max(||b||_inf(t), 1e-6) for [T, B, P] arrays."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.max(np.abs(a - b), axis=0)
    den = np.maximum(np.max(np.abs(b), axis=0), 1e-6)
    return float(np.max(num / den)) if num.size else 0.0
