"""The smoother as a differentiable layer (Section 2.3): z = f(x, lambda | W, D).

Forward: the CUDA smooth (with one refinement step by default). Backward: the CUDA adjoint
(Eqs. 4-5): dL/dx = W Omega^{-1} dL/dz and dL/dlambda_k = -sum_b (D g_b)_k (D z_b)_k.
`store_factor=True` keeps the factor of Omega from the forward pass ((d+1) words per
pixel-day) and reuses it in the backward pass, which saves the backward pass's rotation
arithmetic (not time: its kernels stream one series per thread without staging and measured
slower than the recompute on the three-year 4-band layer workload); the default recomputes
the factor from (w, lambda), which also saves that memory. The weights w get a gradient when they require one (soft
weights of Eq. 1: dL/dw_t = sum_b g_tb (x_tb - z_tb), x taken as 0 on days with w_t = 0;
x is then kept for the backward pass). For a log-lambda
parametrisation pass lam = loglam.exp(): autograd applies the chain rule outside the layer.

Tensors use the tile layout: x [T, B, P], w [T, P], lam [T, P] (per day) or [P] (scalar).
"""
from __future__ import annotations

import torch

from . import ws


class WhittakerSmooth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, lam, d: int = 2, refine: bool = True, store_factor: bool = False):
        x, w, lam = x.contiguous(), w.contiguous(), lam.contiguous()
        fac = None
        if store_factor:
            T, _, P = x.shape
            fac = torch.empty((T, d + 1, P), dtype=x.dtype, device=x.device)
        z, status = ws.smooth(x, w, lam, d, factor=fac, refine=refine)
        ctx.d = d
        ctx.store = store_factor
        ctx.save_for_backward(w, lam, z, fac if store_factor else z.new_empty(0),
                              x if ctx.needs_input_grad[1] else z.new_empty(0))
        ctx.mark_non_differentiable(status)
        return z, status

    @staticmethod
    def backward(ctx, gz, gstatus):
        w, lam, z, fac, x = ctx.saved_tensors
        need_x, need_w, need_lam = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        if gz is None or not (need_x or need_w or need_lam):
            return None, None, None, None, None, None
        if need_w:
            gx, glam, gw, _ = ws.smooth_adjoint_weights(x, w, lam, z, gz.contiguous(), ctx.d, want_gx=need_x,
                                                        want_glam=need_lam, factor=fac if ctx.store else None)
            return gx, gw, glam, None, None, None
        gx, glam, _ = ws.smooth_adjoint(w, lam, z, gz.contiguous(), ctx.d, want_gx=need_x, want_glam=need_lam,
                                        factor=fac if ctx.store else None)
        return gx, None, glam, None, None, None


def whittaker_smooth(x, w, lam, d: int = 2, refine: bool = True, store_factor: bool = False):
    """z = (W + D^T Lambda D)^{-1} W x, differentiable in x, w and lam. Returns (z, status)."""
    return WhittakerSmooth.apply(x, w, lam, d, refine, store_factor)


class WhittakerSmoothDates(torch.autograd.Function):
    """The layer on unevenly spaced sample times t [T, P] (the divided-difference operator):
    forward ws.smooth_dates, backward ws.smooth_dates_adjoint; differentiable in x and lam."""

    @staticmethod
    def forward(ctx, t, x, w, lam, d: int = 2):
        t, x, w, lam = t.contiguous(), x.contiguous(), w.contiguous(), lam.contiguous()
        z, status = ws.smooth_dates(t, x, w, lam, d)
        ctx.d = d
        ctx.save_for_backward(t, w, lam, z)
        ctx.mark_non_differentiable(status)
        return z, status

    @staticmethod
    def backward(ctx, gz, gstatus):
        t, w, lam, z = ctx.saved_tensors
        need_x, need_lam = ctx.needs_input_grad[1], ctx.needs_input_grad[3]
        if gz is None or not (need_x or need_lam):
            return None, None, None, None, None
        gx, glam, _ = ws.smooth_dates_adjoint(t, w, lam, z, gz.contiguous(), ctx.d, want_glam=need_lam)
        return None, gx if need_x else None, None, glam, None


def whittaker_smooth_dates(t, x, w, lam, d: int = 2):
    """z = (W + D^T Lambda D)^{-1} W x on sample times t, differentiable in x and lam."""
    return WhittakerSmoothDates.apply(t, x, w, lam, d)
