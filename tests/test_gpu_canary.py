"""Out-of-bounds writes (compute-sanitizer is not available on the GPU pool): every output
array and the workspace of the C-ABI calls are views into larger buffers whose margins hold
a known bit pattern; after each call the margins must be untouched. Odd sizes (T = 37, not
a multiple of any chunk; P = 301, not a multiple of 4 or 128, which also takes the plain-load
staging paths; P = 300 the TMA paths), every order, one and several band groups."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_00048_b300 import synth
from tests.gpu_util import tile_inputs

pytestmark = pytest.mark.gpu

PAD = 8192  # elements of margin on each side


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    mod.tune_set(0, 0)
    return mod


class Padded:
    """A tensor of `shape` inside a buffer with PAD-element margins filled with a pattern."""

    def __init__(self, shape, dtype, zero=False):
        n = int(np.prod(shape)) if len(shape) else 1
        self.dtype = dtype
        if dtype == torch.uint8:
            self.buf = torch.full((n + 2 * PAD,), 0xA5, dtype=torch.uint8, device="cuda")
        else:
            self.buf = torch.full((n + 2 * PAD,), -7.25e29, dtype=dtype, device="cuda")
        self.t = self.buf[PAD:PAD + n].view(shape)
        if zero:
            self.t.zero_()
        self.ref = self.buf.clone()

    def margins_intact(self) -> bool:
        torch.cuda.synchronize()
        a, r = self.buf, self.ref
        return bool(torch.equal(a[:PAD], r[:PAD]) and torch.equal(a[-PAD:], r[-PAD:]))


def _workspace(ws, pb, flags):
    need = ws.workspace_size(pb, flags)
    assert need > 0
    return Padded((need,), torch.uint8, zero=True)


@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("B", [3, 10])
def test_smooth_refine_adjoint_margins(ws, P, d, B):
    rc, g, c = tile_inputs("layer", P, T=37, B=B, revisit=1, p_valid=0.6)
    x, w, lam = g["x"], g["w"], g["lam"]
    T = x.shape[0]
    pb = ws.make_problem(T, B, P, d, ws.F32, ws.LAM_PER_DAY)
    wsp = _workspace(ws, pb, ws.REFINE_ADJOINT | ws.REFINE)
    z, st = Padded(x.shape, torch.float32), Padded((P,), torch.uint8)
    ws.smooth(x, w, lam, d, z=z.t, status=st.t, refine=True, workspace_buf=wsp.t)
    gz = torch.randn_like(x)
    gx, gl, st2 = Padded(x.shape, torch.float32), Padded(lam.shape, torch.float32), Padded((P,), torch.uint8)
    ws.smooth_adjoint(w, lam, z.t, gz, d, gx=gx.t, glam=gl.t, status=st2.t, log_lambda=True, refine=True,
                      workspace_buf=wsp.t)
    fac = Padded((T, d + 1, P), torch.float32)
    ws.factor(w, lam, d, out=fac.t)
    gxf = Padded(x.shape, torch.float32)
    ws.smooth_adjoint(w, lam, z.t, gz, d, gx=gxf.t, want_glam=False, factor=fac.t, workspace_buf=wsp.t)
    ws.sync_status()
    for buf in (z, st, gx, gl, st2, fac, gxf, wsp):
        assert buf.margins_intact()


@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_posterior_weight_grad_margins(ws, P, d):
    rc, g, c = tile_inputs("layer", P, T=37, B=3, revisit=1, p_valid=0.6)
    x, w, lam = g["x"], g["w"], g["lam"]
    T, B, _ = x.shape
    z, _ = ws.smooth(x, w, lam, d)
    pb = ws.make_problem(T, B, P, d, ws.F32, ws.LAM_PER_DAY)
    wsp = _workspace(ws, pb, ws.POSTERIOR | ws.REFINE)
    outs = (Padded((T, P), torch.float32), Padded((B, P), torch.float32), Padded(x.shape, torch.float32),
            Padded((P,), torch.uint8))
    ws.posterior(x, w, lam, z, d, out=tuple(o.t for o in outs), workspace_buf=wsp.t)
    gx, gl, gw = Padded(x.shape, torch.float32), Padded(lam.shape, torch.float32), Padded((T, P), torch.float32)
    gz = torch.randn_like(x)
    ws.smooth_adjoint_weights(x, w, lam, z, gz, d, gx=gx.t, glam=gl.t, gw=gw.t, workspace_buf=wsp.t)
    torch.cuda.synchronize()
    for buf in outs + (gx, gl, gw, wsp):
        assert buf.margins_intact()


@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_dates_margins(ws, P, d):
    """Smooth with refinement, adjoint and posterior on acquisition dates (10 bands: groups
    of 5 and of 4 + 4 + 2)."""
    rc = synth.Recipe(**{**synth.RECIPES["hetero_tile"].__dict__, "T": 201, "n_bands": 10})
    out = synth.generate_dates_tile(rc, P, device="cuda")
    t, x, w, lam = out["t"], out["x"], out["w"], out["lam"]
    T, B, _ = x.shape
    pb = ws.make_problem(T, B, P, d, ws.F32, ws.LAM_PER_DAY)
    wsp = _workspace(ws, pb, ws.DATES | ws.REFINE | ws.POSTERIOR)
    z, st = Padded(x.shape, torch.float32), Padded((P,), torch.uint8)
    ws.smooth_dates(t, x, w, lam, d, z=z.t, status=st.t, refine=True, workspace_buf=wsp.t)
    gz = torch.randn_like(x)
    gx, gl = Padded(x.shape, torch.float32), Padded(lam.shape, torch.float32)
    ws.smooth_dates_adjoint(t, w, lam, z.t, gz, d, gx=gx.t, glam=gl.t, log_lambda=True, workspace_buf=wsp.t)
    outs = (Padded((T, P), torch.float32), Padded((B, P), torch.float32), Padded(x.shape, torch.float32),
            Padded((P,), torch.uint8))
    ws.posterior(x, w, lam, z.t, d, out=tuple(o.t for o in outs), workspace_buf=wsp.t, t=t)
    torch.cuda.synchronize()
    for buf in (z, st, gx, gl, wsp) + outs:
        assert buf.margins_intact()


@pytest.mark.parametrize("dates", [False, True])
@pytest.mark.parametrize("P", [300, 301])
def test_gcv_margins(ws, P, dates):
    """ws_gcv_smooth / ws_gcv_smooth_dates through the C-ABI with padded z, lam_best, scores
    and status (16 series per CTA: 301 leaves a partial group)."""
    base = synth.RECIPES["learned"].__dict__
    rc = synth.Recipe(**{**base, "T": 120})
    if dates:
        out = synth.generate_dates_tile(rc, P, device="cuda")
        t = out["t"]
    else:
        out = synth.generate_tile(rc, P, device="cuda")
        t = None
    x, w = out["x"], out["w"]
    T = x.shape[0]
    grid = [10.0 ** (i / 3.0) for i in range(16)]
    pb = ws.make_problem(T, 1, P, 2, ws.F32, ws.LAM_SCALAR)
    wsp = _workspace(ws, pb, ws.GCV | ws.REFINE | (ws.DATES if dates else 0))
    z, lb = Padded(x.shape, torch.float32), Padded((P,), torch.float32)
    sc, st = Padded((16, P), torch.float32), Padded((P,), torch.uint8)
    arr = (ctypes.c_float * 16)(*grid)
    P_ = ws._ptr
    if dates:
        rc_ = ws.lib().ws_gcv_smooth_dates(ctypes.byref(pb), P_(t), P_(x), P_(w), arr, 16, P_(z.t), P_(lb.t),
                                           P_(sc.t), P_(st.t), ws.REFINE, P_(wsp.t), wsp.t.numel(), None)
    else:
        rc_ = ws.lib().ws_gcv_smooth(ctypes.byref(pb), P_(x), P_(w), arr, 16, P_(z.t), P_(lb.t), P_(sc.t),
                                     P_(st.t), ws.REFINE, P_(wsp.t), wsp.t.numel(), None)
    assert rc_ == 0, ws.last_error()
    torch.cuda.synchronize()
    for buf in (z, lb, sc, st, wsp):
        assert buf.margins_intact()


def test_binding_rejects_wrong_output_arrays(ws):
    """Output arrays a caller passes to the binding must have exactly the shape the kernels
    write (and be contiguous, of the inputs' dtype, on their device): anything else is a
    ValueError before any launch."""
    rc, g, c = tile_inputs("layer", 64, T=30, B=2)
    x, w, lam = g["x"], g["w"], g["lam"]
    T, B, P = x.shape
    short = torch.empty(T, B, P - 1, device="cuda")
    with pytest.raises(ValueError):
        ws.smooth(x, w, lam, 2, z=short)
    with pytest.raises(ValueError):
        ws.smooth(x, w, lam, 2, status=torch.empty(P + 1, dtype=torch.uint8, device="cuda"))
    z, _ = ws.smooth(x, w, lam, 2)
    gz = torch.randn_like(x)
    with pytest.raises(ValueError):
        ws.smooth_adjoint(w, lam, z, gz, 2, gx=short)
    with pytest.raises(ValueError):
        ws.smooth_adjoint(w, lam, z, gz, 2, glam=torch.empty(T - 1, P, device="cuda"))
    with pytest.raises(ValueError):
        ws.posterior(x, w, lam, z, 2, out=(torch.empty(T, P, device="cuda"), torch.empty(B, P, device="cuda"),
                                           short, torch.empty(P, dtype=torch.uint8, device="cuda")))
    with pytest.raises(ValueError):
        ws.smooth_adjoint_weights(x, w, lam, z, gz, 2, gw=torch.empty(T, P, 2, device="cuda"))
    with pytest.raises(ValueError):
        ws.factor(w, lam, 2, out=torch.empty(T, 2, P, device="cuda"))
    fac, _ = ws.factor(w, lam, 2)
    with pytest.raises(ValueError):
        ws.solve(fac[:, :2].contiguous(), w, x, 2)
    with pytest.raises(ValueError):
        ws.solve(fac, w, x, 2, z=x.transpose(0, 2))
    t = torch.arange(T, dtype=torch.float32, device="cuda").view(T, 1).expand(T, P).contiguous()
    with pytest.raises(ValueError):
        ws.smooth_dates(t, x, w, lam, 2, z=short)
    with pytest.raises(ValueError):
        ws.smooth_dates_adjoint(t, w, lam, z, gz, 2, gx=short)


@pytest.mark.parametrize("P", [300, 301])
@pytest.mark.parametrize("d", [1, 3])
@pytest.mark.parametrize("B", [3, 10])
def test_adjoint_mse_margins(ws, P, d, B):
    """The adjoint with the fused masked-MSE loss: gx, glam, the per-series loss, status
    and the workspace."""
    rc, g, c = tile_inputs("layer", P, T=37, B=B, revisit=1, p_valid=0.6)
    x, w, lam = g["x"], g["w"], g["lam"]
    T = x.shape[0]
    z, _ = ws.smooth(x, w, lam, d)
    pb = ws.make_problem(T, B, P, d, ws.F32, ws.LAM_PER_DAY)
    wsp = _workspace(ws, pb, 0)
    mask = (torch.rand(T, P, device="cuda") < 0.3).float()
    gx, gl = Padded(x.shape, torch.float32), Padded(lam.shape, torch.float32)
    ls, st = Padded((P,), torch.float32), Padded((P,), torch.uint8)
    ws.smooth_adjoint_mse(w, lam, z, x, d, mask=mask, scale=0.01, gx=gx.t, glam=gl.t, loss=ls.t, status=st.t,
                          log_lambda=True, workspace_buf=wsp.t)
    ws.sync_status()
    for buf in (gx, gl, ls, st, wsp):
        assert buf.margins_intact()


@pytest.mark.parametrize("P", [5, 301])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
@pytest.mark.parametrize("T", [37, 150])
def test_partitioned_margins(ws, P, d, T):
    """The partitioned solve: z, status and the workspace, with one domain (T = 37) and
    several with a short last one (T = 150)."""
    rc, g, c = tile_inputs("layer", P, T=T, B=3, revisit=1, p_valid=0.6)
    x, w, lam = g["x"], g["w"], g["lam"]
    pb = ws.make_problem(T, 3, P, d, ws.F32, ws.LAM_PER_DAY)
    wsp = _workspace(ws, pb, ws.PARTITIONED)
    z, st = Padded(x.shape, torch.float32), Padded((P,), torch.uint8)
    ws.smooth_partitioned(x, w, lam, d, z=z.t, status=st.t, workspace_buf=wsp.t)
    ws.sync_status()
    for buf in (z, st, wsp):
        assert buf.margins_intact()


@pytest.mark.parametrize("tiles", [False, True])
def test_ragged_margins(ws, tiles):
    """The ragged plan's execute on caller scratch: z, status and the workspace, with the
    refinement step (and the length-class tiles)."""
    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 333, device="cuda", t_range=(1, 300))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    need = plan.workspace_size(refine=True, tiles=tiles)
    wsp = Padded((need,), torch.uint8, zero=True)
    z, st = Padded(out["x"].shape, torch.float32), Padded((333,), torch.uint8)
    plan.execute(out["x"], out["w"], out["lam"], z=z.t, status=st.t, refine=True, tiles=tiles, workspace_buf=wsp.t)
    ws.sync_status()
    for buf in (z, st, wsp):
        assert buf.margins_intact()
