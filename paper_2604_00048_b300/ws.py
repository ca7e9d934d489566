"""Thin Python binding of libws_b300.so (C-ABI in include/ws.h).

Argument marshalling only: shapes, dtypes and device pointers of torch tensors are
checked and passed to the CUDA library, which does every step of the computation.
There is no CPU fallback; if the shared library is missing, importing this module
raises (build it with `python -m paper_2604_00048_b300.build`).

Tensors use the tile layout of the C-ABI:
    x, z   [T, B, P]   (pixel fastest)
    w      [T, P]
    lam    [T, P] per day (entry k weights difference row k) or [P] scalar
    factor [T, d+1, P] (ws_factor layout)
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libws_b300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ws.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} (run python -m paper_2604_00048_b300.build)")
_lib = ctypes.CDLL(LIB_PATH)

WS_OK, WS_EINVAL, WS_ENOMEM_WS, WS_ECUDA, WS_ETIMEOUT, WS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
SERIES_OK, SERIES_NOT_PD, SERIES_NONFINITE, SERIES_BADARG = 0, 1, 2, 3
LAYOUT_TILE = 0
F32, F64 = 0, 1
LAM_PER_DAY, LAM_SCALAR = 0, 1
GRAD_LOGLAM = 0x1
REFINE = 0x2
REFINE_ADJOINT = 0x4


class Problem(ctypes.Structure):
    _fields_ = [("n_series", ctypes.c_int64), ("T", ctypes.c_int32), ("d", ctypes.c_int32),
                ("n_bands", ctypes.c_int32), ("layout", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("lam_mode", ctypes.c_int32)]


_vp, _sz, _u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32
_PP = ctypes.POINTER(Problem)
_lib.ws_workspace_size.restype = _sz
_lib.ws_workspace_size.argtypes = [_PP, _u32]
_lib.ws_smooth_batch.restype = ctypes.c_int
_lib.ws_smooth_batch.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _sz, _vp]
_lib.ws_factor.restype = ctypes.c_int
_lib.ws_factor.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.ws_solve.restype = ctypes.c_int
_lib.ws_solve.argtypes = [_PP, _vp, _vp, _vp, _vp, _u32, _vp, _sz, _vp]
_lib.ws_solve_adjoint.restype = ctypes.c_int
_lib.ws_solve_adjoint.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _vp, _sz, _vp]
_lib.ws_refine.restype = ctypes.c_int
_lib.ws_refine.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.ws_gcv_smooth.restype = ctypes.c_int
_lib.ws_gcv_smooth.argtypes = [_PP, _vp, _vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int, _vp, _vp, _vp, _vp,
                               _u32, _vp, _sz, _vp]
_lib.ws_smooth_dates.restype = ctypes.c_int
_lib.ws_smooth_dates.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _sz, _vp]
_lib.ws_smooth_dates_adjoint.restype = ctypes.c_int
_lib.ws_smooth_dates_adjoint.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp, _vp, _sz, _vp]
_lib.ws_gcv_smooth_dates.restype = ctypes.c_int
_lib.ws_gcv_smooth_dates.argtypes = [_PP, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int, _vp, _vp, _vp,
                                     _vp, _u32, _vp, _sz, _vp]
_lib.ws_posterior_dates.restype = ctypes.c_int
_lib.ws_posterior_dates.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.ws_weight_grad.restype = ctypes.c_int
_lib.ws_weight_grad.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.ws_posterior.restype = ctypes.c_int
_lib.ws_posterior.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.ws_smooth_batch_noalloc.restype = ctypes.c_int
_lib.ws_smooth_batch_noalloc.argtypes = [_PP, _vp, _vp, _vp, _vp, _vp, _vp, _u32, _vp]
NOALLOC_MAX_BYTES = 64 << 20
_lib.ws_tune_set.restype = ctypes.c_int
_lib.ws_tune_set.argtypes = [ctypes.c_int32, ctypes.c_int32]
_lib.ws_solve_adjoint_mse.restype = ctypes.c_int
_lib.ws_solve_adjoint_mse.argtypes = [ctypes.POINTER(Problem)] + [ctypes.c_void_p] * 5 + [ctypes.c_double] + \
    [ctypes.c_void_p] * 3 + [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, _sz, ctypes.c_void_p]
_lib.ws_smooth_partitioned.restype = ctypes.c_int
_lib.ws_smooth_partitioned.argtypes = [ctypes.POINTER(Problem)] + [ctypes.c_void_p] * 6 + [_sz, ctypes.c_void_p]
_lib.ws_tune_pixels_per_cta.restype = ctypes.c_int
_lib.ws_tune_pixels_per_cta.argtypes = [ctypes.c_int32]
_lib.ws_tune_checkpoint_group.restype = ctypes.c_int
_lib.ws_tune_checkpoint_group.argtypes = [ctypes.c_int32]
_lib.ws_selftest_wait.restype = ctypes.c_int
_lib.ws_selftest_wait.argtypes = [_vp, _sz, _vp]
_lib.ws_sync_status.restype = ctypes.c_int
_lib.ws_sync_status.argtypes = [_vp, _sz, _vp]
_lib.ws_last_error.restype = ctypes.c_int
_lib.ws_last_error.argtypes = [ctypes.c_char_p, _sz]
_lib.ws_version.restype = ctypes.c_char_p
_lib.ws_version.argtypes = []


class Ragged(ctypes.Structure):
    _fields_ = [("n_series", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("d_per_series", ctypes.c_void_p),
                ("d_uniform", ctypes.c_int32), ("n_bands", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("lam_mode", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("chunk_days", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("tuned", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("tuned_ms", ctypes.c_float), ("hp_series", ctypes.c_int32), ("tiles", ctypes.c_int32)]


PLAN_AUTOTUNE, PLAN_GRAPH, PLAN_REFINE, PLAN_TILES = 0x1, 0x2, 0x4, 0x8
_lib.ws_plan_create.restype = ctypes.c_int
_lib.ws_plan_create.argtypes = [ctypes.POINTER(Ragged), ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
_lib.ws_plan_execute.restype = ctypes.c_int
_lib.ws_plan_execute.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5 + [ctypes.c_uint32, ctypes.c_void_p,
                                                                               _sz, ctypes.c_void_p]
_lib.ws_plan_workspace_size.restype = _sz
_lib.ws_plan_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
_lib.ws_plan_info.restype = ctypes.c_int
_lib.ws_plan_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(PlanStats)]
_lib.ws_plan_destroy.restype = None
_lib.ws_plan_destroy.argtypes = [ctypes.c_void_p]


class WSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ws error {code}: {msg}")
        self.code = code


def lib():
    return _lib


def declared_symbols(header: str = HEADER):
    """Function names declared in include/ws.h."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ws_[a-z0-9_]+)\s*\(", txt)))


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    _lib.ws_last_error(buf, 512)
    return buf.value.decode()


def _check(rc: int):
    if rc != WS_OK:
        raise WSError(rc, last_error())


def version() -> str:
    return _lib.ws_version().decode()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype} (float32 or float64)")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_problem(T: int, B: int, P: int, d: int, dtype: int, lam_mode: int) -> Problem:
    return Problem(n_series=P, T=T, d=d, n_bands=B, layout=LAYOUT_TILE, dtype=dtype, lam_mode=lam_mode)


def workspace_size(pb: Problem, flags: int = 0) -> int:
    return int(_lib.ws_workspace_size(ctypes.byref(pb), flags))


_ws_cache = {}


def workspace(pb: Problem, device, flags: int = 0, given: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Device scratch for `pb`: `given` if not None (a uint8 tensor the caller owns, e.g. one
    per stream for concurrent calls; its first 256 bytes must start at zero), else the
    per-device cache (grown on demand; header zeroed once). Calls that may run at the same
    time on different streams need different workspaces."""
    need = workspace_size(pb, flags)
    if given is not None:
        if given.numel() < need or given.dtype != torch.uint8 or not given.is_cuda:
            raise ValueError(f"workspace needs {need} bytes (uint8, CUDA)")
        return given
    if need == 0:
        raise WSError(WS_EINVAL, last_error() or "invalid problem")
    dev = torch.device(device)
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < need:
        if buf is not None:
            # kernels on any stream may still use the old scratch: drain before freeing it
            torch.cuda.synchronize(dev)
            _ws_cache[key] = None
            del buf
        buf = torch.zeros(need, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize(dev)
        _ws_cache[key] = buf
    return buf


def _check_tile(x, w, lam, d):
    if x.dim() != 3:
        raise ValueError("x must be [T, B, P]")
    T, B, P = x.shape
    if tuple(w.shape) != (T, P):
        raise ValueError("w must be [T, P]")
    if lam.dim() == 2 and tuple(lam.shape) != (T, P):
        raise ValueError("per-day lam must be [T, P]")
    if lam.dim() == 1 and lam.shape[0] != P:
        raise ValueError("scalar lam must be [P]")
    for t in (x, w, lam):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != x.dtype:
            raise ValueError("x, w, lam must be contiguous CUDA tensors of one dtype")
    return T, B, P, (LAM_SCALAR if lam.dim() == 1 else LAM_PER_DAY)


def _check_out(t, shape, dtype, device, name):
    """An array the caller passes for an output: the kernels write every element of exactly
    `shape`, so it must have that shape, be contiguous and match the dtype and device."""
    if t is None:
        return
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous() or t.dtype != dtype or t.device != device:
        raise ValueError(f"{name} must be a contiguous {tuple(shape)} {dtype} tensor on {device}")


def smooth(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, d: int = 2, *, z=None, status=None,
           factor=None, refine: bool = False, stream=None, workspace_buf=None):
    """z = (W + D^T Lambda D)^{-1} W x per series and band (Eq. 3; Eq. 2 for scalar lam).

    refine: one step of iterative refinement with a double-word residual.
    Returns (z, status). `factor` (optional [T, d+1, P]) receives the factor."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    _check_out(z, x.shape, x.dtype, x.device, "z")
    _check_out(status, (P,), torch.uint8, x.device, "status")
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    flags = REFINE if refine else 0
    if z is None:
        z = torch.empty_like(x)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=x.device)
    if factor is not None and (tuple(factor.shape) != (T, d + 1, P) or factor.dtype != x.dtype):
        raise ValueError("factor must be [T, d+1, P] of x's dtype")
    ws = workspace(pb, x.device, flags, workspace_buf)
    rc = _lib.ws_smooth_batch(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(factor),
                              _ptr(status), flags, _ptr(ws), ws.numel(), _stream_ptr(stream))
    _check(rc)
    return z, status


GCV = 0x8
GCV_GRID = [10.0 ** (i / 3.0) for i in range(16)]  # log10 lambda in {0, 1/3, ..., 5}


def gcv_smooth(x: torch.Tensor, w: torch.Tensor, lam_grid=None, d: int = 2, *, refine: bool = False,
               want_scores: bool = True, stream=None, t=None):
    """Per-series lambda by GCV over a grid of scalar values, then the smoothing at it.

    x: [T, 1, P] FP32, w: [T, P]. lam_grid: up to 16 positive values (default GCV_GRID).
    t: optional [T, P] sample times (the uneven-spacing operator of smooth_dates).
    Returns (z, lam_best [P], scores [n_grid, P] or None, status [P])."""
    grid = [float(v) for v in (GCV_GRID if lam_grid is None else lam_grid)]
    lam_dummy = torch.empty(x.shape[2], dtype=x.dtype, device=x.device)
    T, B, P, _ = _check_tile(x, w, lam_dummy, d)
    pb = make_problem(T, B, P, d, _dtype_code(x), LAM_SCALAR)
    flags = REFINE if refine else 0
    z = torch.empty_like(x)
    lam_best = torch.empty(P, dtype=torch.float32, device=x.device)
    scores = torch.empty(len(grid), P, dtype=torch.float32, device=x.device) if want_scores else None
    status = torch.empty(P, dtype=torch.uint8, device=x.device)
    ws = workspace(pb, x.device, GCV | flags | (DATES if t is not None else 0))
    arr = (ctypes.c_float * len(grid))(*grid)
    if t is not None:
        if tuple(t.shape) != (T, P) or t.dtype != x.dtype or not t.is_cuda or not t.is_contiguous():
            raise ValueError("t must be a contiguous [T, P] CUDA tensor of x's dtype")
        _check(_lib.ws_gcv_smooth_dates(ctypes.byref(pb), _ptr(t), _ptr(x), _ptr(w), arr, len(grid), _ptr(z),
                                        _ptr(lam_best), _ptr(scores), _ptr(status), flags, _ptr(ws), ws.numel(),
                                        _stream_ptr(stream)))
        return z, lam_best, scores, status
    _check(_lib.ws_gcv_smooth(ctypes.byref(pb), _ptr(x), _ptr(w), arr, len(grid), _ptr(z), _ptr(lam_best),
                              _ptr(scores), _ptr(status), flags, _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return z, lam_best, scores, status


POSTERIOR = 0x10


def posterior(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, d: int = 2, *,
              want_sd: bool = True, stream=None, workspace_buf=None, out=None, t=None):
    """Posterior spread of the smooth z of x (the credibility intervals of Fig. 4):
    diag(Omega^{-1}) per day, the residual variance sigma2_b = RSS_b / (n - tr H) per band,
    and sd = sqrt(sigma2_b diag_t); the interval at level q is z +- q sd.

    x, z: [T, B, P]; w: [T, P]; lam: [T, P] or [P]. out: optional (diag, sigma2, sd, status)
    to write into. t: optional [T, P] sample times (the uneven-spacing operator of
    smooth_dates; z is then the smooth on those dates). Returns (diag [T, P], sigma2 [B, P],
    sd [T, B, P] or None, status [P])."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    if tuple(z.shape) != tuple(x.shape) or z.dtype != x.dtype or not z.is_cuda or not z.is_contiguous():
        raise ValueError("z must be a contiguous CUDA tensor shaped and typed like x")
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    if out is not None:
        diag, sigma2, sd, status = out
        _check_out(diag, (T, P), x.dtype, x.device, "diag")
        _check_out(sigma2, (B, P), x.dtype, x.device, "sigma2")
        _check_out(sd, x.shape, x.dtype, x.device, "sd")
        _check_out(status, (P,), torch.uint8, x.device, "status")
    else:
        diag = torch.empty(T, P, dtype=x.dtype, device=x.device)
        sigma2 = torch.empty(B, P, dtype=x.dtype, device=x.device)
        sd = torch.empty_like(x) if want_sd else None
        status = torch.empty(P, dtype=torch.uint8, device=x.device)
    ws = workspace(pb, x.device, POSTERIOR, workspace_buf)
    if t is not None:
        if tuple(t.shape) != (T, P) or t.dtype != x.dtype or not t.is_cuda or not t.is_contiguous():
            raise ValueError("t must be a contiguous [T, P] CUDA tensor of x's dtype")
        _check(_lib.ws_posterior_dates(ctypes.byref(pb), _ptr(t), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(diag),
                                       _ptr(sigma2), _ptr(sd), _ptr(status), _ptr(ws), ws.numel(),
                                       _stream_ptr(stream)))
        return diag, sigma2, sd, status
    _check(_lib.ws_posterior(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(diag), _ptr(sigma2),
                             _ptr(sd), _ptr(status), _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return diag, sigma2, sd, status


def smooth_noalloc(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, d: int = 2, *, z, status,
                   refine: bool = False, stream=None):
    """smooth() through ws_smooth_batch_noalloc: the scratch is the library's static device
    array (NOALLOC_MAX_BYTES), so nothing is allocated; z and status must be given.
    Raises WSError (code ENOMEM_WS) when the problem's workspace exceeds the array."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    if tuple(z.shape) != tuple(x.shape) or z.dtype != x.dtype or not z.is_contiguous():
        raise ValueError("z must be a contiguous tensor shaped and typed like x")
    if status.numel() != P or status.dtype != torch.uint8:
        raise ValueError("status must hold P uint8 codes")
    _check(_lib.ws_smooth_batch_noalloc(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), None,
                                        _ptr(status), REFINE if refine else 0, _stream_ptr(stream)))
    return z, status


def refine(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, d: int = 2, *, stream=None,
           workspace_buf=None):
    """One step of iterative refinement of z (in place) with a double-word residual."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    ws = workspace(pb, x.device, REFINE, workspace_buf)
    _check(_lib.ws_refine(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(ws), ws.numel(),
                          _stream_ptr(stream)))
    return z


PARTITIONED = 0x80


def smooth_partitioned(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, d: int = 2, *, z=None, status=None,
                       stream=None, workspace_buf=None):
    """z = Omega^{-1} W x by the partitioned parallel-in-time solve (few long series):
    returns (z, status), tile layout as smooth()."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    _check_out(z, x.shape, x.dtype, x.device, "z")
    _check_out(status, (P,), torch.uint8, x.device, "status")
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    if z is None:
        z = torch.empty_like(x)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=x.device)
    ws = workspace(pb, x.device, PARTITIONED, workspace_buf)
    _check(_lib.ws_smooth_partitioned(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(status),
                                      _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return z, status


def smooth_adjoint(w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, gz: torch.Tensor, d: int = 2, *,
                   gx=None, glam=None, want_gx: bool = True, want_glam: bool = True, log_lambda: bool = False,
                   factor=None, status=None, refine: bool = False, stream=None, workspace_buf=None,
                   _raw_g: bool = False):
    """Vector-Jacobian products of z = Omega^{-1} W x (Eqs. 4-5): returns (gx, glam, status).

    gx = W Omega^{-1} gz; glam_k = -sum_b (D g_b)_k (D z_b)_k (k < T-d, 0 after), times
    lambda_k with log_lambda. factor: a stored factor ([T, d+1, P]) or None to recompute."""
    T, B, P, lm = _check_tile(gz, w, lam, d)
    if tuple(z.shape) != tuple(gz.shape) or not z.is_contiguous() or z.dtype != gz.dtype:
        raise ValueError("z must match gz")
    _check_out(gx, gz.shape, gz.dtype, gz.device, "gx")
    _check_out(glam, lam.shape, gz.dtype, gz.device, "glam")
    _check_out(status, (P,), torch.uint8, gz.device, "status")
    _check_out(factor, (T, d + 1, P), gz.dtype, gz.device, "factor")
    pb = make_problem(T, B, P, d, _dtype_code(gz), lm)
    if gx is None and want_gx:
        gx = torch.empty_like(gz)
    if glam is None and want_glam:
        glam = torch.empty_like(lam)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=gz.device)
    flags = (GRAD_LOGLAM if log_lambda else 0) | (REFINE_ADJOINT if refine else 0)
    ws = workspace(pb, gz.device, flags | (REFINE if factor is not None else 0), workspace_buf)
    if _raw_g:
        flags |= ADJ_RAW_G
    rc = _lib.ws_solve_adjoint(ctypes.byref(pb), _ptr(factor), _ptr(w), _ptr(lam), _ptr(z), _ptr(gz), _ptr(gx),
                               _ptr(glam), flags, _ptr(status), _ptr(ws), ws.numel(), _stream_ptr(stream))
    _check(rc)
    return gx, glam, status



def smooth_adjoint_mse(w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, target: torch.Tensor, d: int = 2, *,
                       mask=None, scale: float = 1.0, gx=None, glam=None, loss=None, want_gx: bool = True,
                       want_glam: bool = True, want_loss: bool = True, log_lambda: bool = False, status=None,
                       stream=None, workspace_buf=None):
    """Adjoint of the masked MSE loss L_p = scale/2 sum m (z - target)^2 with the loss gradient
    formed inside the kernel (Section 4.3; Eqs. 4-5): returns (gx, glam, loss [P], status)."""
    T, B, P, lm = _check_tile(target, w, lam, d)
    if tuple(z.shape) != tuple(target.shape) or not z.is_contiguous() or z.dtype != target.dtype:
        raise ValueError("z must match target")
    _check_out(mask, (T, P), target.dtype, target.device, "mask")
    _check_out(gx, target.shape, target.dtype, target.device, "gx")
    _check_out(glam, lam.shape, target.dtype, target.device, "glam")
    _check_out(loss, (P,), target.dtype, target.device, "loss")
    _check_out(status, (P,), torch.uint8, target.device, "status")
    pb = make_problem(T, B, P, d, _dtype_code(target), lm)
    if gx is None and want_gx:
        gx = torch.empty_like(target)
    if glam is None and want_glam:
        glam = torch.empty_like(lam)
    if loss is None and want_loss:
        loss = torch.empty(P, dtype=target.dtype, device=target.device)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=target.device)
    ws = workspace(pb, target.device, 0, workspace_buf)
    flags = GRAD_LOGLAM if log_lambda else 0
    _check(_lib.ws_solve_adjoint_mse(ctypes.byref(pb), _ptr(w), _ptr(lam), _ptr(z), _ptr(target), _ptr(mask),
                                     float(scale), _ptr(gx), _ptr(glam), _ptr(loss), flags, _ptr(status), _ptr(ws),
                                     ws.numel(), _stream_ptr(stream)))
    return gx, glam, loss, status

DATES = 0x40


def smooth_dates(t: torch.Tensor, x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, d: int = 2, *, z=None,
                 status=None, refine: bool = False, stream=None, workspace_buf=None):
    """z = (W + D^T Lambda D)^{-1} W x on unevenly spaced sample times: t [T, P] (each
    series' strictly increasing dates, x's dtype), D the uneven-spacing discrete derivative
    (row k: d! times the divided-difference weights on t_k..t_{k+d}). x [T, B, P], w [T, P],
    lam [T, P] or [P]. refine: one step of iterative refinement. Returns (z, status)."""
    T, B, P, lm = _check_tile(x, w, lam, d)
    if tuple(t.shape) != (T, P) or t.dtype != x.dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError("t must be a contiguous [T, P] CUDA tensor of x's dtype")
    _check_out(z, x.shape, x.dtype, x.device, "z")
    _check_out(status, (P,), torch.uint8, x.device, "status")
    pb = make_problem(T, B, P, d, _dtype_code(x), lm)
    if z is None:
        z = torch.empty_like(x)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=x.device)
    flags = REFINE if refine else 0
    ws = workspace(pb, x.device, DATES | flags, workspace_buf)
    _check(_lib.ws_smooth_dates(ctypes.byref(pb), _ptr(t), _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(status),
                                flags, _ptr(ws), ws.numel(), _stream_ptr(stream)))
    return z, status


def smooth_dates_adjoint(t: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, gz: torch.Tensor,
                         d: int = 2, *, gx=None, glam=None, want_glam: bool = True, log_lambda: bool = False,
                         status=None, stream=None, workspace_buf=None):
    """Vector-Jacobian products of smooth_dates (Eqs. 4-5 on sample times): returns
    (gx = W Omega^{-1} gz, glam or None, status); glam_k = -sum_b (D g_b)_k (D z_b)_k, times
    lambda_k with log_lambda."""
    T, B, P, lm = _check_tile(gz, w, lam, d)
    if tuple(z.shape) != tuple(gz.shape) or z.dtype != gz.dtype or not z.is_contiguous():
        raise ValueError("z must match gz")
    if tuple(t.shape) != (T, P) or t.dtype != gz.dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError("t must be a contiguous [T, P] CUDA tensor of gz's dtype")
    _check_out(gx, gz.shape, gz.dtype, gz.device, "gx")
    _check_out(glam, lam.shape, gz.dtype, gz.device, "glam")
    _check_out(status, (P,), torch.uint8, gz.device, "status")
    pb = make_problem(T, B, P, d, _dtype_code(gz), lm)
    if gx is None:
        gx = torch.empty_like(gz)
    if glam is None and want_glam:
        glam = torch.empty_like(lam)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=gz.device)
    ws = workspace(pb, gz.device, DATES, workspace_buf)
    _check(_lib.ws_smooth_dates_adjoint(ctypes.byref(pb), _ptr(t), _ptr(w), _ptr(lam), _ptr(z), _ptr(gz), _ptr(gx),
                                        _ptr(glam), GRAD_LOGLAM if log_lambda else 0, _ptr(status), _ptr(ws),
                                        ws.numel(), _stream_ptr(stream)))
    return gx, glam, status


ADJ_RAW_G = 0x20


def smooth_adjoint_weights(x: torch.Tensor, w: torch.Tensor, lam: torch.Tensor, z: torch.Tensor, gz: torch.Tensor,
                           d: int = 2, *, gx=None, glam=None, gw=None, want_gx: bool = True,
                           want_glam: bool = True, log_lambda: bool = False, factor=None, refine: bool = False,
                           stream=None, workspace_buf=None):
    """smooth_adjoint() plus the gradient with respect to the weights (soft weights of Eq. 1):
    dL/dw_t = sum_b g_tb (x_tb [w_t > 0] - z_tb), g = Omega^{-1} gz. Two C-ABI calls: the
    adjoint with WS_ADJ_RAW_G (g into the gx buffer), then ws_weight_grad (gw, and gx = W g
    in place). Returns (gx or None, glam or None, gw [T, P], status)."""
    T, B, P, lm = _check_tile(gz, w, lam, d)
    if tuple(x.shape) != tuple(gz.shape) or x.dtype != gz.dtype or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must match gz")
    _check_out(gx, gz.shape, gz.dtype, gz.device, "gx")
    _check_out(gw, w.shape, gz.dtype, gz.device, "gw")
    g = gx if gx is not None else torch.empty_like(gz)
    if gw is None:
        gw = torch.empty_like(w)
    _, glam, status = smooth_adjoint(w, lam, z, gz, d, gx=g, glam=glam, want_glam=want_glam, log_lambda=log_lambda,
                                     factor=factor, refine=refine, stream=stream, workspace_buf=workspace_buf,
                                     _raw_g=True)
    pb = make_problem(T, B, P, d, _dtype_code(gz), lm)
    _check(_lib.ws_weight_grad(ctypes.byref(pb), _ptr(x), _ptr(w), _ptr(z), _ptr(g), _ptr(g) if want_gx else None,
                               _ptr(gw), _stream_ptr(stream)))
    return (g if want_gx else None), glam, gw, status


def factor(w: torch.Tensor, lam: torch.Tensor, d: int = 2, *, out=None, status=None, stream=None):
    """Factor of Omega (ws_factor layout [T, d+1, P]): 1/D_t and L[t+j][t]. Returns (factor, status)."""
    if w.dim() != 2:
        raise ValueError("w must be [T, P]")
    T, P = w.shape
    if lam.dim() == 2 and tuple(lam.shape) != (T, P) or lam.dim() == 1 and lam.shape[0] != P or lam.dim() > 2:
        raise ValueError("lam must be [T, P] (per day) or [P] (scalar)")
    for tt in (w, lam):
        if not tt.is_cuda or not tt.is_contiguous() or tt.dtype != w.dtype or tt.device != w.device:
            raise ValueError("w and lam must be contiguous CUDA tensors of one dtype and device")
    _check_out(out, (T, d + 1, P), w.dtype, w.device, "out")
    _check_out(status, (P,), torch.uint8, w.device, "status")
    lm = LAM_SCALAR if lam.dim() == 1 else LAM_PER_DAY
    pb = make_problem(T, 1, P, d, _dtype_code(w), lm)
    if out is None:
        out = torch.empty((T, d + 1, P), dtype=w.dtype, device=w.device)
    if status is None:
        status = torch.empty(P, dtype=torch.uint8, device=w.device)
    _check(_lib.ws_factor(ctypes.byref(pb), _ptr(w), _ptr(lam), _ptr(out), _ptr(status), None, 0,
                          _stream_ptr(stream)))
    return out, status


def solve(fac: torch.Tensor, w: torch.Tensor, x: torch.Tensor, d: int = 2, *, z=None, stream=None):
    """z = Omega^{-1} W x with a stored factor."""
    if x.dim() != 3:
        raise ValueError("x must be [T, B, P]")
    T, B, P = x.shape
    for tt, shp, name in ((fac, (T, d + 1, P), "fac"), (w, (T, P), "w")):
        if tuple(tt.shape) != shp or not tt.is_cuda or not tt.is_contiguous() or tt.dtype != x.dtype or \
                tt.device != x.device:
            raise ValueError(f"{name} must be a contiguous {shp} CUDA tensor of x's dtype")
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    _check_out(z, x.shape, x.dtype, x.device, "z")
    pb = make_problem(T, B, P, d, _dtype_code(x), LAM_PER_DAY)
    if z is None:
        z = torch.empty_like(x)
    _check(_lib.ws_solve(ctypes.byref(pb), _ptr(fac), _ptr(w), _ptr(x), _ptr(z), 0, None, 0, _stream_ptr(stream)))
    return z


def tune_set(ctas_per_sm: int = 0, chunk_days: int = 0, pixels_per_cta: int = 0, checkpoint_group: int = 0):
    """Process-wide tile tuning knobs (0 = automatic): CTAs per SM, a chunk-size cap, the
    pixel series per CTA (64 or 128) and the chunks per checkpoint (1 or 2)."""
    _check(_lib.ws_tune_set(int(ctas_per_sm), int(chunk_days)))
    _check(_lib.ws_tune_pixels_per_cta(int(pixels_per_cta)))
    _check(_lib.ws_tune_checkpoint_group(int(checkpoint_group)))


def sync_status(device=None, stream=None):
    """Synchronise and read/clear the device error word of the cached workspace."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = dev.index if dev.index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(key)
    if buf is None:
        torch.cuda.synchronize(dev)
        return
    _check(_lib.ws_sync_status(_ptr(buf), buf.numel(), _stream_ptr(stream)))


class RaggedPlan:
    """Plan for a packed ragged batch (ws_plan_*): offsets [n+1] int64 and optional orders
    [n] int8 on the device; x/w/lam/z flat FP32 arrays (band b of series i at
    b*N + offsets[i] + t)."""

    def __init__(self, offsets: torch.Tensor, order=None, d: int = 2, n_bands: int = 1, lam_scalar: bool = False,
                 stream=None):
        if offsets.dtype != torch.int64 or not offsets.is_cuda:
            raise ValueError("offsets must be a CUDA int64 tensor")
        if order is not None and (order.dtype != torch.int8 or not order.is_cuda):
            raise ValueError("order must be a CUDA int8 tensor")
        self.offsets, self.order = offsets, order
        self.n = offsets.numel() - 1
        self.n_bands = n_bands
        self._rg = Ragged(self.n, offsets.data_ptr(), None if order is None else order.data_ptr(), int(d), n_bands,
                          F32, LAM_SCALAR if lam_scalar else LAM_PER_DAY)
        h = ctypes.c_void_p()
        _check(_lib.ws_plan_create(ctypes.byref(self._rg), ctypes.byref(h), _stream_ptr(stream)))
        self._h = h
        self._ws = None

    @staticmethod
    def _flags(autotune=False, graph=False, refine=False, tiles=False) -> int:
        return ((PLAN_AUTOTUNE if autotune else 0) | (PLAN_GRAPH if graph else 0) | (PLAN_REFINE if refine else 0)
                | (PLAN_TILES if tiles else 0))

    def workspace_size(self, autotune=False, graph=False, refine=False, tiles=False) -> int:
        need = int(_lib.ws_plan_workspace_size(self._h, self._flags(autotune, graph, refine, tiles)))
        if need == 0:
            raise WSError(WS_EINVAL, last_error())
        return need

    def execute(self, x, w, lam, z=None, status=None, autotune: bool = False, graph: bool = False,
                refine: bool = False, tiles: bool = False, stream=None, workspace_buf=None):
        """workspace_buf: a uint8 CUDA tensor of at least workspace_size(...) bytes the caller
        owns (e.g. to capture the call into its own CUDA graph); else the plan keeps one,
        grown on demand (the library itself never allocates on this call)."""
        if z is None:
            z = torch.empty_like(x)
        if status is None:
            status = torch.empty(self.n, dtype=torch.uint8, device=x.device)
        flags = self._flags(autotune, graph, refine, tiles)
        need = int(_lib.ws_plan_workspace_size(self._h, flags))
        if need == 0:
            raise WSError(WS_EINVAL, last_error())
        if workspace_buf is not None:
            if workspace_buf.numel() < need or workspace_buf.dtype != torch.uint8 or not workspace_buf.is_cuda:
                raise ValueError(f"workspace needs {need} bytes (uint8, CUDA)")
            wsb = workspace_buf
        else:
            if self._ws is None or self._ws.numel() < need:
                if self._ws is not None:
                    torch.cuda.synchronize(x.device)  # earlier calls may still use the old scratch
                self._ws = None
                self._ws = torch.empty(need, dtype=torch.uint8, device=x.device)
            wsb = self._ws
        _check(_lib.ws_plan_execute(self._h, _ptr(x), _ptr(w), _ptr(lam), _ptr(z), _ptr(status), flags,
                                    _ptr(wsb), wsb.numel(), _stream_ptr(stream)))
        return z, status

    def info(self) -> dict:
        st = PlanStats()
        _check(_lib.ws_plan_info(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in PlanStats._fields_}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.ws_plan_destroy(h)
            self._h = None


# ---- learned lambda: temporal convolution network ----------------------------------------
class TcnBatch(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("n_series", ctypes.c_int32), ("log_lam_min", ctypes.c_float),
                ("log_lam_max", ctypes.c_float)]


TCN_PARAMS, TCN_PACKED_BYTES, TCN_GAP = 75649, 304512, 4
TCN_LOG_LAM = (float(np.log(1e-1)), float(np.log(1e6)))
_TB = ctypes.POINTER(TcnBatch)
_lib.ws_tcn_scratch_size.restype = _sz
_lib.ws_tcn_scratch_size.argtypes = [_TB, ctypes.c_int]
_lib.ws_tcn_pack.restype = ctypes.c_int
_lib.ws_tcn_pack.argtypes = [_vp, _vp, _vp]
_lib.ws_tcn_forward.restype = ctypes.c_int
_lib.ws_tcn_forward.argtypes = [_TB, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, ctypes.c_int, _vp]
_lib.ws_tcn_backward.restype = ctypes.c_int
_lib.ws_tcn_backward.argtypes = [_TB, _vp, _vp, _vp, _vp, _sz, _vp]
_lib.ws_tcn_conv64.restype = ctypes.c_int
_lib.ws_tcn_conv64.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
_lib.ws_adam_step.restype = ctypes.c_int
_lib.ws_adam_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, _vp]
_lib.ws_mse_grad.restype = ctypes.c_int
_lib.ws_mse_grad.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_float, _vp]

TCN_OFFSETS = {"W1": (0, (64, 2, 9)), "b1": (1152, (64,)), "W2": (1216, (64, 64, 9)), "b2": (38080, (64,)),
               "W3": (38144, (64, 64, 9)), "b3": (75008, (64,)), "W4": (75072, (1, 64, 9)), "b4": (75648, (1,))}


def tcn_init(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-normal conv weights (std sqrt(2 / fan_in)), zero biases, last layer std 1e-2."""
    g = torch.Generator().manual_seed(seed)
    theta = torch.zeros(TCN_PARAMS, dtype=torch.float32)
    for name, (off, shape) in TCN_OFFSETS.items():
        if name.startswith("W"):
            fan_in = shape[1] * shape[2]
            std = 1e-2 if name == "W4" else (2.0 / fan_in) ** 0.5
            n = int(np.prod(shape))
            theta[off:off + n] = torch.randn(n, generator=g) * std
    return theta.to(device)


def tcn_pack(theta: torch.Tensor, packed: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if packed is None:
        packed = torch.empty(TCN_PACKED_BYTES // 2, dtype=torch.bfloat16, device=theta.device)
    _check(_lib.ws_tcn_pack(_ptr(theta), _ptr(packed), _stream_ptr(stream)))
    return packed


class Tcn:
    """The lambda network's parameters (FP32 master, Adam moments, gradient, BF16 copy) and
    its forward / backward / update calls."""

    def __init__(self, theta: torch.Tensor, log_lam=TCN_LOG_LAM):
        self.theta = theta.contiguous()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.packed = tcn_pack(self.theta)
        self.log_lam = log_lam
        self.step_count = 0
        self._scratch = None

    def _batch(self, T, P):
        return TcnBatch(T, P, self.log_lam[0], self.log_lam[1])

    def _scratch_for(self, b, training, device):
        need = int(_lib.ws_tcn_scratch_size(ctypes.byref(b), int(training)))
        if need == 0:
            raise WSError(WS_EINVAL, last_error())
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = None
            self._scratch = torch.zeros(need, dtype=torch.uint8, device=device)
        return self._scratch

    def forward(self, x: torch.Tensor, w: torch.Tensor, training: bool = False, stream=None,
                want_loglam: bool = True):
        """x, w: [T, P] FP32 (one band). Returns (lam, loglam), both [T, P] (loglam None
        unless want_loglam)."""
        T, P = w.shape
        x2 = x.reshape(T, P)
        b = self._batch(T, P)
        sc = self._scratch_for(b, training, x.device)
        lam = torch.empty(T, P, dtype=torch.float32, device=x.device)
        loglam = torch.empty_like(lam) if want_loglam else None
        _check(_lib.ws_tcn_forward(ctypes.byref(b), _ptr(self.packed), _ptr(self.theta), _ptr(x2), _ptr(w),
                                   _ptr(lam), _ptr(loglam), _ptr(sc), sc.numel(), int(training),
                                   _stream_ptr(stream)))
        return lam, loglam

    def backward(self, g_loglam: torch.Tensor, stream=None):
        """grad += dL/dtheta for dL/dlog lambda (after a training forward on the same batch)."""
        T, P = g_loglam.shape
        b = self._batch(T, P)
        sc = self._scratch_for(b, True, g_loglam.device)
        _check(_lib.ws_tcn_backward(ctypes.byref(b), _ptr(self.packed), _ptr(g_loglam.contiguous()), _ptr(self.grad),
                                    _ptr(sc), sc.numel(), _stream_ptr(stream)))

    def step(self, lr: float, betas=(0.9, 0.999), eps: float = 1e-8, stream=None):
        self.step_count += 1
        _check(_lib.ws_adam_step(_ptr(self.theta), _ptr(self.m), _ptr(self.v), _ptr(self.grad), TCN_PARAMS,
                                 self.step_count, lr, betas[0], betas[1], eps, _stream_ptr(stream)))
        tcn_pack(self.theta, self.packed, stream)


def mse_grad(z: torch.Tensor, target: torch.Tensor, scale: float, loss: Optional[torch.Tensor] = None, stream=None):
    """gz = scale (z - target); loss (1 FP32 element) += scale/2 sum (z - target)^2."""
    gz = torch.empty_like(z)
    _check(_lib.ws_mse_grad(_ptr(z), _ptr(target), _ptr(gz), _ptr(loss), z.numel(), scale, _stream_ptr(stream)))
    return gz


def tcn_conv64(inp: torch.Tensor, wplanes: torch.Tensor, T: int, mode: int, bias=None, mask=None, stream=None):
    """One 64 -> 64 layer (mode 0: ReLU(conv + bias), zero gaps; 1: data gradient with mask)."""
    rows = inp.shape[0]
    out = torch.empty_like(inp)
    err = torch.zeros(64, dtype=torch.int32, device=inp.device)
    _check(_lib.ws_tcn_conv64(_ptr(inp), _ptr(wplanes), _ptr(bias), _ptr(mask), _ptr(out), rows, T, mode, _ptr(err),
                              _stream_ptr(stream)))
    return out, err
