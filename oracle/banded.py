"""ctypes front-end of oracle/banded.c (Algorithm 1 in FP64 C): test infrastructure only."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "banded.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_banded.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile banded.c with gcc -O2 -fopenmp into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        _lib.wh_banded_smooth_tile.restype = ctypes.c_long
        _lib.wh_banded_smooth_tile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                               dp, dp, dp, ctypes.c_int, dp, u8p, ctypes.c_int]
        _lib.wh_banded_vjp_tile.restype = ctypes.c_long
        _lib.wh_banded_vjp_tile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                            dp, dp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, u8p,
                                            ctypes.c_int]
        _lib.wh_banded_factor_one.restype = ctypes.c_int
        _lib.wh_banded_factor_one.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.wh_banded_assemble_one.restype = None
        _lib.wh_banded_assemble_one.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        _lib.wh_banded_max_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def smooth_tile(x, w, lam, d: int, nthreads: int = 0):
    """Tile layout x[t,b,p], w[t,p], lam[t,p] or lam[p] -> (z[t,b,p], status[p])."""
    x, w, lam = _c64(x), _c64(w), _c64(lam)
    T, B, P = x.shape
    z = np.zeros_like(x)
    st = np.zeros(P, dtype=np.uint8)
    lib().wh_banded_smooth_tile(T, d, B, P, _p(x), _p(w), _p(lam), int(lam.ndim == 1), _p(z),
                                st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nthreads)
    return z, st


def vjp_tile(w, lam, d: int, z, gz, log_lambda: bool = False, nthreads: int = 0):
    """Tile-layout VJP -> (gx[t,b,p], glam[t,p] or [p], status[p])."""
    w, lam, z, gz = _c64(w), _c64(lam), _c64(z), _c64(gz)
    T, B, P = z.shape
    gx = np.zeros_like(z)
    glam = np.zeros((T, P)) if lam.ndim == 2 else np.zeros(P)
    st = np.zeros(P, dtype=np.uint8)
    lib().wh_banded_vjp_tile(T, d, B, P, _p(w), _p(lam), int(lam.ndim == 1), _p(z), _p(gz), _p(gx),
                             _p(glam), int(log_lambda),
                             st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nthreads)
    return gx, glam, st


def factor_one(w, lam_rows, d: int):
    """Band after Algorithm 1 for one series: ab[j, t] = L[t+j, t]; returns (ab, status)."""
    w = _c64(w)
    T = w.shape[0]
    lk = np.zeros(T)
    lk[: len(lam_rows)] = lam_rows
    ab = np.zeros((d + 1) * T)
    st = lib().wh_banded_factor_one(T, d, _p(w), _p(lk), _p(ab))
    return ab.reshape(d + 1, T), st


def assemble_one(w, lam_rows, d: int):
    """Omega in lower band storage for one series: ab[j, t] = Omega[t+j, t]."""
    w = _c64(w)
    T = w.shape[0]
    lk = np.zeros(T)
    lk[: len(lam_rows)] = lam_rows
    ab = np.zeros((d + 1) * T)
    lib().wh_banded_assemble_one(T, d, _p(w), _p(lk), _p(ab))
    return ab.reshape(d + 1, T)


def max_threads() -> int:
    return int(lib().wh_banded_max_threads())
