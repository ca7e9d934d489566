"""Multi-precision oracle for ill-conditioned series (test infrastructure).

Same definition as the FP64 oracles, z = Omega^{-1} W x with Omega = W + D^T Lambda D
(Eq. 3; Eq. 2 for a scalar lambda), evaluated with mpmath at `dps` decimal digits. It is
for the cases where FP64 itself is not accurate enough to judge an FP32 result: with
per-day lambda spanning 1 .. 1e5 without smoothing, sparse weights and d = 3, cond(Omega)
reaches ~1e13 and the FP64 banded and dense oracles differ from each other by up to ~2e-3.
Inputs are FP64 numbers, converted exactly; the only rounding is at `dps` digits.

Only the test-suite may import it; it shares no code with the CUDA path.

Method: assemble the band of Omega exactly from its definition, then an LDL^T
elimination of the symmetric positive definite band without pivoting, forward and back
substitution (the plain textbook banded LDL^T; no reordering).
"""
from __future__ import annotations

from math import comb

import mpmath
import numpy as np


def _coeffs(d: int):
    """c_i = (-1)^(d-i) C(d, i): row k of D is c at columns k..k+d (Section 2)."""
    return [(-1) ** (d - i) * comb(d, i) for i in range(d + 1)]


def omega_band(w, lam, d: int):
    """Upper band of Omega = W + D^T Lambda D: A[t][r] = Omega[t, t+r], r = 0..d, as mpf.
    lam is a scalar (Eq. 2) or a per-day array whose entries k < T-d weight row k of D."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    c = _coeffs(d)
    lam = np.asarray(lam, dtype=np.float64)
    lrow = [mpmath.mpf(float(lam))] * max(T - d, 0) if lam.ndim == 0 else [mpmath.mpf(float(v)) for v in lam[:max(T - d, 0)]]
    A = [[mpmath.mpf(0) for _ in range(d + 1)] for _ in range(T)]
    for t in range(T):
        A[t][0] += mpmath.mpf(float(w[t]))
    for k in range(T - d):
        for i in range(d + 1):
            for j in range(i, d + 1):
                A[k + i][j - i] += lrow[k] * c[i] * c[j]
    return A


def _ldl_band(A, d: int):
    """Omega = L diag(piv) L^T for the upper band A of Omega (no pivoting); L unit lower with
    L[t+r][t] stored as Lb[t+r][r]. Raises ValueError if a pivot is not positive."""
    T = len(A)
    Lb = [[mpmath.mpf(0) for _ in range(d + 1)] for _ in range(T)]
    piv = [mpmath.mpf(0)] * T
    for t in range(T):
        s = A[t][0]
        for j in range(1, d + 1):
            if t - j >= 0:
                s -= Lb[t][j] ** 2 * piv[t - j]
        if not s > 0:
            raise ValueError(f"Omega is not positive definite (pivot {t})")
        piv[t] = s
        for r in range(1, d + 1):
            if t + r >= T:
                break
            s = A[t][r]
            # Omega[t+r, t] = sum_j L[t+r, t-j] piv[t-j] L[t, t-j]
            for j in range(1, d + 1 - r):
                if t - j >= 0:
                    s -= Lb[t + r][r + j] * Lb[t][j] * piv[t - j]
            Lb[t + r][r] = s / piv[t]
    return Lb, piv


def _ldl_solve(Lb, piv, b, d: int):
    """Omega^{-1} b from the banded LDL^T factor: forward, diagonal, back substitution."""
    T = len(b)
    y = [mpmath.mpf(0)] * T
    for t in range(T):
        s = b[t]
        for j in range(1, d + 1):
            if t - j >= 0:
                s -= Lb[t][j] * y[t - j]
        y[t] = s
    z = [mpmath.mpf(0)] * T
    for t in range(T - 1, -1, -1):
        s = y[t] / piv[t]
        for j in range(1, d + 1):
            if t + j < T:
                s -= Lb[t + j][j] * z[t + j]
        z[t] = s
    return z


def smooth_mp(x, w, lam, d: int, dps: int = 50) -> np.ndarray:
    """z = Omega^{-1} W x for one series at `dps` digits, returned rounded to FP64.
    Raises ZeroDivisionError / ValueError if Omega is not positive definite."""
    with mpmath.workdps(dps):
        x = np.asarray(x, dtype=np.float64)
        w = np.asarray(w, dtype=np.float64)
        Lb, piv = _ldl_band(omega_band(w, lam, d), d)
        b = [mpmath.mpf(float(wt)) * mpmath.mpf(float(xt)) for wt, xt in zip(w, x)]
        return np.array([float(v) for v in _ldl_solve(Lb, piv, b, d)])


def vjp_mp(w, lam, d: int, z, gz, dps: int = 50, per_day: bool = True):
    """Reverse-mode derivatives of one series at `dps` digits (Section 2.3, Eqs. 4-5):
    g_b = Omega^{-1} gz_b, dL/dx_b = W g_b, dL/dlambda_k = -sum_b (D g_b)_k (D z_b)_k for the
    rows k < T-d (zeros after; their sum for a scalar lambda). z, gz: [T] or [T, B] FP64
    values, converted exactly. Returns (gx, glam) rounded to FP64, shaped like the FP64
    oracle's vjp_one. For series where FP64 cannot resolve D g: g carries a large component
    along the polynomials D annihilates, and its FP64 rounding alone swamps D g."""
    with mpmath.workdps(dps):
        w = np.asarray(w, dtype=np.float64)
        T = w.shape[0]
        z2 = np.asarray(z, dtype=np.float64).reshape(T, -1)
        g2 = np.asarray(gz, dtype=np.float64).reshape(T, -1)
        c = _coeffs(d)
        Lb, piv = _ldl_band(omega_band(w, lam, d), d)
        gx = np.zeros_like(g2)
        rows = [mpmath.mpf(0)] * max(T - d, 0)
        for b in range(g2.shape[1]):
            g = _ldl_solve(Lb, piv, [mpmath.mpf(float(v)) for v in g2[:, b]], d)
            zz = [mpmath.mpf(float(v)) for v in z2[:, b]]
            for t in range(T):
                gx[t, b] = float(mpmath.mpf(float(w[t])) * g[t])
            for k in range(T - d):
                dg = sum(c[i] * g[k + i] for i in range(d + 1))
                dz = sum(c[i] * zz[k + i] for i in range(d + 1))
                rows[k] -= dg * dz
        if per_day:
            glam = np.zeros(T)
            glam[: max(T - d, 0)] = [float(v) for v in rows]
        else:
            glam = np.array(float(sum(rows)))
        return gx.reshape(np.shape(z)), glam


def residual_mp(x, w, lam, d: int, z, dps: int = 50) -> float:
    """max_t |(W x - Omega z)_t| / max_t |(W x)_t| at `dps` digits, from the band of Omega."""
    with mpmath.workdps(dps):
        x = np.asarray(x, dtype=np.float64)
        w = np.asarray(w, dtype=np.float64)
        T = x.shape[0]
        A = omega_band(w, lam, d)
        zz = [mpmath.mpf(float(v)) for v in z]
        worst, scale = mpmath.mpf(0), mpmath.mpf(0)
        for t in range(T):
            b = mpmath.mpf(float(w[t])) * mpmath.mpf(float(x[t]))
            s = A[t][0] * zz[t]
            for r in range(1, d + 1):
                if t + r < T:
                    s += A[t][r] * zz[t + r]
                if t - r >= 0:
                    s += A[t - r][r] * zz[t - r]
            worst = max(worst, abs(b - s))
            scale = max(scale, abs(b))
        return float(worst / scale) if scale > 0 else float(worst)
