"""Pins for the multi-precision oracle (oracle/multiprec.py) against exact rational
arithmetic and the FP64 oracles, and a record of where FP64 stops being a reference."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import banded, dense, multiprec


def _exact_solve(x, w, lam, d, rhs=None):
    """z = Omega^{-1} W x (or Omega^{-1} rhs) in exact rationals: Omega assembled entry by
    entry from its definition W + D^T Lambda D (Eq. 3), Gauss-Jordan elimination with
    Fractions."""
    T = len(w)
    c = [Fraction(v) for v in dense.diff_coeffs(d)]
    lam = np.asarray(lam, dtype=np.float64)
    lr = [Fraction(float(lam))] * (T - d) if lam.ndim == 0 else [Fraction(float(v)) for v in lam[:T - d]]
    M = [[Fraction(0)] * T for _ in range(T)]
    for t in range(T):
        M[t][t] += Fraction(float(w[t]))
    for k in range(T - d):
        for i in range(d + 1):
            for j in range(d + 1):
                M[k + i][k + j] += lr[k] * c[i] * c[j]
    if rhs is None:
        b = [Fraction(float(w[t])) * Fraction(float(x[t])) for t in range(T)]
    else:
        b = [Fraction(float(v)) for v in rhs]
    for col in range(T):
        piv = next(r for r in range(col, T) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(T):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[col])]
                b[r] -= f * b[col]
    return [b[t] / M[t][t] for t in range(T)]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_mp_equals_exact_rational(d):
    """Dyadic inputs (exact in binary), ill-conditioned lambda mix: the 50-digit solve equals
    the exact rational solution to 1e-40 relative."""
    rng = np.random.default_rng(100 + d)
    T = 14
    x = np.round(rng.normal(size=T) * 64) / 64
    w = (rng.random(T) < 0.4).astype(float)
    w[0] = w[-1] = 1.0
    w[T // 2] = 0.5
    lam = 2.0 ** rng.integers(-4, 30, size=T).astype(float)
    zx = _exact_solve(x, w, lam, d)
    import mpmath
    with mpmath.workdps(50):
        zm = multiprec.smooth_mp(x, w, lam, d, dps=50)
    scale = max(abs(float(v)) for v in zx)
    err = max(abs(Fraction(float(a)) - b) for a, b in zip(zm, zx))
    # zm is returned rounded to FP64: the comparison is at FP64 rounding of exact values
    assert float(err) <= 2.3e-16 * scale


@pytest.mark.parametrize("d", [1, 2, 3])
def test_mp_polynomial_reproduction(d):
    """A polynomial of degree < d is left unchanged for any lambda (D annihilates it)."""
    rng = np.random.default_rng(7)
    T = 40
    t = np.arange(T, dtype=float)
    x = sum(rng.normal() * (t / T) ** p for p in range(d))
    w = (rng.random(T) < 0.5).astype(float) + 0.25
    lam = 10.0 ** rng.uniform(0, 7, T)
    z = multiprec.smooth_mp(x, w, lam, d)
    assert np.max(np.abs(z - x)) <= 1e-14 * np.max(np.abs(x))


def test_mp_agrees_with_fp64_when_well_conditioned():
    rng = np.random.default_rng(3)
    T, d = 200, 2
    x = rng.normal(size=T)
    w = np.ones(T)
    lam = 10.0 ** rng.uniform(0, 2, T)
    zm = multiprec.smooth_mp(x, w, lam, d)
    zd = dense.smooth_one(x, w, lam, d)
    assert np.max(np.abs(zm - zd)) <= 1e-12 * np.max(np.abs(zd))
    # z is rounded to FP64: the residual is bounded by u * max row sum of |Omega| * max|z|
    A = np.abs(dense.omega(w, lam, d)).sum(axis=1).max()
    assert multiprec.residual_mp(x, w, lam, d, zm) <= 1.2e-16 * A * np.max(np.abs(zm)) / np.max(np.abs(x))


def test_fp64_is_not_a_reference_at_cond_1e13():
    """Sparse 5-day weights, unsmoothed lambda = 10^U[0,5], d = 3: the two FP64 oracles
    disagree by far more than 1e-4, while 50- and 70-digit solves agree to FP64 rounding.
    This is why the ragged tests judge such series against the multi-precision solve."""
    from paper_2604_00048_b300 import synth

    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 500, t_range=(120, 600))
    off = out["offsets"].numpy()
    x, w, lam = (out[k].double().numpy() for k in ("x", "w", "lam"))
    i = 263  # d = 3, T = 528
    assert int(out["order"][i]) == 3
    a, b = off[i], off[i + 1]
    zb, st = banded.smooth_tile(x[a:b, None, None], w[a:b, None], lam[a:b, None], 3)
    zd = dense.smooth_one(x[a:b], w[a:b], lam[a:b], 3)
    z50 = multiprec.smooth_mp(x[a:b], w[a:b], lam[a:b], 3, dps=50)
    z70 = multiprec.smooth_mp(x[a:b], w[a:b], lam[a:b], 3, dps=70)
    sc = np.max(np.abs(z50))
    assert np.max(np.abs(z50 - z70)) <= 1e-15 * sc
    assert np.max(np.abs(zb[:, 0, 0] - zd)) / sc > 1e-4
    assert max(np.max(np.abs(zb[:, 0, 0] - z50)), np.max(np.abs(zd - z50))) / sc > 1e-4


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_vjp_mp_equals_exact_rational(d):
    """Dyadic inputs, ill-conditioned lambda mix: the 50-digit VJP (g = Omega^{-1} gz,
    W g, -(D g)_k (D z)_k summed over two bands) equals the one computed from the exact
    rational solve, to the FP64 rounding of the returned values. The exact side solves by
    Gauss-Jordan on the dense Omega and applies D as the matrix of dense.difference_matrix
    (rows of binomial coefficients), so it shares neither the banded LDL^T nor the
    coefficient loop of the oracle."""
    rng = np.random.default_rng(200 + d)
    T, B = 13, 2
    w = (rng.random(T) < 0.4).astype(float)
    w[0] = w[-1] = 1.0
    w[T // 2] = 0.5
    lam = 2.0 ** rng.integers(-4, 30, size=T).astype(float)
    z = np.round(rng.normal(size=(T, B)) * 256) / 256
    gz = np.round(rng.normal(size=(T, B)) * 256) / 256
    Dm = dense.difference_matrix(T, d).astype(int)
    rows = [Fraction(0)] * (T - d)
    gx_exact = np.zeros((T, B), dtype=object)
    for b in range(B):
        g = _exact_solve(None, w, lam, d, rhs=gz[:, b])
        for t in range(T):
            gx_exact[t, b] = Fraction(float(w[t])) * g[t]
        for k in range(T - d):
            dg = sum(int(Dm[k, j]) * g[j] for j in range(T))
            dz = sum(int(Dm[k, j]) * Fraction(float(z[j, b])) for j in range(T))
            rows[k] -= dg * dz
    gx, glam = multiprec.vjp_mp(w, lam, d, z, gz)
    sx = max(abs(float(v)) for v in gx_exact.ravel())
    assert max(abs(Fraction(float(a)) - b) for a, b in zip(gx.ravel(), gx_exact.ravel())) <= 2.3e-16 * sx
    sl = max(abs(float(v)) for v in rows)
    assert max(abs(Fraction(float(a)) - b) for a, b in zip(glam[:T - d], rows)) <= 2.3e-16 * sl
    assert np.all(glam[T - d:] == 0)
    _, gsum = multiprec.vjp_mp(w, lam, d, z, gz, per_day=False)
    assert abs(Fraction(float(gsum)) - sum(rows)) <= 2.3e-16 * max(sl, abs(float(sum(rows)))) * (T - d)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_vjp_mp_agrees_with_fp64_when_well_conditioned(d):
    """Daily weights and lambda in [1, 100]: the 50-digit VJP equals the dense FP64 oracle's
    (whose Eqs. 4-5 are pinned by finite differences and the dot-product identity)."""
    rng = np.random.default_rng(30 + d)
    T = 80
    w = (rng.random(T) < 0.7).astype(float)
    lam = 10.0 ** rng.uniform(0, 2, T)
    z = rng.normal(size=(T, 3))
    gz = rng.normal(size=(T, 3))
    gxm, glm = multiprec.vjp_mp(w, lam, d, z, gz)
    gxd, gld = dense.vjp_one(w, lam, d, z, gz)
    assert np.max(np.abs(gxm - gxd)) <= 1e-11 * np.max(np.abs(gxd))
    assert np.max(np.abs(glm - gld)) <= 1e-11 * np.max(np.abs(gld))
