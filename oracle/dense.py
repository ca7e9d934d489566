"""Dense FP64 oracle for the Whittaker-Henderson smoother (test infrastructure).

This is the plain, slow, obviously correct CPU statement of what the GPU path
computes. Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does. It shares no code with the
CUDA path: it builds the full T x T matrices and calls LAPACK.

Notation (Section 2 of the paper): x in R^T observations, W = diag(w) observation
weights, D in R^{(T-d) x T} the order-d difference operator (the paper's order
k+1, written d here), Lambda = diag(lam_0 .. lam_{T-d-1}) per-row smoothing
weights, Omega = W + D^T Lambda D (Section 3).

Readings of the paper used here (each one also appears in the design notes):
  * Lambda has one entry per row of D; the per-day input array has length T and
    its last d entries are ignored (their gradient is 0).
  * D is the unscaled binomial forward difference on a regular daily grid.
  * Eq. 5 prints W Omega^{-1}; the vector-Jacobian product is dL/dx = W Omega^{-1} g.
  * GCV (not defined in the paper) is the Craven-Wahba score
    V = n_eff * RSS / (n_eff - tr H)^2 with H = Omega^{-1} W, summed over bands.
"""
from __future__ import annotations

from math import comb

import numpy as np
import scipy.linalg as sla


def diff_coeffs(d: int) -> np.ndarray:
    """c_i = (-1)^(d-i) C(d, i), i = 0..d: row k of D is c at columns k..k+d (Section 2)."""
    return np.array([(-1) ** (d - i) * comb(d, i) for i in range(d + 1)], dtype=np.float64)


def difference_matrix(T: int, d: int) -> np.ndarray:
    """The order-d discrete difference operator D in R^{(T-d) x T} (Section 2)."""
    c = diff_coeffs(d)
    D = np.zeros((max(T - d, 0), T), dtype=np.float64)
    for k in range(T - d):
        D[k, k:k + d + 1] = c
    return D


def difference_matrix_dates(t, d: int) -> np.ndarray:
    """The order-d discrete difference operator on unevenly spaced sample times t_0 < ... <
    t_{T-1} (Section 2 takes the discrete-derivative construction of the divided-difference
    literature it cites for uneven spacing): row k is d! times the weights of the divided
    difference f[t_k, ..., t_{k+d}],
        c_{k,j} = d! / prod_{m != j} (t_{k+j} - t_{k+m}),   j = 0..d.
    On t = 0, 1, ..., T-1 this is the binomial difference matrix."""
    t = np.asarray(t, dtype=np.float64)
    T = t.shape[0]
    D = np.zeros((max(T - d, 0), T), dtype=np.float64)
    fact = float(np.prod(np.arange(1, d + 1)))
    for k in range(T - d):
        for j in range(d + 1):
            den = 1.0
            for m in range(d + 1):
                if m != j:
                    den *= t[k + j] - t[k + m]
            D[k, k + j] = fact / den
    return D


def omega_dates(w, lam, d: int, t) -> np.ndarray:
    """Omega = W + D^T Lambda D with D on the sample times t (difference_matrix_dates)."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    D = difference_matrix_dates(t, d)
    return np.diag(w) + D.T @ (lam_rows(lam, T, d)[:, None] * D)


def smooth_one_dates(x, w, lam, d: int, t) -> np.ndarray:
    """z = Omega^{-1} W x with the uneven-spacing operator (dense Cholesky; x [T] or [T, B])."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    L = np.linalg.cholesky(omega_dates(w, lam, d, t))
    wx = np.where(w[:, None] > 0, w[:, None] * np.nan_to_num(x.reshape(len(w), -1)), 0.0)
    y = sla.solve_triangular(L, wx, lower=True)
    return sla.solve_triangular(L.T, y, lower=False).reshape(x.shape)


def vjp_one_dates(w, lam, d: int, t, z, gz, per_day: bool = True):
    """Reverse-mode derivatives through z = Omega^{-1} W x with the uneven-spacing operator
    (Section 2.3 on sample times t): g = Omega^{-1} dL/dz, dL/dx = W g (Eq. 5, transposed),
    dL/dlam_k = -sum_b (D g_b)_k (D z_b)_k (Eq. 4, k < T-d; zeros after, or the sum over k
    for a scalar lambda)."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    z2 = np.asarray(z, dtype=np.float64).reshape(T, -1)
    L = np.linalg.cholesky(omega_dates(w, lam, d, t))
    r = np.asarray(gz, dtype=np.float64).reshape(T, -1)
    g2 = sla.solve_triangular(L.T, sla.solve_triangular(L, r, lower=True), lower=False)
    D = difference_matrix_dates(t, d)
    rows = -np.sum((D @ g2) * (D @ z2), axis=1)
    if per_day:
        glam = np.zeros(T)
        glam[: T - d] = rows
    else:
        glam = np.array(rows.sum())
    return (w[:, None] * g2).reshape(np.shape(z)), glam


def lam_rows(lam, T: int, d: int) -> np.ndarray:
    """Diagonal of Lambda (length T-d) from a scalar (Eq. 2) or a length-T per-day array (Eq. 3)."""
    lam = np.asarray(lam, dtype=np.float64)
    if lam.ndim == 0:
        return np.full(max(T - d, 0), float(lam))
    return lam[: max(T - d, 0)].copy()


def omega(w, lam, d: int) -> np.ndarray:
    """Omega = W + D^T Lambda D (Eq. 3; Eq. 2 when lam is a scalar)."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    D = difference_matrix(T, d)
    return np.diag(w) + D.T @ (lam_rows(lam, T, d)[:, None] * D)


def smooth_one(x, w, lam, d: int) -> np.ndarray:
    """z = Omega^{-1} W x for one series; x may be [T] or [T, B] (bands as right-hand sides).

    Dense Cholesky Omega = L L^T, then L y = W x and L^T z = y (Section 3.1).
    Raises numpy.linalg.LinAlgError when Omega is not positive definite."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    O = omega(w, lam, d)
    L = np.linalg.cholesky(O)
    wx = np.where(w[:, None] > 0, w[:, None] * np.nan_to_num(x.reshape(len(w), -1)), 0.0)
    y = sla.solve_triangular(L, wx, lower=True)
    z = sla.solve_triangular(L.T, y, lower=False)
    return z.reshape(x.shape)


def solve_one(w, lam, d: int, rhs) -> np.ndarray:
    """g = Omega^{-1} rhs (rhs [T] or [T, B])."""
    O = omega(w, lam, d)
    L = np.linalg.cholesky(O)
    r = np.asarray(rhs, dtype=np.float64).reshape(O.shape[0], -1)
    y = sla.solve_triangular(L, r, lower=True)
    return sla.solve_triangular(L.T, y, lower=False).reshape(np.shape(rhs))


def vjp_one(w, lam, d: int, z, gz, per_day: bool = True):
    """Reverse-mode derivatives of L(z) through z = Omega^{-1} W x (Section 2.3).

    g = Omega^{-1} dL/dz (Omega is symmetric), then
      dL/dx_b     = W g_b                                  (Eq. 5, transposed)
      dL/dlam_k   = - sum_b (d_k^T g_b)(d_k^T z_b)          (Eq. 4, k < T-d)
    Per-day lambda: returns an array of length T with zeros in the last d entries.
    Scalar lambda: returns the sum over k (lambda multiplies every row of D)."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    z2 = np.asarray(z, dtype=np.float64).reshape(T, -1)
    g2 = solve_one(w, lam, d, np.asarray(gz, dtype=np.float64).reshape(T, -1))
    gx = w[:, None] * g2
    D = difference_matrix(T, d)
    glam_rows = -np.sum((D @ g2) * (D @ z2), axis=1)
    if per_day:
        glam = np.zeros(T)
        glam[: T - d] = glam_rows
    else:
        glam = np.array(glam_rows.sum())
    return gx.reshape(np.shape(z)), glam


def vjp_w_one(x, w, lam, d: int, z, gz):
    """dL/dw through z = Omega^{-1} W x, the weights of the objective (Eq. 1) taken as
    parameters (soft weights). Differentiating Omega z = W x in w_t: e_t z_t + Omega dz =
    e_t x_t, so dz/dw_t = Omega^{-1} e_t (x_t - z_t) and, with g = Omega^{-1} dL/dz
    (Omega symmetric), dL/dw_t = sum_b g_tb (x_tb - z_tb). A day with w_t = 0 contributes
    x_t = 0 (the smoother ignores the value observed there). Returns an array of length T."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    x2 = np.where(w[:, None] > 0, np.asarray(x, dtype=np.float64).reshape(T, -1), 0.0)
    z2 = np.asarray(z, dtype=np.float64).reshape(T, -1)
    g2 = solve_one(w, lam, d, np.asarray(gz, dtype=np.float64).reshape(T, -1))
    return np.sum(g2 * (x2 - z2), axis=1)


def vjp_w_tile(x, w, lam, d: int, z, gz):
    """Tile layout: x, z, gz [t, b, p], w [t, p], lam [t, p] or [p]. Returns dL/dw [t, p],
    zero for series whose Omega is not positive definite."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    gz = np.asarray(gz, dtype=np.float64)
    T, B, P = x.shape
    gw = np.zeros((T, P))
    for p in range(P):
        lp = lam[p] if lam.ndim == 1 else lam[:, p]
        if is_pd(w[:, p], lp, d):
            gw[:, p] = vjp_w_one(x[:, :, p], w[:, p], lp, d, z[:, :, p], gz[:, :, p])
    return gw


def is_pd(w, lam, d: int) -> bool:
    """Omega = W + D^T Lambda D is positive definite iff every lambda row weight is > 0
    (finite), every w >= 0 (finite), and at least min(d, T) weights are positive: the
    null space of D^T Lambda D is the polynomials of degree < d, and a nonzero one has
    fewer than d roots. (Deciding this by attempting a Cholesky factorisation is not
    reliable: on an exactly singular Omega rounding can leave every pivot positive.)"""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    lr = lam_rows(lam, T, d)
    if not (np.all(np.isfinite(w)) and np.all(w >= 0) and np.all(np.isfinite(lr)) and np.all(lr > 0)):
        return False
    return int(np.sum(w > 0)) >= min(d, T)


def smooth_tile(x, w, lam, d: int):
    """Batch over pixels in the tile layout x[t, b, p], w[t, p], lam[t, p] or lam[p].

    Returns (z[t, b, p], ok[p]); series whose Omega is not positive definite (is_pd)
    get ok = False and z = 0."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    T, B, P = x.shape
    z = np.zeros_like(x)
    ok = np.ones(P, dtype=bool)
    for p in range(P):
        lp = lam[p] if lam.ndim == 1 else lam[:, p]
        if not is_pd(w[:, p], lp, d):
            ok[p] = False
            continue
        z[:, :, p] = smooth_one(x[:, :, p], w[:, p], lp, d)
    return z, ok


def vjp_tile(w, lam, d: int, z, gz, log_lambda: bool = False):
    """Tile-layout VJP: returns (gx[t,b,p], glam[t,p]); with log_lambda, dL/dlog(lam) = lam * dL/dlam.
    Series whose Omega is not positive definite (is_pd) get zeros."""
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    gz = np.asarray(gz, dtype=np.float64)
    T, B, P = z.shape
    gx = np.zeros_like(z)
    glam = np.zeros((T, P)) if lam.ndim == 2 else np.zeros(P)
    for p in range(P):
        lp = lam[p] if lam.ndim == 1 else lam[:, p]
        if not is_pd(w[:, p], lp, d):
            continue                       # singular Omega: gradients zero-filled
        a, b = vjp_one(w[:, p], lp, d, z[:, :, p], gz[:, :, p], per_day=(lam.ndim == 2))
        gx[:, :, p] = a
        if lam.ndim == 2:
            glam[:, p] = b * lp if log_lambda else b
        else:
            glam[p] = b * lp if log_lambda else b
    return gx, glam


def masked_mse(z, target, mask, scale: float):
    """The training loss of Section 4.3 (mean squared error of z against held-out
    observations), as a weighted sum: per series p, L_p = scale/2 * sum_{t,b} m_tp (z_tbp -
    target_tbp)^2 with day weights m (1 on held-out days, 0 elsewhere; None: all ones), and
    its gradient dL/dz = scale * m * (z - target). With scale = 2 / (number of held-out
    entries) the sum of L_p over the series is their mean squared error. Days with m = 0
    contribute nothing whatever the target holds there. Returns (L [P], gz [T, B, P])."""
    z = np.asarray(z, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    T, B, P = z.shape
    m = np.ones((T, P)) if mask is None else np.asarray(mask, dtype=np.float64)
    e = np.where(m[:, None, :] > 0, z - np.nan_to_num(target), 0.0)
    gz = scale * m[:, None, :] * e
    loss = 0.5 * scale * np.sum(m[:, None, :] * e * e, axis=(0, 1))
    return loss, gz


def hat_trace(w, lam, d: int, t=None) -> float:
    """tr H with H = Omega^{-1} W: sum_t w_t (Omega^{-1})_tt, from the dense inverse (t: sample
    times for the uneven-spacing operator, None for the daily grid)."""
    w = np.asarray(w, dtype=np.float64)
    Oi = np.linalg.inv(omega(w, lam, d) if t is None else omega_dates(w, lam, d, t))
    return float(np.sum(w * np.diag(Oi)))


def inverse_diag(w, lam, d: int) -> np.ndarray:
    """diag(Omega^{-1}) from the dense inverse."""
    return np.diag(np.linalg.inv(omega(np.asarray(w, dtype=np.float64), lam, d))).copy()


def gcv_one(x, w, lam_grid, d: int, t=None):
    """Grid search of a scalar lambda by generalized cross-validation.

    For each grid value: z = Omega^{-1} W x (bands as right-hand sides),
    RSS = sum_b sum_t w_t (x_tb - z_tb)^2, tr H = sum_t w_t (Omega^{-1})_tt,
    n = sum_t w_t, and V = (n B) RSS / (n B - B tr H)^2. The smallest V wins;
    ties go to the smaller lambda. t: sample times for the uneven-spacing operator (None: the
    daily grid). Returns (best index, scores, z at the best)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    x2 = x.reshape(T, -1)
    B = x2.shape[1]
    n = float(np.sum(w))
    scores = []
    solve = (lambda lv: smooth_one(x2, w, lv, d)) if t is None else (lambda lv: smooth_one_dates(x2, w, lv, d, t))
    for lam in lam_grid:
        z = solve(float(lam))
        rss = float(np.sum(w[:, None] * (np.where(w[:, None] > 0, x2, 0.0) - z) ** 2))
        tr = hat_trace(w, float(lam), d, t)
        scores.append(n * B * rss / (n * B - B * tr) ** 2)
    scores = np.array(scores)
    best = int(np.argmin(scores))          # argmin returns the first (smallest lambda) on ties
    zb = solve(float(lam_grid[best])).reshape(x.shape)
    return best, scores, zb


def posterior_one(x, w, lam, d: int, z=None, t=None):
    """Posterior spread of the smooth, the credibility intervals of Fig. 4 (the paper takes
    them from the Bayesian reading of the smoother it cites and does not restate them).

    Reading: z is the posterior mean of the Gaussian model in which, on days with w_t > 0,
    x_t given the signal s has precision w_t / sigma^2, and s has the (improper) prior density
    proportional to exp(-s^T D^T Lambda D s / (2 sigma^2)). The posterior covariance of s is
    then sigma^2 Omega^{-1}. sigma^2 is estimated per band by the residual variance
    RSS_b / (n - tr H), RSS_b = sum_t w_t (x_tb - z_tb)^2, n = sum_t w_t, tr H =
    sum_t w_t (Omega^{-1})_tt (H = Omega^{-1} W, the hat matrix).

    x: [T] or [T, B]; z: the smooth (computed here when None); t: sample times for the
    uneven-spacing operator (None: the daily grid). Returns (diag(Omega^{-1}) [T], sigma2 [B],
    sd [T, B]) with sd_tb = sqrt(sigma2_b (Omega^{-1})_tt); the interval at level q is
    z +- q sd."""
    w = np.asarray(w, dtype=np.float64)
    T = w.shape[0]
    x2 = np.asarray(x, dtype=np.float64).reshape(T, -1)
    if z is None:
        z = smooth_one(x2, w, lam, d) if t is None else smooth_one_dates(x2, w, lam, d, t)
    z2 = np.asarray(z, dtype=np.float64).reshape(T, -1)
    Oi = np.linalg.inv(omega(w, lam, d) if t is None else omega_dates(w, lam, d, t))
    dg = np.diag(Oi).copy()
    n = float(np.sum(w))
    trh = float(np.sum(w * dg))
    xv = np.where(w[:, None] > 0, x2, 0.0)
    rss = np.sum(w[:, None] * (xv - z2) ** 2, axis=0)
    sigma2 = rss / (n - trh)
    sd = np.sqrt(sigma2[None, :] * dg[:, None])
    return dg, sigma2, sd


def posterior_tile(x, w, lam, d: int, z=None, t=None):
    """Tile layout: x, z [t, b, p], w [t, p], lam [t, p] or [p], t (sample times) [t, p] or
    None. Returns (diag [t, p],
    sigma2 [b, p], sd [t, b, p], ok [p]); series whose Omega is not positive definite get
    zeros and ok = False."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    T, B, P = x.shape
    dg = np.zeros((T, P))
    s2 = np.zeros((B, P))
    sd = np.zeros((T, B, P))
    ok = np.zeros(P, dtype=bool)
    for p in range(P):
        lp = lam[p] if lam.ndim == 1 else lam[:, p]
        if not is_pd(w[:, p], lp, d):
            continue
        ok[p] = True
        zp = None if z is None else np.asarray(z, dtype=np.float64)[:, :, p]
        tp = None if t is None else np.asarray(t, dtype=np.float64)[:, p]
        dg[:, p], s2[:, p], sd[:, :, p] = posterior_one(x[:, :, p], w[:, p], lp, d, zp, tp)
    return dg, s2, sd, ok


def mse_maxe(z, x, w):
    """Reconstruction metrics of Section 4.4: MSE = T^-1 sum_t W_tt (z_t - x_t)^2 and
    MaxE = max_t W_tt |z_t - x_t|."""
    z = np.asarray(z, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    r = w * np.abs(z - np.where(w > 0, x, 0.0))
    return float(np.sum(w * (z - np.where(w > 0, x, 0.0)) ** 2) / z.shape[0]), float(np.max(r))


def rel_err(a, b, axis_t: int = 0) -> float:
    """Max over series/bands of ||a - b||_inf / max(||b||_inf, 1e-6), the inf-norm taken over time."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.max(np.abs(a - b), axis=axis_t)
    den = np.maximum(np.max(np.abs(b), axis=axis_t), 1e-6)
    return float(np.max(num / den)) if num.size else 0.0
