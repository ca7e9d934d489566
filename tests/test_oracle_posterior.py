"""Pins of the posterior-spread oracle (credibility intervals, Fig. 4) against facts that
the mathematics fixes, independently of the oracle's own formula (CPU only)."""
import numpy as np
import pytest

from oracle import dense


def test_inverse_diag_closed_form_first_order_full_weights():
    """d = 1, w = 1, scalar lambda: D^T D is the path-graph Laplacian, diagonalised by the
    DCT-II basis v_j(t) = c_j cos(pi j (t + 1/2) / T) with eigenvalues 4 sin^2(pi j / 2T), so
    (Omega^{-1})_tt = sum_j v_j(t)^2 / (1 + lambda 4 sin^2(pi j / 2T))."""
    for T, lam in [(7, 0.3), (40, 25.0), (64, 1e4)]:
        t = np.arange(T)
        dg = np.zeros(T)
        for j in range(T):
            c = np.sqrt((1.0 if j == 0 else 2.0) / T)
            v = c * np.cos(np.pi * j * (t + 0.5) / T)
            dg += v * v / (1.0 + lam * 4.0 * np.sin(np.pi * j / (2 * T)) ** 2)
        got, _, _ = dense.posterior_one(np.zeros(T), np.ones(T), lam, 1)
        assert np.max(np.abs(got - dg) / dg) < 1e-11


def test_posterior_covariance_by_sampling():
    """The Bayesian reading: with the prior made proper by a tiny ridge (precision
    (D^T Lambda D + eps I) / sigma^2) and x = s + noise of precision w / sigma^2 on the valid
    days, the error s - z of the posterior mean has covariance sigma^2 Omega^{-1}. Checked on
    40,000 draws against sigma^2 diag(Omega^{-1}) (sampling error ~0.7%)."""
    rng = np.random.default_rng(7)
    T, d, sigma, eps, N = 12, 2, 0.3, 1e-6, 40000
    w = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1, 1, 0, 1], dtype=float)
    lam = 10 ** rng.uniform(-0.5, 1.0, T)
    Dm = dense.difference_matrix(T, d)
    prior_prec = Dm.T @ np.diag(dense.lam_rows(lam, T, d)) @ Dm + eps * np.eye(T)
    Lc = np.linalg.cholesky(np.linalg.inv(prior_prec))
    s = sigma * (Lc @ rng.normal(size=(T, N)))
    noise = np.where(w[:, None] > 0, sigma * rng.normal(size=(T, N)) / np.sqrt(np.maximum(w, 1e-300))[:, None], 0.0)
    x = np.where(w[:, None] > 0, s + noise, 0.0)
    Om_eps = np.diag(w) + prior_prec
    z = np.linalg.solve(Om_eps, w[:, None] * x)
    emp = np.mean((s - z) ** 2, axis=1)
    dg, _, _ = dense.posterior_one(np.zeros(T), w, lam, d)
    assert np.max(np.abs(emp / (sigma ** 2 * dg) - 1.0)) < 0.04


def test_residual_variance_unbiased_at_polynomial_limit():
    """lambda -> infinity: z is the weighted least-squares fit of a degree d-1 polynomial and
    tr H -> d, so sigma2 = RSS / (n - tr H) is the classical unbiased variance estimate: its
    mean over 3000 series of (polynomial + N(0, sigma^2)) is sigma^2 within sampling error
    (an n denominator would be 11% low here)."""
    rng = np.random.default_rng(11)
    T, d, sigma, lam = 30, 2, 0.1, 1e9
    vals, trs = [], []
    for _ in range(3000):
        w = np.zeros(T)
        w[rng.choice(T, size=18, replace=False)] = 1.0
        t = np.arange(T)
        x = 0.3 + 0.01 * t + sigma * rng.normal(size=T)
        dg, s2, _ = dense.posterior_one(x, w, lam, d)
        vals.append(s2[0])
        trs.append(float(np.sum(w * dg)))
    assert abs(np.mean(trs) - d) < 1e-5
    assert abs(np.mean(vals) / sigma ** 2 - 1.0) < 0.03


@pytest.mark.parametrize("d", [1, 2, 3])
def test_sd_scales_with_data_and_bands_are_independent(d):
    """x -> c x scales sd by |c|; a band's sigma2 depends on that band alone; diag(Omega^{-1})
    does not depend on x."""
    rng = np.random.default_rng(3 + d)
    T = 50
    w = (rng.random(T) < 0.6).astype(float)
    lam = 10 ** rng.uniform(0, 3, T)
    x = rng.normal(size=(T, 3))
    dg, s2, sd = dense.posterior_one(x, w, lam, d)
    dg2, s22, sd2 = dense.posterior_one(-2.5 * x, w, lam, d)
    assert np.allclose(dg, dg2, rtol=1e-13) and np.allclose(sd2, 2.5 * sd, rtol=1e-10)
    for b in range(3):
        _, s1, _ = dense.posterior_one(x[:, b], w, lam, d)
        assert np.isclose(s1[0], s2[b], rtol=1e-10)


def test_posterior_on_sample_times():
    """With the uneven-spacing operator: on t = 0..T-1 it is the daily posterior; on uneven
    dates the error of the posterior mean under the Bayesian model has covariance
    sigma^2 Omega^{-1} (40,000 draws against sigma^2 diag(Omega^{-1}), as for the daily grid)."""
    rng = np.random.default_rng(17)
    T, d = 14, 2
    w = (rng.random(T) < 0.6).astype(float)
    w[[0, 5, 9]] = 1.0
    lam = 10 ** rng.uniform(-0.5, 1.0, T)
    x = rng.normal(size=(T, 2))
    a = dense.posterior_one(x, w, lam, d)
    b = dense.posterior_one(x, w, lam, d, t=np.arange(T, dtype=float))
    for u, v in zip(a, b):
        assert np.allclose(u, v, rtol=1e-11, atol=1e-14)
    t = np.cumsum(rng.integers(1, 4, size=T)).astype(float)
    sigma, eps, N = 0.3, 1e-6, 40000
    Dm = dense.difference_matrix_dates(t, d)
    prior_prec = Dm.T @ np.diag(dense.lam_rows(lam, T, d)) @ Dm + eps * np.eye(T)
    Lc = np.linalg.cholesky(np.linalg.inv(prior_prec))
    s = sigma * (Lc @ rng.normal(size=(T, N)))
    noise = np.where(w[:, None] > 0, sigma * rng.normal(size=(T, N)), 0.0)
    xs = np.where(w[:, None] > 0, s + noise, 0.0)
    z = np.linalg.solve(np.diag(w) + prior_prec, w[:, None] * xs)
    emp = np.mean((s - z) ** 2, axis=1)
    dg, _, _ = dense.posterior_one(np.zeros(T), w, lam, d, t=t)
    assert np.max(np.abs(emp / (sigma ** 2 * dg) - 1.0)) < 0.04
