"""Pins of the FP64 oracle against facts the paper and mathematics fix (CPU only)."""
import os

import numpy as np
import pytest
import scipy.fft as sfft
import sympy as sp

from oracle import banded, dense

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_case(rng, T, d, B=1, p=0.5, lam_lo=-1, lam_hi=3, scalar=False):
    w = (rng.random(T) < p).astype(float)
    w[rng.choice(T, size=min(T, d + 1), replace=False)] = 1.0
    x = rng.normal(size=(T, B)) if B > 1 else rng.normal(size=T)
    lam = 10 ** rng.uniform(lam_lo, lam_hi) if scalar else 10 ** rng.uniform(lam_lo, lam_hi, T)
    return x, w, lam


def _sym_diff(z, d):
    """d-th forward difference defined recursively (textbook definition, no binomials)."""
    v = list(z)
    for _ in range(d):
        v = [v[i + 1] - v[i] for i in range(len(v) - 1)]
    return v


@pytest.mark.parametrize("d", [1, 2, 3])
def test_objective_stationarity_exact(d):
    """Eq. 3 solves the minimisation of the (weighted-penalty) objective of Eq. 1:
    the exact rational minimiser from sympy (gradient of the objective = 0) equals the oracle."""
    T = 6
    rs = np.random.default_rng(d)
    xs = [sp.Rational(int(v), 7) for v in rs.integers(-20, 20, T)]
    ws = [1, 0, 1, 1, 0, 1]
    ls = [sp.Rational(int(v), 3) for v in rs.integers(1, 30, T - d)]
    z = sp.symbols(f"z0:{T}")
    J = sum(ws[t] * (xs[t] - z[t]) ** 2 for t in range(T))
    J += sum(ls[k] * dk ** 2 for k, dk in enumerate(_sym_diff(z, d)))
    sol = sp.solve([sp.diff(J, zi) for zi in z], z, dict=True)[0]
    exact = np.array([float(sol[zi]) for zi in z])
    lam = np.zeros(T)
    lam[: T - d] = [float(v) for v in ls]
    got = dense.smooth_one(np.array([float(v) for v in xs]), np.array(ws, float), lam, d)
    assert np.max(np.abs(got - exact)) <= 1e-12 * max(1.0, np.max(np.abs(exact)))


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_stacked_least_squares(rng, d):
    """z also solves min ||sqrt(W)(x - z)||^2 + ||sqrt(Lambda) D z||^2 as a stacked
    least-squares problem, solved by SVD with D from numpy.diff (independent of the oracle's D)."""
    T = 40
    x, w, lam = _rand_case(rng, T, d)
    Dn = np.diff(np.eye(T), n=d, axis=0)
    A = np.vstack([np.sqrt(w)[:, None] * np.eye(T), np.sqrt(lam[: T - d])[:, None] * Dn])
    rhs = np.concatenate([np.sqrt(w) * x, np.zeros(T - d)])
    ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
    got = dense.smooth_one(x, w, lam, d)
    assert dense.rel_err(got, ref) <= 1e-9


@pytest.mark.parametrize("lam", [0.1, 3.0, 250.0])
def test_dct_closed_form_first_order(rng, lam):
    """d = 1, w = 1: D^T D is the Neumann Laplacian, diagonalised by the DCT-II with
    eigenvalues 4 sin^2(pi j / 2T); z = DCT^-1[X_j / (1 + lam 4 sin^2(pi j / 2T))]."""
    T = 64
    x = rng.normal(size=T)
    j = np.arange(T)
    X = sfft.dct(x, type=2, norm="ortho")
    ref = sfft.idct(X / (1.0 + lam * 4.0 * np.sin(np.pi * j / (2 * T)) ** 2), type=2, norm="ortho")
    got = dense.smooth_one(x, np.ones(T), lam, 1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    tr_ref = np.sum(1.0 / (1.0 + lam * 4.0 * np.sin(np.pi * j / (2 * T)) ** 2))
    assert abs(dense.hat_trace(np.ones(T), lam, 1) - tr_ref) <= 1e-9 * tr_ref


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_polynomial_reproduction(rng, d):
    """A polynomial of degree < d lies in the null space of D: it is reproduced on
    every day, gaps included, for any lambda and any W with at least d valid days."""
    T = 50
    t = np.arange(T) / T
    poly = np.polyval(rng.normal(size=d), t)
    # exactly d valid days makes Omega ill-conditioned (cond up to ~1e10 in FP64), so the
    # bound follows the condition number; a wrong difference coefficient gives O(1) errors
    for nvalid in (d, 3 * d):
        w = np.zeros(T)
        w[rng.choice(T, size=nvalid, replace=False)] = 1.0
        for lam in [1e-2, 1.0, 1e4, 10 ** rng.uniform(-2, 4, T)]:
            got = dense.smooth_one(poly * w, w, lam, d)
            tol = max(1e-12, 1e-13 * np.linalg.cond(dense.omega(w, lam, d)))
            assert np.max(np.abs(got - poly)) <= tol


def test_lambda_to_zero_returns_x(rng):
    T, d = 30, 2
    x = rng.normal(size=T)
    errs = [np.max(np.abs(dense.smooth_one(x, np.ones(T), lam, d) - x)) for lam in (1e-4, 1e-6)]
    assert errs[1] <= 1e-4
    assert errs[1] < errs[0] * 0.05          # error shrinks like lambda


@pytest.mark.parametrize("d", [1, 2, 3])
def test_lambda_to_infinity_weighted_polyfit(rng, d):
    """lambda -> infinity: z tends to the weighted least-squares polynomial of degree d-1."""
    T = 40
    t = np.arange(T, dtype=float)
    x = rng.normal(size=T)
    w = (rng.random(T) < 0.6).astype(float)
    w[:d + 1] = 1.0
    V = np.vander(t / T, d)
    coef = np.linalg.lstsq(np.sqrt(w)[:, None] * V, np.sqrt(w) * x, rcond=None)[0]
    fit = V @ coef
    e6 = np.max(np.abs(dense.smooth_one(x * w, w, 1e6, d) - fit))
    e8 = np.max(np.abs(dense.smooth_one(x * w, w, 1e8, d) - fit))
    assert e8 <= 1e-3 and e8 < e6 * 0.05


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_structure_symmetric_banded_pd(rng, d):
    """Omega is symmetric with bandwidth d (Section 3), positive definite iff at least
    d weights are positive (lambda > 0)."""
    T = 25
    lam = 10 ** rng.uniform(0, 3, T)
    w = np.zeros(T)
    w[rng.choice(T, size=d, replace=False)] = 1.0
    O = dense.omega(w, lam, d)
    assert np.max(np.abs(O - O.T)) <= 1e-14 * np.max(np.abs(O))
    i, j = np.indices(O.shape)
    assert np.all(O[np.abs(i - j) > d] == 0)
    assert np.min(np.linalg.eigvalsh(O)) > 0
    np.linalg.cholesky(O)
    w2 = w.copy()
    w2[np.flatnonzero(w2)[0]] = 0.0              # d - 1 weights: singular
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(dense.omega(w2, lam, d) - 1e-9 * np.eye(T))
    assert np.min(np.linalg.eigvalsh(dense.omega(w2, lam, d))) < 1e-6


def test_band_storage_matches_fig2():
    """Band layout of Fig. 2 (Section 3.1), T = 4, bandwidth 1 (golden fixture)."""
    T, d = 4, 1
    w = np.array([1.0, 2.0, 3.0, 4.0])
    lam = np.array([5.0, 6.0, 7.0])
    O = dense.omega(w, np.concatenate([lam, [0.0]]), d)
    ab = banded.assemble_one(w, lam, d)
    rows = [l.split() for l in open(os.path.join(GOLD, "fig2_band_storage.txt")) if not l.startswith("#")]
    assert len(rows) == (d + 1) * T
    for j, t, fi, fj in rows:
        j, t = int(j), int(t)
        if fi == "pad":
            assert ab[j, t] == 0.0
        else:
            assert ab[j, t] == O[int(fi) - 1, int(fj) - 1]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_algorithm1_equals_dense_cholesky(rng, d):
    """Algorithm 1 run on band storage gives the dense Cholesky factor."""
    for T in (d + 1, 17, 200):
        _, w, lam = _rand_case(rng, T, d)
        L = np.linalg.cholesky(dense.omega(w, lam, d))
        ab, st = banded.factor_one(w, lam[: T - d], d)
        assert st == 0
        for j in range(d + 1):
            ref = np.diagonal(L, -j)
            assert np.max(np.abs(ab[j, : T - j] - ref)) <= 1e-10 * np.max(np.abs(L))
            assert np.all(ab[j, T - j:] == 0.0)


@pytest.mark.parametrize("d,B,scalar", [(1, 1, False), (2, 3, False), (3, 2, True), (4, 1, False), (2, 10, False)])
def test_banded_tile_equals_dense(rng, d, B, scalar):
    T, P = 70, 9
    x = rng.normal(size=(T, B, P))
    w = (rng.random((T, P)) < 0.4).astype(float)
    w[:d + 1] = 1.0
    lam = 10 ** rng.uniform(0, 3, P) if scalar else 10 ** rng.uniform(0, 3, (T, P))
    z1, ok = dense.smooth_tile(x, w, lam, d)
    z2, st = banded.smooth_tile(x, w, lam, d)
    assert ok.all() and not st.any()
    assert dense.rel_err(z2, z1) <= 1e-9
    gz = rng.normal(size=(T, B, P))
    a1, b1 = dense.vjp_tile(w, lam, d, z1, gz, log_lambda=True)
    a2, b2, _ = banded.vjp_tile(w, lam, d, z1, gz, log_lambda=True)
    assert dense.rel_err(a2, a1) <= 1e-9
    assert np.max(np.abs(b2 - b1)) <= 1e-9 * np.max(np.abs(b1))


def test_status_for_singular_and_invalid(rng):
    T, d = 20, 2
    x = rng.normal(size=(T, 1, 4))
    w = np.zeros((T, 4))
    w[3, 0] = 1.0                 # one weight < d: not PD
    w[:, 1] = 1.0
    w[:, 2] = 1.0
    w[:, 3] = 1.0
    lam = np.ones((T, 4))
    lam[5, 2] = -1.0              # invalid lambda
    w[7, 3] = np.nan              # invalid weight
    z, st = banded.smooth_tile(x, w, lam, d)
    assert list(st) == [1, 0, 3, 3]
    assert np.all(z[:, :, [0, 2, 3]] == 0.0)


def test_linearity_scale_invariance_band_independence(rng):
    T, d = 45, 2
    x, w, lam = _rand_case(rng, T, d, B=3)
    z = dense.smooth_one(x, w, lam, d)
    a, b = 0.7, -2.5
    z2 = dense.smooth_one(a * x[:, 0] + b * x[:, 1], w, lam, d)
    assert np.max(np.abs(z2 - (a * z[:, 0] + b * z[:, 1]))) <= 1e-10
    z3 = dense.smooth_one(x, 3.0 * w, 3.0 * lam, d)          # (cW, c Lambda)
    assert np.max(np.abs(z3 - z)) <= 1e-10
    for k in range(3):
        assert np.max(np.abs(dense.smooth_one(x[:, k], w, lam, d) - z[:, k])) <= 1e-12


def test_vjp_finite_differences(rng):
    """Eqs. 4-5 against FP64 fourth-order central finite differences on L = <gz, z>:
    dL/dx and dL/dlog(lambda), T = 60, 4 bands, per-day lambda. FD resolves about
    cond(Omega) * eps / h (~1e-8 here), so the bound is 1e-6 of the largest entry;
    a sign error, a dropped term or a shifted difference row is an O(1) error."""
    T, B, d = 60, 4, 2

    def fd4(f, h):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    for _ in range(8):
        x, w, lam = _rand_case(rng, T, d, B=B, p=0.35, lam_lo=1, lam_hi=4)
        gz = rng.normal(size=(T, B))
        z = dense.smooth_one(x, w, lam, d)
        gx, glam = dense.vjp_one(w, lam, d, z, gz)
        L = lambda xx, ll: float(np.sum(gz * dense.smooth_one(xx, w, ll, d)))
        for t in rng.choice(T, 6, replace=False):
            for b in range(B):
                def fx(h):
                    xp = x.copy()
                    xp[t, b] += h
                    return L(xp, lam)
                assert abs(fd4(fx, 1e-3) - gx[t, b]) <= 1e-6 * max(1.0, np.max(np.abs(gx)))
        gll = glam * lam
        for k in list(rng.choice(T - d, 6, replace=False)) + [T - 1]:
            def fl(h):
                lp = lam.copy()
                lp[k] *= np.exp(h)
                return L(x, lp)
            assert abs(fd4(fl, 1e-3) - gll[k]) <= 1e-6 * max(1.0, np.max(np.abs(gll)))


def test_weight_gradient_finite_differences(rng):
    """dL/dw (weights of Eq. 1 as parameters) against FP64 fourth-order central finite
    differences of L = <gz, z(w)>, on valid days and on gaps (x = 0 there, so the map is
    smooth in w_t across 0); T = 60, 3 bands, per-day lambda. A dropped z, a sign flip or
    W applied twice each give O(1) errors."""
    T, B, d = 60, 3, 2

    def fd4(f, h):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    for _ in range(6):
        x, w, lam = _rand_case(rng, T, d, B=B, p=0.35, lam_lo=1, lam_hi=4)
        x = np.where(w[:, None] > 0, x, 0.0)
        gz = rng.normal(size=(T, B))
        z = dense.smooth_one(x, w, lam, d)
        gw = dense.vjp_w_one(x, w, lam, d, z, gz)
        on, off = np.flatnonzero(w > 0), np.flatnonzero(w == 0)
        days = list(rng.choice(on, 4, replace=False)) + list(rng.choice(off, 4, replace=False))
        for t in days:
            def f(h):
                wp = w.copy()
                wp[t] += h
                zz = np.linalg.solve(dense.omega(wp, lam, d), wp[:, None] * x)
                return float(np.sum(gz * zz))
            assert abs(fd4(f, 1e-3) - gw[t]) <= 1e-6 * max(1.0, np.max(np.abs(gw))), (t, w[t])


def test_dot_product_transpose_of_eq5(rng):
    """<g, J v> = <J^T g, v> with J = Omega^{-1} W (forward map) and J^T g = W Omega^{-1} g
    (the VJP): pins the transposed reading of Eq. 5."""
    T, d = 80, 3
    _, w, lam = _rand_case(rng, T, d)
    v = rng.normal(size=T)
    g = rng.normal(size=T)
    Jv = dense.smooth_one(v, w, lam, d)
    JTg, _ = dense.vjp_one(w, lam, d, np.zeros(T), g)
    assert abs(np.dot(g, Jv) - np.dot(JTg, v)) <= 1e-12 * np.linalg.norm(g) * np.linalg.norm(v) * 1e2


@pytest.mark.parametrize("d", [1, 2, 3])
def test_hat_trace_limits(rng, d):
    """tr H -> number of valid days as lambda -> 0 and -> d as lambda -> infinity."""
    T = 50
    w = (rng.random(T) < 0.5).astype(float)
    w[: d + 2] = 1.0
    n = w.sum()
    assert abs(dense.hat_trace(w, 1e-9, d) - n) <= 1e-5
    assert abs(dense.hat_trace(w, 1e9, d) - d) <= 1e-3
    diag = dense.inverse_diag(w, 3.0, d)
    assert np.all(diag > 0)


def test_gcv_selects_and_breaks_ties(rng):
    T, d = 60, 2
    t = np.arange(T)
    w = np.ones(T)
    x = np.sin(t / 9.0) + 0.3 * rng.normal(size=T)
    grid = 10 ** np.linspace(0, 5, 16)
    best, scores, zb = dense.gcv_one(x, w, grid, d)
    assert best == int(np.argmin(scores))
    assert np.allclose(zb, dense.smooth_one(x, w, grid[best], d))
    # a polynomial of degree < d gives RSS = 0 and V = 0 for every lambda: first index wins
    best2, s2, _ = dense.gcv_one(1.0 + 0.5 * t / T, w, grid, d)
    assert best2 == 0 and np.max(s2) < 1e-20


def test_mse_maxe_hand_example():
    """Section 4.4 metrics on a 4-day hand example."""
    z = np.array([1.0, 2.0, 3.0, 4.0])
    x = np.array([1.5, 9.0, 2.0, 4.0])
    w = np.array([1.0, 0.0, 1.0, 1.0])
    mse, maxe = dense.mse_maxe(z, x, w)
    assert mse == pytest.approx((0.25 + 0.0 + 1.0 + 0.0) / 4)
    assert maxe == pytest.approx(1.0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_short_series_edge_cases(rng, d):
    """T <= d: D has no rows, Omega = W; positive definite iff every weight is positive."""
    for T in range(1, d + 2):
        x = rng.normal(size=(T, 2, 3))
        w = np.ones((T, 3))
        w[0, 1] = 0.0
        lam = np.ones((T, 3))
        z, st = banded.smooth_tile(x, w, lam, d)
        zd, ok = dense.smooth_tile(x, w, lam, d)
        assert list(st == 0) == list(ok)
        assert np.max(np.abs(z - zd)) <= 1e-12
        if T <= d:
            assert np.allclose(z[:, :, 0], x[:, :, 0])


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_pd_rule_matches_spectrum(rng, d):
    """is_pd (counting rule) agrees with the smallest eigenvalue of Omega."""
    T = 18
    for trial in range(40):
        w = np.zeros(T)
        k = int(rng.integers(0, d + 2))
        w[rng.choice(T, size=k, replace=False)] = rng.uniform(0.5, 2.0, size=k)
        lam = 10 ** rng.uniform(-1, 2, T)
        ev = np.linalg.eigvalsh(dense.omega(w, lam, d))
        scale = np.max(np.abs(ev))
        assert dense.is_pd(w, lam, d) == (ev[0] > 1e-10 * scale)
    assert not dense.is_pd(np.ones(T), np.concatenate([[-1.0], np.ones(T - 1)]), d)


def _dates(rng, T, gap_hi=12):
    return np.cumsum(rng.integers(1, gap_hi, size=T)).astype(float)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_dates_operator_uniform_grid_is_binomial(d):
    """On t = 0..T-1 the uneven-spacing operator is the binomial difference matrix; on
    t = t0 + h (0..T-1) it is that matrix over h^d."""
    T = 20
    assert np.allclose(dense.difference_matrix_dates(np.arange(T, dtype=float), d), dense.difference_matrix(T, d),
                       rtol=0, atol=1e-12)
    Dh = dense.difference_matrix_dates(7.0 + 5.0 * np.arange(T), d)
    assert np.allclose(Dh * 5.0 ** d, dense.difference_matrix(T, d), rtol=0, atol=1e-10)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_dates_operator_recursive_construction(rng, d):
    """An independent construction: first differences divided by the spacing, applied
    recursively with the k-th level divided by (t_{i+k} - t_i)/k (the discrete-derivative
    recursion); it must equal d! times the divided-difference weights."""
    T = 25
    t = _dates(rng, T)
    Dk = np.eye(T)
    for k in range(1, d + 1):
        n = T - k + 1
        Dbar = np.zeros((n - 1, n))
        for i in range(n - 1):
            Dbar[i, i], Dbar[i, i + 1] = -1.0, 1.0
        scale = k / (t[k:] - t[:-k])
        Dk = scale[:, None] * (Dbar @ Dk)
    assert np.allclose(dense.difference_matrix_dates(t, d), Dk, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dates_operator_on_polynomials(rng, d):
    """Exact on polynomials: degree < d is annihilated; t^d maps to d! (its d-th
    derivative), whatever the spacing."""
    T = 30
    t = _dates(rng, T, gap_hi=6)
    t = t - t.mean()
    D = dense.difference_matrix_dates(t, d)
    for q in range(d):
        assert np.max(np.abs(D @ t ** q)) <= 1e-9 * max(1.0, np.max(np.abs(t)) ** q)
    fact = float(np.prod(np.arange(1, d + 1)))
    assert np.allclose(D @ t ** d, fact, rtol=1e-8)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dates_smoother_limits(rng, d):
    """Polynomials of degree < d in t are reproduced for any lambda; lambda -> infinity gives
    the weighted least-squares polynomial of degree d - 1 in t; lambda -> 0 with w = 1 gives x."""
    T = 40
    t = _dates(rng, T, gap_hi=8)
    w = (rng.random(T) < 0.6).astype(float)
    w[rng.choice(T, d + 1, replace=False)] = 1.0
    lam = 10 ** rng.uniform(0, 3, T)
    tc = (t - t.mean()) / t.std()
    poly = sum(rng.normal() * tc ** q for q in range(d))
    assert np.max(np.abs(dense.smooth_one_dates(poly, w, lam, d, t) - poly)) <= 1e-8
    x = rng.normal(size=T)
    if d <= 2:  # at d = 3 the penalty's smallest nonzero eigenvalue (~(pi/T)^6) puts the
        # limit beyond what FP64 conditioning resolves at T = 40
        ts = t / np.mean(np.diff(t))  # unit mean spacing: the penalty's scale is then lambda
        z = dense.smooth_one_dates(x, w, np.full(T, 1e10), d, ts)
        V = np.vander(tc, d, increasing=True)
        coef = np.linalg.lstsq(np.sqrt(w)[:, None] * V, np.sqrt(w) * x, rcond=None)[0]
        assert np.max(np.abs(z - V @ coef)) <= 1e-4
    z0 = dense.smooth_one_dates(x, np.ones(T), np.full(T, 1e-12), d, t)
    assert np.max(np.abs(z0 - x)) <= 1e-6


def test_dates_vjp_finite_differences(rng):
    """The adjoint on sample times against FP64 fourth-order central finite differences of
    L = <gz, z>: dL/dx and dL/dlog(lambda), T = 50 dates with gaps of 1-11 days, 3 bands;
    plus the dot-product identity that fixes the transposed reading of Eq. 5."""
    T, B, d = 50, 3, 2

    def fd4(f, h):
        return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)

    for _ in range(4):
        t = _dates(rng, T)
        x, w, lam = _rand_case(rng, T, d, B=B, p=0.4, lam_lo=1, lam_hi=4)
        gz = rng.normal(size=(T, B))
        z = dense.smooth_one_dates(x, w, lam, d, t)
        gx, glam = dense.vjp_one_dates(w, lam, d, t, z, gz)
        L = lambda xx, ll: float(np.sum(gz * dense.smooth_one_dates(xx, w, ll, d, t)))
        for tt in rng.choice(T, 4, replace=False):
            b = int(rng.integers(B))

            def fx(h):
                xp = x.copy()
                xp[tt, b] += h
                return L(xp, lam)
            assert abs(fd4(fx, 1e-3) - gx[tt, b]) <= 1e-6 * max(1.0, np.max(np.abs(gx)))
        gll = glam * lam
        for k in list(rng.choice(T - d, 4, replace=False)) + [T - 1]:
            def fl(h):
                lp = lam.copy()
                lp[k] *= np.exp(h)
                return L(x, lp)
            assert abs(fd4(fl, 1e-3) - gll[k]) <= 1e-6 * max(1.0, np.max(np.abs(gll)))
        v, g1 = rng.normal(size=T), rng.normal(size=T)
        Jv = dense.smooth_one_dates(v, w, lam, d, t)
        JTg, _ = dense.vjp_one_dates(w, lam, d, t, np.zeros(T), g1)
        assert abs(np.dot(g1, Jv) - np.dot(JTg, v)) <= 1e-10 * np.linalg.norm(g1) * np.linalg.norm(v)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_dates_hat_trace_limits_and_gcv(rng, d):
    """On sample times: tr H -> number of valid days as lambda -> 0 (w binary) and -> d as
    lambda -> infinity (the weighted polynomial fit of degree d - 1 has d parameters); the
    GCV search on t = 0..T-1 is the daily one."""
    T = 40
    t = _dates(rng, T, gap_hi=6)
    ts = t / np.mean(np.diff(t))
    w = (rng.random(T) < 0.5).astype(float)
    w[rng.choice(T, d + 2, replace=False)] = 1.0
    assert abs(dense.hat_trace(w, 1e-9, d, ts) - w.sum()) <= 1e-5
    assert abs(dense.hat_trace(w, 1e9, d, ts) - d) <= 1e-3
    x = rng.normal(size=T)
    grid = [10.0 ** (i / 2) for i in range(8)]
    a = dense.gcv_one(x, w, grid, d)
    b = dense.gcv_one(x, w, grid, d, t=np.arange(T, dtype=float))
    assert a[0] == b[0] and np.allclose(a[1], b[1], rtol=1e-9)


def test_masked_mse_is_the_held_out_mean_and_its_gradient():
    """Section 4.3's loss: with scale = 2 / n_held the summed loss equals the mean squared
    error over the held-out entries (computed by boolean indexing), masked days are inert
    even where the target is NaN, and gz matches central differences of the loss."""
    rng = np.random.default_rng(11)
    T, B, P = 17, 3, 5
    z = rng.normal(size=(T, B, P))
    tgt = rng.normal(size=(T, B, P))
    m = (rng.random((T, P)) < 0.3).astype(float)
    tgt[:, :, :][np.broadcast_to(m[:, None, :] == 0, tgt.shape)] = np.nan
    sel = np.broadcast_to(m[:, None, :] > 0, z.shape)
    n_held = int(sel.sum())
    loss, gz = dense.masked_mse(z, tgt, m, 2.0 / n_held)
    assert abs(loss.sum() - np.mean((z[sel] - tgt[sel]) ** 2)) <= 1e-14
    assert np.all(np.isfinite(gz)) and np.all(gz[~sel] == 0)
    h = 1e-6
    for (t, b, p) in [(0, 0, 0), (3, 1, 2), (16, 2, 4), (8, 0, 1)]:
        zp, zm = z.copy(), z.copy()
        zp[t, b, p] += h
        zm[t, b, p] -= h
        fd = (dense.masked_mse(zp, tgt, m, 0.7)[0].sum() - dense.masked_mse(zm, tgt, m, 0.7)[0].sum()) / (2 * h)
        assert abs(fd - dense.masked_mse(z, tgt, m, 0.7)[1][t, b, p]) <= 1e-8
    l1, g1 = dense.masked_mse(z, np.nan_to_num(tgt), None, 0.5)
    assert np.allclose(g1, 0.5 * (z - np.nan_to_num(tgt))) and l1.shape == (P,)
