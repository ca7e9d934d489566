/*
 * Banded FP64 oracle for the Whittaker-Henderson smoother (test infrastructure).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load this library; the product path never does. It shares no code with the
 * CUDA path.
 *
 * Per series it follows Section 3 of the paper step by step:
 *   1. assemble Omega = W + D^T Lambda D (Eq. 3) in LAPACK lower band storage,
 *      ab[j][t] = Omega[t+j][t] for j = 0..d (Section 3.1, Fig. 2, whose printed
 *      entries contain index typos; this is the storage the text describes);
 *   2. factor it in place with the right-looking banded Cholesky of Algorithm 1:
 *      for every column t take the pivot, scale the column, and subtract the
 *      rank-one update from the next d columns;
 *   3. forward substitution L y = W x and back substitution L^T z = y, one pass
 *      per spectral band, all bands sharing the factor (Section 3.1);
 *   4. for the adjoint (Section 2.3, Eqs. 4-5): g = Omega^{-1} gz with the same
 *      factor, dx = W g, dlam_k = -sum_b (D g_b)_k (D z_b)_k for k < T-d.
 *
 * Layout: the tile layout of the GPU library, x[(t*B + b)*P + p], w[t*P + p],
 * lam[t*P + p] (per day; entry k weights difference row k, the last d entries
 * are ignored) or lam[p] (scalar). Status per series: 0 ok, 1 Omega not positive
 * definite (fewer than min(d, T) positive weights, or a non-positive pivot),
 * 3 invalid lambda (not > 0 and finite) or weight (not >= 0 and finite).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static long binom(int n, int k) {
  long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

/* c_i = (-1)^(d-i) C(d, i): row k of D holds c at columns k..k+d. */
static void diff_coeffs(int d, double* c) {
  for (int i = 0; i <= d; ++i) c[i] = ((d - i) % 2 ? -1.0 : 1.0) * (double)binom(d, i);
}

/* Step 1: Omega in lower band storage, ab[j*T + t] = Omega[t+j][t]. */
static void assemble_band(int T, int d, const double* w, const double* lamk, double* ab) {
  double c[8];
  diff_coeffs(d, c);
  memset(ab, 0, sizeof(double) * (size_t)(d + 1) * T);
  for (int t = 0; t < T; ++t) ab[t] = w[t];
  for (int k = 0; k < T - d; ++k)
    for (int i = 0; i <= d; ++i)
      for (int j = i; j <= d; ++j) ab[(size_t)(j - i) * T + (k + i)] += lamk[k] * c[i] * c[j];
}

/* Step 2: Algorithm 1, in place. Returns 0 on success, 1 on a non-positive pivot. */
static int band_cholesky(int T, int d, double* ab) {
  double v[8];
  for (int t = 0; t < T; ++t) {
    double om = ab[t];
    for (int j = 0; j < d; ++j) v[j] = ab[(size_t)(j + 1) * T + t];
    if (!(om > 0.0)) return 1;
    double s = sqrt(om);
    ab[t] = s;
    for (int j = 0; j < d; ++j) ab[(size_t)(j + 1) * T + t] = v[j] / s;
    int nu = d < T - t - 1 ? d : T - t - 1;
    for (int u = 0; u < nu; ++u)
      for (int j = 0; j < d - u; ++j) ab[(size_t)j * T + (t + 1 + u)] -= v[u + j] * v[u] / om;
  }
  return 0;
}

/* Step 3: L y = r then L^T z = y, L[t+j][t] = ab[j][t]. In place on r. */
static void band_solve(int T, int d, const double* ab, double* r) {
  for (int t = 0; t < T; ++t) {
    double s = r[t];
    for (int j = 1; j <= d && j <= t; ++j) s -= ab[(size_t)j * T + (t - j)] * r[t - j];
    r[t] = s / ab[t];
  }
  for (int t = T - 1; t >= 0; --t) {
    double s = r[t];
    for (int j = 1; j <= d && t + j < T; ++j) s -= ab[(size_t)j * T + t] * r[t + j];
    r[t] = s / ab[t];
  }
}

static int check_inputs(int T, int d, const double* w, const double* lamk) {
  int npos = 0;
  for (int t = 0; t < T; ++t) {
    if (!(w[t] >= 0.0) || !isfinite(w[t])) return 3;
    npos += w[t] > 0.0;
  }
  for (int k = 0; k < T - d; ++k)
    if (!(lamk[k] > 0.0) || !isfinite(lamk[k])) return 3;
  /* Omega is positive definite iff no nonzero polynomial of degree < d vanishes on the
   * positive-weight days: at least min(d, T) positive weights (for T < d, D is empty and
   * Omega = W). */
  if (npos < (d < T ? d : T)) return 1;
  return 0;
}

/* Gather one series of the tile layout into contiguous buffers. */
static void gather(int T, int B, long P, long p, int lam_scalar, const double* x, const double* w,
                   const double* lam, double* xs, double* ws, double* ls) {
  for (int t = 0; t < T; ++t) {
    ws[t] = w[(size_t)t * P + p];
    ls[t] = lam_scalar ? lam[p] : lam[(size_t)t * P + p];
    if (x)
      for (int b = 0; b < B; ++b) xs[(size_t)b * T + t] = x[((size_t)t * B + b) * P + p];
  }
}

/* z = Omega^{-1} W x for every series of a tile. Returns the number of series with status != 0. */
long wh_banded_smooth_tile(int T, int d, int B, long P, const double* x, const double* w,
                           const double* lam, int lam_scalar, double* z, uint8_t* status,
                           int nthreads) {
  long bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : bad)
  {
    double* ab = (double*)malloc(sizeof(double) * (size_t)(d + 1) * T);
    double* xs = (double*)malloc(sizeof(double) * (size_t)B * T);
    double* ws = (double*)malloc(sizeof(double) * (size_t)T);
    double* ls = (double*)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(static)
    for (long p = 0; p < P; ++p) {
      gather(T, B, P, p, lam_scalar, x, w, lam, xs, ws, ls);
      int st = check_inputs(T, d, ws, ls);
      if (st == 0) {
        assemble_band(T, d, ws, ls, ab);
        st = band_cholesky(T, d, ab);
      }
      for (int b = 0; b < B; ++b) {
        double* r = xs + (size_t)b * T;
        if (st == 0) {
          for (int t = 0; t < T; ++t) r[t] = ws[t] > 0.0 ? ws[t] * r[t] : 0.0;
          band_solve(T, d, ab, r);
        } else {
          for (int t = 0; t < T; ++t) r[t] = 0.0;
        }
        for (int t = 0; t < T; ++t) z[((size_t)t * B + b) * P + p] = r[t];
      }
      if (status) status[p] = (uint8_t)st;
      bad += st != 0;
    }
    free(ab);
    free(xs);
    free(ws);
    free(ls);
  }
  return bad;
}

/* Reverse-mode derivatives for every series of a tile (Eqs. 4-5):
 *   g = Omega^{-1} gz, gx = W g, glam_k = -sum_b (D g_b)_k (D z_b)_k (k < T-d, else 0);
 * with lam_scalar, glam[p] = sum_k of the above. log_lambda multiplies by lambda. */
long wh_banded_vjp_tile(int T, int d, int B, long P, const double* w, const double* lam,
                        int lam_scalar, const double* z, const double* gz, double* gx,
                        double* glam, int log_lambda, uint8_t* status, int nthreads) {
  long bad = 0;
  double c[8];
  diff_coeffs(d, c);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : bad)
  {
    double* ab = (double*)malloc(sizeof(double) * (size_t)(d + 1) * T);
    double* gs = (double*)malloc(sizeof(double) * (size_t)B * T);
    double* zs = (double*)malloc(sizeof(double) * (size_t)B * T);
    double* ws = (double*)malloc(sizeof(double) * (size_t)T);
    double* ls = (double*)malloc(sizeof(double) * (size_t)T);
    double* acc = (double*)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(static)
    for (long p = 0; p < P; ++p) {
      gather(T, B, P, p, lam_scalar, gz, w, lam, gs, ws, ls);
      for (int t = 0; t < T; ++t)
        for (int b = 0; b < B; ++b) zs[(size_t)b * T + t] = z[((size_t)t * B + b) * P + p];
      int st = check_inputs(T, d, ws, ls);
      if (st == 0) {
        assemble_band(T, d, ws, ls, ab);
        st = band_cholesky(T, d, ab);
      }
      for (int t = 0; t < T; ++t) acc[t] = 0.0;
      for (int b = 0; b < B; ++b) {
        double* g = gs + (size_t)b * T;
        const double* zb = zs + (size_t)b * T;
        if (st == 0) {
          band_solve(T, d, ab, g);
          for (int k = 0; k < T - d; ++k) {
            double dg = 0.0, dz = 0.0;
            for (int i = 0; i <= d; ++i) {
              dg += c[i] * g[k + i];
              dz += c[i] * zb[k + i];
            }
            acc[k] -= dg * dz;
          }
        } else {
          for (int t = 0; t < T; ++t) g[t] = 0.0;
        }
        for (int t = 0; t < T; ++t) gx[((size_t)t * B + b) * P + p] = ws[t] * g[t];
      }
      if (lam_scalar) {
        double s = 0.0;
        for (int k = 0; k < T - d; ++k) s += acc[k];
        glam[p] = log_lambda ? s * ls[0] : s;
      } else {
        for (int t = 0; t < T; ++t) glam[(size_t)t * P + p] = log_lambda ? acc[t] * ls[t] : acc[t];
      }
      if (status) status[p] = (uint8_t)st;
      bad += st != 0;
    }
    free(ab);
    free(gs);
    free(zs);
    free(ws);
    free(ls);
    free(acc);
  }
  return bad;
}

/* Exposed for the tests: the band after Algorithm 1 for one series (ab: (d+1)*T). */
int wh_banded_factor_one(int T, int d, const double* w, const double* lamk, double* ab) {
  assemble_band(T, d, w, lamk, ab);
  return band_cholesky(T, d, ab);
}

/* Exposed for the tests: Omega in lower band storage for one series (ab: (d+1)*T). */
void wh_banded_assemble_one(int T, int d, const double* w, const double* lamk, double* ab) {
  assemble_band(T, d, w, lamk, ab);
}

int wh_banded_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
