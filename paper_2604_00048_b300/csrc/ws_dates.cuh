// Rows of the difference operator on unevenly spaced sample times (Section 2): row k is d!
// times the weights of the divided difference f[t_k, ..., t_{k+d}],
//     c_{k,j} = d! / prod_{m != j} (t_{k+j} - t_{k+m}),
// and the rotation step of the factorisation (ws_sweep.cuh) with those coefficients in place
// of the binomial ones. Shared by the uneven-spacing solve and the posterior spread.
#pragma once
#include "ws_sweep.cuh"

namespace ws {

// d! / den: FP32 takes the fast division (two ulp; the coefficients scale the penalty rows,
// where that is far below the solve's own rounding), FP64 the IEEE one.
__device__ __forceinline__ float coef_div(float num, float den) { return __fdividef(num, den); }
__device__ __forceinline__ double coef_div(double num, double den) { return num / den; }

// Row coefficients of day i from the dates tw[0..D] = t_i..t_{i+D}.
template <typename F, int D>
__device__ __forceinline__ void dates_coef(const F (&tw)[D + 1], F (&c)[D + 1]) {
  F fact = F(1);
#pragma unroll
  for (int q = 2; q <= D; ++q) fact *= F(q);
#pragma unroll
  for (int j = 0; j <= D; ++j) {
    F den = F(1);
#pragma unroll
    for (int m = 0; m <= D; ++m)
      if (m != j) den *= tw[j] - tw[m];
    c[j] = coef_div(fact, den);
  }
}

// The rotation step of day i (the plane rotations of Sweep::factor_step) with the row
// coefficients c instead of the binomial ones: difference row i, sqrt(lambda_i) c at
// columns i..i+D, is rotated into the partial rows; its remainder starts row i+D, which
// absorbs sqrt(w_{i+D}); row i is then final.
template <typename F, int D, int NB>
__device__ __forceinline__ void dates_factor_step(Sweep<F, D, NB>& s, bool has_row, F lam, F w_ahead,
                                                  const F (&c)[D + 1], F (&rho)[D], F& invD) {
  F v[D + 1];
  F nd = F(0);
  F inv = F(0);
  if (has_row) {
    const F sl = lam > F(0) ? lam * rsqrt_(lam) : F(0);
#pragma unroll
    for (int n = 0; n <= D; ++n) v[n] = sl * c[n];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const F a = s.pr[m][m], b = v[m];
      const F h = fma_pos(a, a, b * b);
      const F ir = h > F(0) ? rsqrt_(h) : F(0);
      const F cs = h > F(0) ? a * ir : F(1);
      const F sn = b * ir;
      s.pr[m][m] = h * ir;
      if (m == 0) inv = ir;
#pragma unroll
      for (int n = m + 1; n < D; ++n) {
        const F p = s.pr[m][n];
        s.pr[m][n] = fma(cs, p, sn * v[n]);
        v[n] = fma(cs, v[n], -(sn * p));
      }
      s.pr[m][D] = sn * v[D];
      v[D] = cs * v[D];
    }
    const F hn = fma_pos(v[D], v[D], w_ahead > F(0) ? w_ahead : F(0));
    nd = hn > F(0) ? hn * rsqrt_(hn) : F(0);
  } else {
#pragma unroll
    for (int m = 0; m < D; ++m) s.pr[m][D] = F(0);
    const F h0 = s.pr[0][0] * s.pr[0][0];
    inv = h0 > F(0) ? rsqrt_(h0) : F(0);
  }
  invD = inv * inv;
#pragma unroll
  for (int n = 1; n <= D; ++n) rho[n - 1] = s.pr[0][n] * inv;
#pragma unroll
  for (int m = 0; m + 1 < D; ++m)
#pragma unroll
    for (int n = m; n < D; ++n) s.pr[m][n] = s.pr[m + 1][n + 1];
  s.pr[D - 1][D - 1] = nd;
}

}  // namespace ws
