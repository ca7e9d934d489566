// Per-thread time recurrence of the banded solve (one series per thread).
//
// Omega = W + D^T Lambda D (Eq. 3) equals A^T A for the stacked square-root matrix
//   A = [ sqrt(W) ; sqrt(Lambda) D ]      ((2T - d) x T, banded).
// The Cholesky factor R (upper, bandwidth d, R^T R = Omega; the factor Algorithm 1
// computes, transposed) is built row by row with plane (Givens) rotations that fold
// the rows of A into R in time order. Unlike forming Omega and eliminating
// (Algorithm 1), no lambda-sized entries cancel, so FP32 keeps the factor accurate
// at lambda ~ 1e5 where FP32 Algorithm 1 loses ~4 digits to pivot cancellation.
//
// Step i (days 0..T-1):
//   1. difference row i (sqrt(lambda_i) c_0..c_d at columns i..i+d, i < T-d) is rotated
//      into the partial rows i..i+d-1; its remainder starts row i+d, which then
//      absorbs the weight row sqrt(w_{i+d});
//   2. row i of R is now final: 1/D_i = 1/R_ii^2 and rho_{i,j} = R[i][i+j]/R_ii give
//      Omega = L diag(D) L^T with L unit lower, L[i+j][i] = rho_{i,j};
//   3. forward substitution L y = b:  y_i = b_i - sum_j rho_{i-j,j} y_{i-j}; the
//      backward sweep then needs yhat_i = y_i / D_i and rho_{i,1..d}:
//      z_i = yhat_i - sum_j rho_{i,j} z_{i+j}.
// Weight rows 0..d-1 are folded in before step 0.
#pragma once
#include <stdint.h>

namespace ws {

// Binomial coefficient, iterative: a recursive constexpr function is not inlined in
// device code and would become a real call inside the day loop.
__host__ __device__ constexpr int binom(int n, int k) {
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// c_n = (-1)^(D-n) C(D, n): row k of D holds c at columns k..k+D (Section 2).
template <int D>
__host__ __device__ constexpr int dcoef(int n) {
  return ((D - n) % 2 ? -1 : 1) * binom(D, n);
}

// FP32: the hardware reciprocal square root (one MUFU op, relative error ~2^-22): the
// rotations only need it to working precision, and the library rsqrtf is a longer
// sequence with special-case branches. FP64 keeps the library routine.
__device__ __forceinline__ float rsqrt_(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double rsqrt_(double v) { return rsqrt(v); }
__device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
// a * b + c where both terms are known non-negative (sums of squares in the rotations); the
// double-float overload (ws_df.cuh) uses the cheaper same-sign addition there
__device__ __forceinline__ float fma_pos(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_pos(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }

template <typename F, int D, int NB>
struct Sweep {
  // pr[m][n]: partial row i+m of R at column i+n, 0 <= m <= n <= D-1 between steps
  //           (column D is filled transiently inside a step)
  // rr[j][n]: rho_{i-1-j, n+1} of the last D final rows, only n >= j is kept
  // y[b][j]:  y_{i-1-j} of band b
  F pr[D][D + 1];
  F rr[D][D];
  F y[NB][D];

  static constexpr int kFields = D * (D + 1) + NB * D;  // words in a checkpoint

  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int m = 0; m < D; ++m) {
#pragma unroll
      for (int n = 0; n <= D; ++n) pr[m][n] = F(0);
#pragma unroll
      for (int n = 0; n < D; ++n) rr[m][n] = F(0);
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) y[b][j] = F(0);
  }

  // Weight row m (m < D) folded in before step 0: R[m][m] = sqrt(w_m).
  __device__ __forceinline__ void init_weight(int m, F wm) {
#pragma unroll
    for (int q = 0; q < D; ++q)
      if (q == m) pr[q][q] = sqrt_(wm > F(0) ? wm : F(0));
  }

  // Steps 1-2: rotations for day i; returns rho_{i,1..D} and 1/D_i. Reciprocals and
  // square roots come from the rotations' reciprocal square roots (one MUFU op each):
  // row i's final diagonal is sqrt(h0) with h0 from its last rotation, so 1/R_ii = rsqrt(h0).
  __device__ __forceinline__ void factor_step(bool has_row, F lam, F w_ahead, F (&rho)[D], F& invD) {
    F v[D + 1];
    F nd = F(0);
    F inv = F(0);
    if (has_row) {
      const F sl = lam > F(0) ? lam * rsqrt_(lam) : F(0);  // sqrt(lambda) from one MUFU op
#pragma unroll
      for (int n = 0; n <= D; ++n) v[n] = sl * F(dcoef<D>(n));
#pragma unroll
      for (int m = 0; m < D; ++m) {
        const F a = pr[m][m], b = v[m];
        const F h = fma_pos(a, a, b * b);
        const F ir = h > F(0) ? rsqrt_(h) : F(0);
        const F cs = h > F(0) ? a * ir : F(1);
        const F sn = b * ir;
        pr[m][m] = h * ir;
        if (m == 0) inv = ir;
#pragma unroll
        for (int n = m + 1; n < D; ++n) {
          const F p = pr[m][n];
          pr[m][n] = fma(cs, p, sn * v[n]);
          v[n] = fma(cs, v[n], -(sn * p));
        }
        pr[m][D] = sn * v[D];
        v[D] = cs * v[D];
      }
      const F hn = fma_pos(v[D], v[D], w_ahead > F(0) ? w_ahead : F(0));
      nd = hn > F(0) ? hn * rsqrt_(hn) : F(0);
    } else {
#pragma unroll
      for (int m = 0; m < D; ++m) pr[m][D] = F(0);
      const F h0 = pr[0][0] * pr[0][0];
      inv = h0 > F(0) ? rsqrt_(h0) : F(0);
    }
    invD = inv * inv;
#pragma unroll
    for (int n = 1; n <= D; ++n) rho[n - 1] = pr[0][n] * inv;
#pragma unroll
    for (int m = 0; m + 1 < D; ++m)
#pragma unroll
      for (int n = m; n < D; ++n) pr[m][n] = pr[m + 1][n + 1];
    pr[D - 1][D - 1] = nd;
  }

  // Step 3: forward substitution of the NB right-hand sides b for day i.
  __device__ __forceinline__ void subst_step(const F (&rho)[D], F invD, const F (&bv)[NB], F (&yhat)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      F acc = bv[b];
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fma(-rr[j - 1][j - 1], y[b][j - 1], acc);
      yhat[b] = acc * invD;
#pragma unroll
      for (int j = D - 1; j > 0; --j) y[b][j] = y[b][j - 1];
      y[b][0] = acc;
    }
    shift_ring(rho);
  }

  // Ring update alone (factor-only sweeps).
  __device__ __forceinline__ void shift_ring(const F (&rho)[D]) {
#pragma unroll
    for (int j = D - 1; j > 0; --j)
#pragma unroll
      for (int n = j; n < D; ++n) rr[j][n] = rr[j - 1][n];
#pragma unroll
    for (int n = 0; n < D; ++n) rr[0][n] = rho[n];
  }

  static constexpr int kFactorFields = D * (D + 1);

  // Checkpoint in two parts: the factor state (identical for every thread of a pixel)
  // and this thread's forward-substitution state.
  __device__ __forceinline__ void save_factor(F* base, int stride) const {
    int f = 0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int n = m; n < D; ++n) base[(f++) * stride] = pr[m][n];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int n = j; n < D; ++n) base[(f++) * stride] = rr[j][n];
  }
  __device__ __forceinline__ void save_y(F* base, int stride) const {
    int f = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) base[(f++) * stride] = y[b][j];
  }
  __device__ __forceinline__ void load_factor(const F* base, int stride) {
    int f = 0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int n = m; n < D; ++n) pr[m][n] = base[(f++) * stride];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int n = j; n < D; ++n) rr[j][n] = base[(f++) * stride];
  }
  __device__ __forceinline__ void load_y(const F* base, int stride) {
    int f = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) y[b][j] = base[(f++) * stride];
  }

  // Checkpoint: field f of this thread at base[f * stride].
  __device__ __forceinline__ void save(F* base, int stride) const {
    int f = 0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int n = m; n < D; ++n) base[(f++) * stride] = pr[m][n];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int n = j; n < D; ++n) base[(f++) * stride] = rr[j][n];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) base[(f++) * stride] = y[b][j];
  }

  __device__ __forceinline__ void load(const F* base, int stride) {
    int f = 0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int n = m; n < D; ++n) pr[m][n] = base[(f++) * stride];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int n = j; n < D; ++n) rr[j][n] = base[(f++) * stride];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) y[b][j] = base[(f++) * stride];
  }
};

}  // namespace ws
