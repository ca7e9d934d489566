// Residual of the smoothing system for one step of iterative refinement:
//     r = W x - Omega z0 = W (x - z0) - D^T (Lambda (D z0))        (Omega from Eq. 3)
// or, for a right-hand side taken as given (the adjoint solve Omega g = gz),
//     r = x - Omega z0 = x - W z0 - D^T (Lambda (D z0)).
// At a good z0 the two terms cancel to a few parts in 1e5. D z0 and D^T q are taken
// as nested first differences (exact on smooth sequences, where the binomial sums
// would cancel digits), and the final combination is a double word (ws_df.cuh).
// Thread = one pixel x a block of kDays days; all bands stream through rings of the
// last d+1 values of z0 and of q_k = lambda_k (D z0)_k. Every load is coalesced across
// the pixel-fastest tile layout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_sweep.cuh"

namespace ws {

constexpr int kResidDays = 64;

template <typename F, int D, int NBR>
__global__ void __launch_bounds__(128) k_residual(const F* __restrict__ x, const F* __restrict__ w,
                                                  const F* __restrict__ lam, const F* __restrict__ z0,
                                                  F* __restrict__ r, int T, int B, int P, int lam_scalar,
                                                  int raw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int t0 = blockIdx.y * kResidDays;
  const int t1 = min(T, t0 + kResidDays);
  const int b0 = blockIdx.z * NBR;
  const int nb = min(NBR, B - b0);
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  const F ls = lam_scalar ? lam[p] : F(0);
  // Days outer, bands inner: w_t and lambda_k are read once per day for all bands.
  // Per band: z0 at rows u-D..u and q = lambda (D z0) at rows k-D..k. D z0 and D^T q are
  // nested first differences (exact on smooth sequences, where the binomial sums would
  // cancel digits); the two large terms W(x - z0) and D^T Lambda D z0 that cancel in r
  // are combined as a double word.
  F zr[NBR][D + 1];
  F qb[NBR][D + 1];
#pragma unroll
  for (int j = 0; j < NBR; ++j)
#pragma unroll
    for (int n = 0; n <= D; ++n) {
      zr[j][n] = F(0);
      qb[j][n] = F(0);
    }
  // Days are taken in groups of G: every load of a group (z0 and x of each band, w, lambda)
  // is issued before any of them is used, so G days of reads are in flight per thread.
  constexpr int G = 4;
  for (int ug = t0 - D; ug < t1 + D; ug += G) {
    F zl[G][NBR], xl[G][NBR], wl[G], ll[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = ug + g;
      const int k = u - D, t = k;
      const bool live_u = u < t1 + D;
      const bool row = live_u && k >= 0 && k <= T - D - 1;
      const bool emit = live_u && t >= t0 && t < t1;
      ll[g] = row ? (lam_scalar ? ls : lam[(size_t)k * sP + p]) : F(0);
      wl[g] = emit ? w[(size_t)t * sP + p] : F(0);
#pragma unroll
      for (int j = 0; j < NBR; ++j) {
        const size_t col = (size_t)(b0 + j) * sP + p;
        const bool band = j < nb;
        zl[g][j] = (band && live_u && u >= 0 && u < T) ? z0[(size_t)u * sBP + col] : F(0);
        xl[g][j] = (band && emit) ? x[(size_t)t * sBP + col] : F(0);
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = ug + g;
      if (u >= t1 + D) break;
      const int k = u - D;  // difference row whose last day is u
      const bool row = k >= 0 && k <= T - D - 1;
      const F lk = ll[g];
      const int t = k;      // residual day whose rows k-D..k are now all known
      const bool emit = t >= t0 && t < t1;
      const F wt = wl[g];
#pragma unroll
      for (int j = 0; j < NBR; ++j) {
        if (j >= nb) break;
        const size_t col = (size_t)(b0 + j) * sP + p;
#pragma unroll
        for (int n = 0; n < D; ++n) zr[j][n] = zr[j][n + 1];
        zr[j][D] = zl[g][j];
#pragma unroll
        for (int n = 0; n < D; ++n) qb[j][n] = qb[j][n + 1];
        F q = F(0);
        if (row) {
          F lv[D + 1];
#pragma unroll
          for (int n = 0; n <= D; ++n) lv[n] = zr[j][n];
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int n = 0; n < D - i; ++n) lv[n] = lv[n + 1] - lv[n];
          q = lk * lv[0];
        }
        qb[j][D] = q;
        if (emit) {
          // (D^T q)_t = sum_n c_n q_{t-n} = (-1)^D * (D-th backward difference of q at t)
          F lv[D + 1];
#pragma unroll
          for (int n = 0; n <= D; ++n) lv[n] = qb[j][n];
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int n = D; n > i; --n) lv[n] = lv[n] - lv[n - 1];
          const F dtq = (D % 2) ? -lv[D] : lv[D];
          const F xt = xl[g][j];
          DW<F> acc;
          if (raw) {
            const DW<F> wz = two_prod(wt, zr[j][0]);  // zr[j][0] = z0_t (u = t + D)
            acc = dw_add(DW<F>{xt, F(0)}, DW<F>{-wz.hi, -wz.lo});
          } else {
            acc = wt > F(0) ? dw_scale(two_sum(xt, -zr[j][0]), wt) : DW<F>{F(0), F(0)};
          }
          acc = dw_add(acc, DW<F>{-dtq, F(0)});
          r[(size_t)t * sBP + col] = acc.hi + acc.lo;
        }
      }
    }
  }
}

template <typename F, int D>
static int launch_resid_t(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0,
                          void* r, int raw, cudaStream_t st) {
  constexpr int NBR = 5;  // bands per thread
  dim3 grid((unsigned)((pb.n_series + 127) / 128), (unsigned)((pb.T + kResidDays - 1) / kResidDays),
            (unsigned)((pb.n_bands + NBR - 1) / NBR));
  k_residual<F, D, NBR><<<grid, 128, 0, st>>>(static_cast<const F*>(x), static_cast<const F*>(w),
                                         static_cast<const F*>(lam), static_cast<const F*>(z0), static_cast<F*>(r),
                                         pb.T, pb.n_bands, (int)pb.n_series, pb.lam_mode == WS_LAM_SCALAR, raw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "residual kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int launch_residual(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0, void* r,
                    int raw, cudaStream_t st) {
  if (pb.dtype == WS_F32) {
    switch (pb.d) {
      case 1: return launch_resid_t<float, 1>(pb, x, w, lam, z0, r, raw, st);
      case 2: return launch_resid_t<float, 2>(pb, x, w, lam, z0, r, raw, st);
      case 3: return launch_resid_t<float, 3>(pb, x, w, lam, z0, r, raw, st);
      case 4: return launch_resid_t<float, 4>(pb, x, w, lam, z0, r, raw, st);
    }
  } else {
    switch (pb.d) {
      case 1: return launch_resid_t<double, 1>(pb, x, w, lam, z0, r, raw, st);
      case 2: return launch_resid_t<double, 2>(pb, x, w, lam, z0, r, raw, st);
      case 3: return launch_resid_t<double, 3>(pb, x, w, lam, z0, r, raw, st);
      case 4: return launch_resid_t<double, 4>(pb, x, w, lam, z0, r, raw, st);
    }
  }
  return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
}

}  // namespace ws
