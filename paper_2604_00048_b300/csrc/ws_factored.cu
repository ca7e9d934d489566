// Stored-factor kernels (Section 3.1): the factor of Omega = L diag(D) L^T is computed
// once (ws_factor) and reused by solves and adjoints, trading (d+1) words per pixel-day
// of memory for the recomputation the tile kernels do. One series per thread; plain
// coalesced loads across the pixel-fastest layout. The factor comes from the same plane
// rotations as the tile kernels (ws_sweep.cuh).
//
// factor[(t*(d+1) + 0)*P + p] = 1/D_t, factor[(t*(d+1) + j)*P + p] = L[t+j][t] (= rho_{t,j}).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"
#include "ws_sweep.cuh"

namespace ws {

template <typename F, int D>
__global__ void __launch_bounds__(128) k_factor(const F* __restrict__ w, const F* __restrict__ lam, F* __restrict__ fac,
                                                uint8_t* __restrict__ status, int T, int P, int lam_scalar) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P;
  Sweep<F, D, 1> s;
  s.reset();
  for (int m = 0; m < D && m < T; ++m) s.init_weight(m, w[(size_t)m * sP + p]);
  const F ls = lam_scalar ? lam[p] : F(0);
  int npos = 0;
  bool bad = false;
  for (int i = 0; i < T; ++i) {
    const F wi = w[(size_t)i * sP + p];
    const F wa = i + D < T ? w[(size_t)(i + D) * sP + p] : F(0);
    const F li = lam_scalar ? ls : lam[(size_t)i * sP + p];
    const bool has_row = i < T - D;
    bad |= !(wi >= F(0)) || !finite_(wi);
    npos += wi > F(0);
    if (has_row) bad |= !(li > F(0)) || !finite_(li);
    F rho[D], invD;
    s.factor_step(has_row, li, wa, rho, invD);
    s.shift_ring(rho);
    fac[((size_t)i * (D + 1)) * sP + p] = invD;
#pragma unroll
    for (int j = 1; j <= D; ++j) fac[((size_t)i * (D + 1) + j) * sP + p] = rho[j - 1];
  }
  const int dmin = D < T ? D : T;
  const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
  if (code != WS_SERIES_OK)
    for (int i = 0; i < T; ++i)
      for (int j = 0; j <= D; ++j) fac[((size_t)i * (D + 1) + j) * sP + p] = F(0);
  if (status) status[p] = code;
}

// z = Omega^{-1} (W x) (weighted) or Omega^{-1} x, with the stored factor. ŷ goes to out as
// scratch in the forward sweep; the backward sweep overwrites it with the solution.
template <typename F, int D>
__global__ void __launch_bounds__(128) k_solve_factored(const F* __restrict__ fac, const F* __restrict__ w,
                                                        const F* __restrict__ x, F* __restrict__ out, int T,
                                                        int B, int P, int weighted) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  for (int b = 0; b < B; ++b) {
    F yw[D];  // y_{t-1..t-D}
    F rw[D][D];  // rho_{t-1-j, n+1}
#pragma unroll
    for (int j = 0; j < D; ++j) {
      yw[j] = F(0);
#pragma unroll
      for (int n = 0; n < D; ++n) rw[j][n] = F(0);
    }
    for (int t = 0; t < T; ++t) {
      const F xv = x[(size_t)t * sBP + (size_t)b * sP + p];
      F acc = weighted ? (w[(size_t)t * sP + p] > F(0) ? w[(size_t)t * sP + p] * xv : F(0)) : xv;
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fma(-rw[j - 1][j - 1], yw[j - 1], acc);
      const F invD = fac[((size_t)t * (D + 1)) * sP + p];
      out[(size_t)t * sBP + (size_t)b * sP + p] = acc * invD;
#pragma unroll
      for (int j = D - 1; j > 0; --j) {
        yw[j] = yw[j - 1];
#pragma unroll
        for (int n = 0; n < D; ++n) rw[j][n] = rw[j - 1][n];
      }
      yw[0] = acc;
#pragma unroll
      for (int n = 0; n < D; ++n) rw[0][n] = fac[((size_t)t * (D + 1) + n + 1) * sP + p];
    }
    F zw[D];
#pragma unroll
    for (int j = 0; j < D; ++j) zw[j] = F(0);
    for (int t = T - 1; t >= 0; --t) {
      const size_t o = (size_t)t * sBP + (size_t)b * sP + p;
      F acc = out[o];
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fma(-fac[((size_t)t * (D + 1) + j) * sP + p], zw[j - 1], acc);
#pragma unroll
      for (int j = D - 1; j > 0; --j) zw[j] = zw[j - 1];
      zw[0] = acc;
      out[o] = acc;
    }
  }
}

// Adjoint with the stored factor: g = Omega^{-1} gz (per band, g held in `gs`, a scratch
// array of T*B*P), gx = W g, glam_k = -sum_b (D g_b)_k (D z_b)_k [* lambda_k], nested
// first differences as in the tile kernel. loglam: bit 0 gradient in log lambda, bit 1
// gx receives g itself.
template <typename F, int D>
__global__ void __launch_bounds__(128) k_adjoint_factored(const F* __restrict__ fac, const F* __restrict__ w,
                                                          const F* __restrict__ lam, const F* __restrict__ z,
                                                          const F* __restrict__ gs, F* __restrict__ gx,
                                                          F* __restrict__ glam, int T, int B, int P, int lam_scalar,
                                                          int loglam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  F gsum = F(0);
  bool ok = fac[p] != F(0) || T == 0;  // zero-filled factor marks a failed series
  for (int b = 0; b < B; ++b) {
    F gl[D + 1], zl[D + 1];  // g and z of days t..t+D
#pragma unroll
    for (int j = 0; j <= D; ++j) {
      gl[j] = F(0);
      zl[j] = F(0);
    }
    for (int t = T - 1; t >= 0; --t) {
      const size_t o = (size_t)t * sBP + (size_t)b * sP + p;
      const F g = ok ? gs[o] : F(0);
      const F zv = z[o];
#pragma unroll
      for (int j = D; j > 0; --j) {
        gl[j] = gl[j - 1];
        zl[j] = zl[j - 1];
      }
      gl[0] = g;
      zl[0] = zv;
      if (gx) gx[o] = (loglam & 2) ? g : w[(size_t)t * sP + p] * g;
      if (glam && t < T - D) {
        F a[D + 1], c[D + 1];
#pragma unroll
        for (int n = 0; n <= D; ++n) {
          a[n] = gl[n];
          c[n] = zl[n];
        }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int n = 0; n < D - i; ++n) {
            a[n] = a[n + 1] - a[n];
            c[n] = c[n + 1] - c[n];
          }
        F v = -a[0] * c[0];
        if (loglam & 1) v *= lam_scalar ? lam[p] : lam[(size_t)t * sP + p];
        if (lam_scalar)
          gsum += v;
        else {
          F* dst = glam + (size_t)t * sP + p;
          *dst = b == 0 ? v : *dst + v;
        }
      } else if (glam && !lam_scalar && b == 0) {
        glam[(size_t)t * sP + p] = F(0);
      }
    }
  }
  if (glam && lam_scalar) glam[p] = gsum;
}

template <typename F, int D>
static int launch_factored_t(int what, const ws_problem& pb, const void* fac_in, void* fac_out, const void* w,
                             const void* lam, const void* x, void* out, const void* z, const void* gs, void* gx,
                             void* glam, uint8_t* status, int weighted, int loglam, cudaStream_t st) {
  const unsigned grid = (unsigned)((pb.n_series + 127) / 128);
  const int T = pb.T, B = pb.n_bands, P = (int)pb.n_series, ls = pb.lam_mode == WS_LAM_SCALAR;
  if (what == 0)
    k_factor<F, D><<<grid, 128, 0, st>>>((const F*)w, (const F*)lam, (F*)fac_out, status, T, P, ls);
  else if (what == 1)
    k_solve_factored<F, D><<<grid, 128, 0, st>>>((const F*)fac_in, (const F*)w, (const F*)x, (F*)out, T, B, P,
                                                 weighted);
  else
    k_adjoint_factored<F, D><<<grid, 128, 0, st>>>((const F*)fac_in, (const F*)w, (const F*)lam, (const F*)z,
                                                   (const F*)gs, (F*)gx, (F*)glam, T, B, P, ls, loglam);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "factored kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int launch_factored(int what, const ws_problem& pb, const void* fac_in, void* fac_out, const void* w,
                    const void* lam, const void* x, void* out, const void* z, const void* gs, void* gx, void* glam,
                    uint8_t* status, int weighted, int loglam, cudaStream_t st) {
#define WS_FAC_CASE(FT, DD) \
  return launch_factored_t<FT, DD>(what, pb, fac_in, fac_out, w, lam, x, out, z, gs, gx, glam, status, weighted, loglam, st)
  if (pb.dtype == WS_F32) {
    switch (pb.d) {
      case 1: WS_FAC_CASE(float, 1);
      case 2: WS_FAC_CASE(float, 2);
      case 3: WS_FAC_CASE(float, 3);
      case 4: WS_FAC_CASE(float, 4);
    }
  } else {
    switch (pb.d) {
      case 1: WS_FAC_CASE(double, 1);
      case 2: WS_FAC_CASE(double, 2);
      case 3: WS_FAC_CASE(double, 3);
      case 4: WS_FAC_CASE(double, 4);
    }
  }
#undef WS_FAC_CASE
  return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
}

}  // namespace ws
