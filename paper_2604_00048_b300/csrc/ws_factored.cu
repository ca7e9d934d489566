// Stored-factor kernels (Section 3.1): the factor of Omega = L diag(D) L^T is computed
// once (ws_factor) and reused by solves and adjoints, trading (d+1) words per pixel-day
// of memory for the recomputation the tile kernels do. One series per thread; plain
// coalesced loads across the pixel-fastest layout; bands in groups of up to four per pass,
// so a day's factor row is read once per sweep for the group. The factor comes from the
// same plane rotations as the tile kernels (ws_sweep.cuh).
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

// z = Omega^{-1} (W x) (weighted) or Omega^{-1} x, with the stored factor, for the band group
// [b0, b0 + NB): the factor row of each day is read once per sweep for the whole group. yhat
// goes to out as scratch in the forward sweep; the backward sweep overwrites it with the
// solution.
template <typename F, int D, int NB>
__global__ void __launch_bounds__(128) k_solve_factored(const F* __restrict__ fac, const F* __restrict__ w,
                                                        const F* __restrict__ x, F* __restrict__ out, int T,
                                                        int B, int P, int b0, int weighted) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  F yw[NB][D];  // y_{t-1..t-D} per band
  F rw[D][D];   // rho_{t-1-j, n+1}
#pragma unroll
  for (int j = 0; j < D; ++j) {
#pragma unroll
    for (int b = 0; b < NB; ++b) yw[b][j] = F(0);
#pragma unroll
    for (int n = 0; n < D; ++n) rw[j][n] = F(0);
  }
#pragma unroll 4
  for (int t = 0; t < T; ++t) {
    const F invD = fac[((size_t)t * (D + 1)) * sP + p];
    const F wt = weighted ? w[(size_t)t * sP + p] : F(1);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const size_t o = (size_t)t * sBP + (size_t)(b0 + b) * sP + p;
      const F xv = x[o];
      F acc = weighted ? (wt > F(0) ? wt * xv : F(0)) : xv;
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fma(-rw[j - 1][j - 1], yw[b][j - 1], acc);
      out[o] = acc * invD;
#pragma unroll
      for (int j = D - 1; j > 0; --j) yw[b][j] = yw[b][j - 1];
      yw[b][0] = acc;
    }
#pragma unroll
    for (int j = D - 1; j > 0; --j)
#pragma unroll
      for (int n = 0; n < D; ++n) rw[j][n] = rw[j - 1][n];
#pragma unroll
    for (int n = 0; n < D; ++n) rw[0][n] = fac[((size_t)t * (D + 1) + n + 1) * sP + p];
  }
  F zw[NB][D];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j < D; ++j) zw[b][j] = F(0);
#pragma unroll 4
  for (int t = T - 1; t >= 0; --t) {
    F rho[D];
#pragma unroll
    for (int j = 1; j <= D; ++j) rho[j - 1] = fac[((size_t)t * (D + 1) + j) * sP + p];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const size_t o = (size_t)t * sBP + (size_t)(b0 + b) * sP + p;
      F acc = out[o];
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fma(-rho[j - 1], zw[b][j - 1], acc);
#pragma unroll
      for (int j = D - 1; j > 0; --j) zw[b][j] = zw[b][j - 1];
      zw[b][0] = acc;
      out[o] = acc;
    }
  }
}

// Adjoint with the stored factor for the band group [b0, b0 + NB), in one kernel: the
// forward sweep of g = Omega^{-1} gz writes yhat to `gs` (scratch, T*B*P); the backward
// sweep forms g day by day and with it gx = W g (or g) and the day's
// -sum_b (D g_b)_t (D z_b)_t over the group (nested first differences of windows of g and z,
// as in the tile kernel), written once per day (added to the earlier groups' sum).
// loglam: bit 0 gradient in log lambda, bit 1 gx receives g itself.
template <typename F, int D, int NB>
__global__ void __launch_bounds__(128) k_adjoint_factored(const F* __restrict__ fac, const F* __restrict__ w,
                                                          const F* __restrict__ lam, const F* __restrict__ z,
                                                          const F* __restrict__ gz, F* __restrict__ gs,
                                                          F* __restrict__ gx, F* __restrict__ glam, int T, int B,
                                                          int P, int b0, int lam_scalar, int loglam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  const bool ok = T == 0 || fac[p] != F(0);  // a zero-filled factor marks a failed series
  // forward sweep (unweighted right-hand side gz)
  {
    F yw[NB][D];
    F rw[D][D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
      for (int b = 0; b < NB; ++b) yw[b][j] = F(0);
#pragma unroll
      for (int n = 0; n < D; ++n) rw[j][n] = F(0);
    }
  #pragma unroll 4
  for (int t = 0; t < T; ++t) {
      const F invD = fac[((size_t)t * (D + 1)) * sP + p];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const size_t o = (size_t)t * sBP + (size_t)(b0 + b) * sP + p;
        F acc = gz[o];
#pragma unroll
        for (int j = 1; j <= D; ++j) acc = fma(-rw[j - 1][j - 1], yw[b][j - 1], acc);
        gs[o] = acc * invD;
#pragma unroll
        for (int j = D - 1; j > 0; --j) yw[b][j] = yw[b][j - 1];
        yw[b][0] = acc;
      }
#pragma unroll
      for (int j = D - 1; j > 0; --j)
#pragma unroll
        for (int n = 0; n < D; ++n) rw[j][n] = rw[j - 1][n];
#pragma unroll
      for (int n = 0; n < D; ++n) rw[0][n] = fac[((size_t)t * (D + 1) + n + 1) * sP + p];
    }
  }
  // backward sweep with the epilogue
  F gl[NB][D + 1], zl[NB][D + 1];  // g and z of days t..t+D per band
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int j = 0; j <= D; ++j) {
      gl[b][j] = F(0);
      zl[b][j] = F(0);
    }
  F gsum = F(0);
#pragma unroll 4
  for (int t = T - 1; t >= 0; --t) {
    F rho[D];
#pragma unroll
    for (int j = 1; j <= D; ++j) rho[j - 1] = fac[((size_t)t * (D + 1) + j) * sP + p];
    const F wt = w[(size_t)t * sP + p];
    F dl = F(0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const size_t o = (size_t)t * sBP + (size_t)(b0 + b) * sP + p;
      F g = gs[o];
#pragma unroll
      for (int j = 1; j <= D; ++j) g = fma(-rho[j - 1], gl[b][j - 1], g);
      g = ok ? g : F(0);
#pragma unroll
      for (int j = D; j > 0; --j) {
        gl[b][j] = gl[b][j - 1];
        zl[b][j] = zl[b][j - 1];
      }
      gl[b][0] = g;
      zl[b][0] = z[o];
      if (gx) gx[o] = (loglam & 2) ? g : wt * g;
      if (glam && t < T - D) {
        F a[D + 1], c[D + 1];
#pragma unroll
        for (int n = 0; n <= D; ++n) {
          a[n] = gl[b][n];
          c[n] = zl[b][n];
        }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int n = 0; n < D - i; ++n) {
            a[n] = a[n + 1] - a[n];
            c[n] = c[n + 1] - c[n];
          }
        dl = fma(a[0], c[0], dl);
      }
    }
    if (glam) {
      F v = t < T - D ? -dl : F(0);
      if ((loglam & 1) && t < T - D) v *= lam_scalar ? lam[p] : lam[(size_t)t * sP + p];
      if (lam_scalar) {
        gsum += v;
      } else {
        F* dst = glam + (size_t)t * sP + p;
        *dst = b0 == 0 ? v : *dst + v;
      }
    }
  }
  if (glam && lam_scalar) glam[p] = b0 == 0 ? gsum : glam[p] + gsum;
}

template <typename F, int D, int NB>
static void launch_group(int what, const ws_problem& pb, unsigned grid, const void* fac_in, const void* w,
                         const void* lam, const void* x, void* out, const void* z, void* gs, void* gx, void* glam,
                         int b0, int weighted, int loglam, cudaStream_t st) {
  const int T = pb.T, B = pb.n_bands, P = (int)pb.n_series, ls = pb.lam_mode == WS_LAM_SCALAR;
  if (what == 1)
    k_solve_factored<F, D, NB><<<grid, 128, 0, st>>>((const F*)fac_in, (const F*)w, (const F*)x, (F*)out, T, B, P,
                                                     b0, weighted);
  else
    k_adjoint_factored<F, D, NB><<<grid, 128, 0, st>>>((const F*)fac_in, (const F*)w, (const F*)lam, (const F*)z,
                                                       (const F*)x, (F*)gs, (F*)gx, (F*)glam, T, B, P, b0, ls,
                                                       loglam);
}

// what: 0 factor; 1 solve (x -> out); 2 adjoint (x = gz, out unused, gs = yhat scratch).
template <typename F, int D>
static int launch_factored_t(int what, const ws_problem& pb, const void* fac_in, void* fac_out, const void* w,
                             const void* lam, const void* x, void* out, const void* z, const void* gs, void* gx,
                             void* glam, uint8_t* status, int weighted, int loglam, cudaStream_t st) {
  const unsigned grid = (unsigned)((pb.n_series + 127) / 128);
  const int T = pb.T, P = (int)pb.n_series, ls = pb.lam_mode == WS_LAM_SCALAR;
  if (what == 0) {
    k_factor<F, D><<<grid, 128, 0, st>>>((const F*)w, (const F*)lam, (F*)fac_out, status, T, P, ls);
  } else {
    void* scratch = const_cast<void*>(gs);
    for (int b0 = 0; b0 < pb.n_bands;) {
      const int nb = pb.n_bands - b0 >= 4 ? 4 : pb.n_bands - b0;
      switch (nb) {
        case 4: launch_group<F, D, 4>(what, pb, grid, fac_in, w, lam, x, out, z, scratch, gx, glam, b0, weighted, loglam, st); break;
        case 3: launch_group<F, D, 3>(what, pb, grid, fac_in, w, lam, x, out, z, scratch, gx, glam, b0, weighted, loglam, st); break;
        case 2: launch_group<F, D, 2>(what, pb, grid, fac_in, w, lam, x, out, z, scratch, gx, glam, b0, weighted, loglam, st); break;
        default: launch_group<F, D, 1>(what, pb, grid, fac_in, w, lam, x, out, z, scratch, gx, glam, b0, weighted, loglam, st); break;
      }
      b0 += nb;
    }
  }
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
