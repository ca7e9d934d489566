// Posterior spread of the smooth: the pointwise credibility intervals drawn in Fig. 4.
//
// The paper plots them and takes their formula from the Bayesian reading of the smoother
// that it cites. In that reading z = Omega^{-1} W x (Eq. 3) is the posterior mean of a
// signal s whose observations on days with w_t > 0 have precision w_t / sigma^2 and whose
// (improper) prior density is proportional to exp(-s^T D^T Lambda D s / (2 sigma^2)); the
// posterior covariance is sigma^2 Omega^{-1}. sigma^2 is estimated per band from the
// residuals: sigma2_b = RSS_b / (n - tr H), RSS_b = sum_t w_t (x_tb - z_tb)^2, n = sum_t w_t,
// tr H = sum_t w_t (Omega^{-1})_tt (H = Omega^{-1} W, the hat matrix). The interval at
// level q is z_tb +- q sd_tb with sd_tb = sqrt(sigma2_b (Omega^{-1})_tt).
//
// Two kernels:
//   k_post_diag: diag(Omega^{-1}) for every day, n and tr H. The factor comes from the same
//     plane-rotation recurrence as the solve (ws_sweep.cuh, rows of R in time order), and
//     the diagonal from the banded selected-inverse recursion (Takahashi, Fagan and Chin,
//     1973) run backwards over it: with Omega = U^T diag(1/invD) U, U unit upper with
//     U[t][t+j] = rho_{t,j},
//         Sigma[t][t+m] = - sum_{j=1..d} rho_{t,j} Sigma[t+j][t+m]      (m = 1..d)
//         Sigma[t][t]   = invD_t - sum_{j=1..d} rho_{t,j} Sigma[t][t+j].
//     The d x d window of Sigma is carried in double-word arithmetic in FP32 (for large
//     lambda, rho approaches the difference coefficients and each new entry is a d-th
//     difference of a smooth sequence, which single precision loses digits on); rho and
//     invD are FP32. One series per thread, 128 per CTA (64 in FP64); each thread stages its
//     own column of w and lambda (chunks of 8 days, two stages, LDGSTS), so no block barrier
//     is needed. On sample times (ws_posterior_dates) it also stages its column of t and
//     forms the rows of D per day (ws_dates.cuh). Pass 1 runs the factor forward and stores its state (the d(d+1)/2 partial
//     row entries) per chunk; pass 2 goes back over the chunks, recomputes each chunk's
//     rho and invD into registers from its checkpoint, and runs the recursion, writing
//     diag[t][p] and summing tr H.
//   k_post_sd: per (series, band) thread: RSS over the days (compensated sum), sigma2_b,
//     then sd over the days from diag. Pure streaming; the CTAs of the bands of one block
//     of series are adjacent in launch order, so w and diag reach them through L2. FP32 with
//     P % 4 == 0 takes the 16-byte form k_post_sd4 (four series per thread).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"
#include "ws_dates.cuh"

namespace ws {

// series per CTA of k_post_diag (one per thread): 128 in FP32, 64 in FP64 (static shared memory)
template <typename F>
constexpr int post_np() { return sizeof(F) == 8 ? 64 : 128; }
constexpr int kPostC = 8;     // days per chunk (pass 2 holds a chunk's factor rows in registers)
constexpr int kSdNP = 128;    // series per CTA of k_post_sd

template <typename F>
struct PostArgs {
  int T, P, nch, n_tiles, lam_scalar;
  const F* w;        // [T][P]
  const F* lam;      // [T][P] or [P]
  F* diag;           // [T][P] output
  F* den;            // [P]: n - tr H; -1 where the series has no posterior, NaN where the
                     // residual degrees of freedom are within rounding of zero
  uint8_t* status;   // [P] or null
  F* ckpt;           // per CTA: nch * kPr * (series per CTA)
  const F* t;        // sample times [T][P] (the uneven-spacing operator) or null (daily grid)
};

template <typename F>
__device__ __forceinline__ bool finite_post(F v) { return isfinite(v); }

// DT: the rows of D come from each series' sample times (staged like w) instead of the
// binomial coefficients of the daily grid.
template <typename F, int D, bool DT>
__global__ void __launch_bounds__(post_np<F>(), sizeof(F) == 4 ? (D <= 2 ? (DT ? 6 : 7) : (D == 3 ? 6 : 4)) : 1)
    k_post_diag(const PostArgs<F> a) {
  constexpr int kPostNP = post_np<F>();
  using SW = Sweep<F, D, 1>;
  constexpr int kPr = D * (D + 1) / 2;  // partial-row words in a checkpoint
  constexpr bool kDW = sizeof(F) == 4;  // double-word window in FP32
  __shared__ F sw[2][kPostC + D][kPostNP];
  __shared__ F sl[2][kPostC][kPostNP];
  __shared__ F stt[2][DT ? kPostC + D : 1][kPostNP];
  const int tid = threadIdx.x;
  const int T = a.T, nch = a.nch, P = a.P;
  F* const ck = a.ckpt + (size_t)blockIdx.x * nch * kPr * kPostNP + tid;

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int p = tile * kPostNP + tid;
    const bool act = p < P;
    // this thread's column of chunk c: C + D days of w, C days of lambda (zero outside)
    auto issue = [&](int c, int st) {
      const int t0 = c * kPostC;
#pragma unroll
      for (int k = 0; k < kPostC + D; ++k) {
        const int t = t0 + k;
        const bool v = act && t < T;
        cp_async_elem<sizeof(F)>(&sw[st][k][tid], v ? a.w + (size_t)t * P + p : a.w, v);
        if constexpr (DT) cp_async_elem<sizeof(F)>(&stt[st][k][tid], v ? a.t + (size_t)t * P + p : a.t, v);
      }
      if (!a.lam_scalar) {
#pragma unroll
        for (int k = 0; k < kPostC; ++k) {
          const int t = t0 + k;
          const bool v = act && t < T;
          cp_async_elem<sizeof(F)>(&sl[st][k][tid], v ? a.lam + (size_t)t * P + p : a.lam, v);
        }
      }
      cp_async_commit();
    };

    // ---- pass 1: factor forward in time, checkpoints ----
    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    F n = F(0);
    const F lam_s = (a.lam_scalar && act) ? a.lam[p] : F(0);
    issue(0, 0);
    if (nch > 1) issue(1, 1);
    for (int c = 0; c < nch; ++c) {
      if (c + 1 < nch) cp_async_wait<1>(); else cp_async_wait<0>();
      const int st = c & 1;
      if (c == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m)
          if (m < T) s.init_weight(m, sw[0][m][tid]);
      }
      {
        F* ckc = ck + (size_t)c * kPr * kPostNP;
        int f = 0;
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int q = m; q < D; ++q) ckc[(size_t)(f++) * kPostNP] = s.pr[m][q];
      }
      const int nd = min(kPostC, T - c * kPostC);
#pragma unroll 2
      for (int k = 0; k < nd; ++k) {
        const int i = c * kPostC + k;
        const F wi = sw[st][k][tid], wa = sw[st][k + D][tid];
        const F li = a.lam_scalar ? lam_s : sl[st][k][tid];
        const bool has_row = i < T - D;
        bad |= !(wi >= F(0)) || !finite_post(wi);
        if (has_row) bad |= !(li > F(0)) || !finite_post(li);
        npos += wi > F(0);
        n += wi;
        F rho[D], invD;
        if constexpr (DT) {
          F tw[D + 1], cf[D + 1];
#pragma unroll
          for (int j = 0; j <= D; ++j) tw[j] = stt[st][k + j][tid];
          bad |= !finite_post(tw[0]);
          if (i + 1 < T) bad |= !(tw[1] > tw[0]);
          if (has_row) dates_coef<F, D>(tw, cf);
          dates_factor_step(s, has_row, li, wa, cf, rho, invD);
        } else {
          s.factor_step(has_row, li, wa, rho, invD);
        }
      }
      if (c + 2 < nch) issue(c + 2, st);
    }
    const int dmin = D < T ? D : T;
    const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
    const bool okser = act && code == WS_SERIES_OK;

    // ---- pass 2: selected inverse backwards in time ----
    using DWt = DW<F>;
    DWt Sg[D][D];  // Sg[a][b] = Sigma[t+1+a][t+1+b] before day t
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int m = 0; m < D; ++m) Sg[j][m] = DWt{F(0), F(0)};
    DWt trh = {F(0), F(0)};
    F nanacc = F(0);
    for (int c = nch - 1; c >= 0; --c) {
      const int st = c & 1;
      if (c < nch - 2) {
        if (c >= 1) cp_async_wait<1>(); else cp_async_wait<0>();
      }
      {
        const F* ckc = ck + (size_t)c * kPr * kPostNP;
        int f = 0;
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int q = m; q < D; ++q) s.pr[m][q] = ckc[(size_t)(f++) * kPostNP];
      }
      const int nd = min(kPostC, T - c * kPostC);
      F ik[kPostC], rk[kPostC][D];
#pragma unroll
      for (int k = 0; k < kPostC; ++k) {
        if (k < nd) {
          const int i = c * kPostC + k;
          const F wa = sw[st][k + D][tid];
          const F li = a.lam_scalar ? lam_s : sl[st][k][tid];
          F rho[D], invD;
          if constexpr (DT) {
            F tw[D + 1], cf[D + 1];
#pragma unroll
            for (int j = 0; j <= D; ++j) tw[j] = stt[st][k + j][tid];
            if (i < T - D) dates_coef<F, D>(tw, cf);
            dates_factor_step(s, i < T - D, li, wa, cf, rho, invD);
          } else {
            s.factor_step(i < T - D, li, wa, rho, invD);
          }
          ik[k] = invD;
#pragma unroll
          for (int j = 0; j < D; ++j) rk[k][j] = rho[j];
        }
      }
#pragma unroll
      for (int k = kPostC - 1; k >= 0; --k) {
        if (k < nd) {
          const int i = c * kPostC + k;
          DWt sm[D];  // Sigma[t][t+1+m]
          DWt s0 = {ik[k], F(0)};
          if (kDW) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
              DWt acc = dw_scale(Sg[0][m], rk[k][0]);
#pragma unroll
              for (int j = 1; j < D; ++j) acc = dw_fma(acc, rk[k][j], Sg[j][m]);
              sm[m] = DWt{-acc.hi, -acc.lo};
            }
#pragma unroll
            for (int j = 0; j < D; ++j) s0 = dw_fma(s0, -rk[k][j], sm[j]);
          } else {  // FP64: plain window (the lo parts stay zero)
#pragma unroll
            for (int m = 0; m < D; ++m) {
              F acc = F(0);
#pragma unroll
              for (int j = 0; j < D; ++j) acc = fma(rk[k][j], Sg[j][m].hi, acc);
              sm[m] = DWt{-acc, F(0)};
            }
            F s0h = ik[k];
#pragma unroll
            for (int j = 0; j < D; ++j) s0h = fma(-rk[k][j], sm[j].hi, s0h);
            s0 = DWt{s0h, F(0)};
          }
#pragma unroll
          for (int aa = D - 1; aa > 0; --aa)
#pragma unroll
            for (int bb = D - 1; bb > 0; --bb) Sg[aa][bb] = Sg[aa - 1][bb - 1];
          Sg[0][0] = s0;
#pragma unroll
          for (int m = 1; m < D; ++m) Sg[0][m] = Sg[m][0] = sm[m - 1];
          const F dv = s0.hi + s0.lo;
          const F wi = sw[st][k][tid];
          if (wi > F(0)) {  // tr H: each term rounded once, the running sum kept exact
            const DWt s2 = two_sum(trh.hi, wi * dv);
            trh.hi = s2.hi;
            trh.lo += s2.lo;
          }
          nanacc = fma(dv, F(0), nanacc);
          if (act) a.diag[(size_t)i * P + p] = okser ? dv : F(0);
        }
      }
      if (c >= 2) issue(c - 2, st);
    }
    // n - tr H is the residual degrees of freedom; where it is within rounding of zero the
    // smoother interpolates the observations and sigma^2 is not determined (NaN)
    const F den = n - (trh.hi + trh.lo);
    const bool undetermined = !(den > n * F(sizeof(F) == 4 ? 1e-4 : 1e-10));
    const bool nonfin = okser && (!(nanacc == F(0)) || undetermined);
    if (act) {
      a.den[p] = okser ? (undetermined ? F(NAN) : den) : F(-1);
      if (a.status != nullptr) a.status[p] = code != WS_SERIES_OK ? code : (nonfin ? WS_SERIES_NONFINITE : WS_SERIES_OK);
    }
  }
}

// One thread per (series p, band b); CTA index = series block * B + b.
template <typename F>
__global__ void __launch_bounds__(kSdNP) k_post_sd(int T, int B, int P, const F* __restrict__ x,
                                                   const F* __restrict__ z, const F* __restrict__ w,
                                                   const F* __restrict__ den, const F* __restrict__ diag,
                                                   F* __restrict__ sigma2, F* __restrict__ sd) {
  const int b = blockIdx.x % B;
  const int p = (blockIdx.x / B) * kSdNP + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P;
  const F* xp = x + (size_t)b * P + p;
  const F* zp = z + (size_t)b * P + p;
  const F* wp = w + p;
  // RSS_b = sum_t w_t (x_t - z_t)^2 over days with w_t > 0, as a compensated sum
  F sum = F(0), comp = F(0);
#pragma unroll 4
  for (int t = 0; t < T; ++t) {
    const F wt = wp[(size_t)t * sP];
    const F xv = xp[(size_t)t * sBP], zv = zp[(size_t)t * sBP];
    const F r = xv - zv;
    const F term = wt > F(0) ? wt * r * r : F(0);
    const F y = term - comp;
    const F s2 = sum + y;
    comp = (s2 - sum) - y;
    sum = s2;
  }
  const F dn = den[p];  // -1: no posterior (status NOT_PD or BADARG): zeros; NaN: undetermined
  const F s2b = dn < F(0) ? F(0) : sum / dn;
  sigma2[(size_t)b * P + p] = s2b;
  if (sd == nullptr) return;
  F* sp = sd + (size_t)b * P + p;
  const F* dp = diag + p;
#pragma unroll 4
  for (int t = 0; t < T; ++t) sp[(size_t)t * sBP] = sqrt(s2b * dp[(size_t)t * sP]);
}

// k_post_sd for FP32 with P % 4 == 0 and 16-byte aligned arrays: one thread per (4
// consecutive series, band), 16-byte loads and stores (512 bytes per warp instruction), four
// days of loads in flight per thread.
__global__ void __launch_bounds__(kSdNP) k_post_sd4(int T, int B, int P4, const float4* __restrict__ x,
                                                    const float4* __restrict__ z, const float4* __restrict__ w,
                                                    const float4* __restrict__ den, const float4* __restrict__ diag,
                                                    float4* __restrict__ sigma2, float4* __restrict__ sd) {
  const int b = blockIdx.x % B;
  const int q = (blockIdx.x / B) * kSdNP + threadIdx.x;
  if (q >= P4) return;
  const size_t sP = (size_t)P4, sBP = (size_t)B * P4;
  const float4* xp = x + (size_t)b * P4 + q;
  const float4* zp = z + (size_t)b * P4 + q;
  const float4* wp = w + q;
  float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
  auto acc = [&](int j, float wt, float xv, float zv) {
    const float r = xv - zv;
    const float term = wt > 0.f ? wt * r * r : 0.f;
    const float y = term - comp[j];
    const float s2 = sum[j] + y;
    comp[j] = (s2 - sum[j]) - y;
    sum[j] = s2;
  };
#pragma unroll 4
  for (int t = 0; t < T; ++t) {
    const float4 wt = __ldg(wp + (size_t)t * sP);
    const float4 xv = __ldcs(xp + (size_t)t * sBP), zv = __ldcs(zp + (size_t)t * sBP);
    acc(0, wt.x, xv.x, zv.x);
    acc(1, wt.y, xv.y, zv.y);
    acc(2, wt.z, xv.z, zv.z);
    acc(3, wt.w, xv.w, zv.w);
  }
  const float4 dn = den[q];
  const float dv[4] = {dn.x, dn.y, dn.z, dn.w};
  float s2b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) s2b[j] = dv[j] < 0.f ? 0.f : sum[j] / dv[j];
  sigma2[(size_t)b * P4 + q] = make_float4(s2b[0], s2b[1], s2b[2], s2b[3]);
  if (sd == nullptr) return;
  float4* sp = sd + (size_t)b * P4 + q;
  const float4* dp = diag + q;
#pragma unroll 4
  for (int t = 0; t < T; ++t) {
    const float4 g = __ldg(dp + (size_t)t * sP);
    __stcs(sp + (size_t)t * sBP, make_float4(sqrtf(s2b[0] * g.x), sqrtf(s2b[1] * g.y), sqrtf(s2b[2] * g.z),
                                            sqrtf(s2b[3] * g.w)));
  }
}

template <typename F, int D, bool DT = false>
static int post_occ(int& occ) {
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_post_diag<F, D, DT>, post_np<F>(), 0) != cudaSuccess ||
      occ < 1)
    return set_error(WS_ECUDA, "posterior: occupancy query");
  return WS_OK;
}

template <bool DT>
static int post_plan_t(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  const bool f64 = pb.dtype == WS_F64;
  int occ = 0;
  switch (pb.d) {
    case 1: rc = f64 ? post_occ<double, 1, DT>(occ) : post_occ<float, 1, DT>(occ); break;
    case 2: rc = f64 ? post_occ<double, 2, DT>(occ) : post_occ<float, 2, DT>(occ); break;
    case 3: rc = f64 ? post_occ<double, 3, DT>(occ) : post_occ<float, 3, DT>(occ); break;
    case 4: rc = f64 ? post_occ<double, 4, DT>(occ) : post_occ<float, 4, DT>(occ); break;
    default: return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
  }
  if (rc != WS_OK) return rc;
  const int np = f64 ? post_np<double>() : post_np<float>();
  const int n_tiles = (int)((pb.n_series + np - 1) / np);
  grid = std::max(1, std::min(n_tiles, di.sm_count * occ));
  nch = (pb.T + kPostC - 1) / kPostC;
  const int kpr = pb.d * (pb.d + 1) / 2;
  ck_bytes = (size_t)grid * nch * kpr * np * (f64 ? 8 : 4);
  return WS_OK;
}

int post_plan(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  return post_plan_t<false>(pb, grid, nch, ck_bytes);
}
int post_plan_dates(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  return post_plan_t<true>(pb, grid, nch, ck_bytes);
}

int post_plan_dates(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes);
int launch_posterior_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const void* lam,
                           const void* z, void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den,
                           cudaStream_t st);

template <typename F>
static int launch_post_t(const ws_problem& pb, const void* tt, const void* x, const void* w, const void* lam,
                         const void* z, void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den,
                         cudaStream_t st) {
  int grid = 0, nch = 0;
  size_t ckb = 0;
  const bool dt = tt != nullptr;
  int rc = dt ? post_plan_dates(pb, grid, nch, ckb) : post_plan(pb, grid, nch, ckb);
  if (rc != WS_OK) return rc;
  PostArgs<F> a;
  memset(&a, 0, sizeof(a));
  a.T = pb.T;
  a.P = (int)pb.n_series;
  a.nch = nch;
  constexpr int np = post_np<F>();
  a.n_tiles = (int)((pb.n_series + np - 1) / np);
  a.lam_scalar = pb.lam_mode == WS_LAM_SCALAR;
  a.w = static_cast<const F*>(w);
  a.lam = static_cast<const F*>(lam);
  a.diag = static_cast<F*>(diag);
  a.den = static_cast<F*>(den);
  a.status = status;
  a.ckpt = static_cast<F*>(ckpt);
  a.t = static_cast<const F*>(tt);
  if (dt) {
    switch (pb.d) {
      case 1: k_post_diag<F, 1, true><<<grid, np, 0, st>>>(a); break;
      case 2: k_post_diag<F, 2, true><<<grid, np, 0, st>>>(a); break;
      case 3: k_post_diag<F, 3, true><<<grid, np, 0, st>>>(a); break;
      case 4: k_post_diag<F, 4, true><<<grid, np, 0, st>>>(a); break;
    }
  } else {
    switch (pb.d) {
      case 1: k_post_diag<F, 1, false><<<grid, np, 0, st>>>(a); break;
      case 2: k_post_diag<F, 2, false><<<grid, np, 0, st>>>(a); break;
      case 3: k_post_diag<F, 3, false><<<grid, np, 0, st>>>(a); break;
      case 4: k_post_diag<F, 4, false><<<grid, np, 0, st>>>(a); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "posterior diagonal kernel launch: %s", cudaGetErrorString(e));
  const int B = pb.n_bands;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  const bool vec = sizeof(F) == 4 && pb.n_series % 4 == 0 && al16(x) && al16(z) && al16(w) && al16(den) &&
                   al16(diag) && al16(sigma2) && (sd == nullptr || al16(sd));
  const long long per = vec ? pb.n_series / 4 : pb.n_series;
  const long long blocks = ((per + kSdNP - 1) / kSdNP) * (long long)B;
  if (blocks > 0x7fffffffLL) return set_error(WS_EINVAL, "posterior: too many series x bands");
  if (vec)
    k_post_sd4<<<(unsigned)blocks, kSdNP, 0, st>>>(pb.T, B, (int)per, static_cast<const float4*>(x),
                                                   static_cast<const float4*>(z), static_cast<const float4*>(w),
                                                   static_cast<const float4*>(den), static_cast<const float4*>(diag),
                                                   static_cast<float4*>(sigma2), static_cast<float4*>(sd));
  else
    k_post_sd<F><<<(unsigned)blocks, kSdNP, 0, st>>>(pb.T, B, (int)pb.n_series, static_cast<const F*>(x),
                                                     static_cast<const F*>(z), static_cast<const F*>(w),
                                                     static_cast<const F*>(den), static_cast<const F*>(diag),
                                                     static_cast<F*>(sigma2), static_cast<F*>(sd));
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "posterior spread kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int launch_posterior(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z,
                     void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den, cudaStream_t st) {
  return launch_posterior_dates(pb, nullptr, x, w, lam, z, diag, sigma2, sd, status, ckpt, den, st);
}

int launch_posterior_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const void* lam,
                           const void* z, void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den,
                           cudaStream_t st) {
  if (pb.dtype == WS_F64)
    return launch_post_t<double>(pb, t, x, w, lam, z, diag, sigma2, sd, status, ckpt, den, st);
  return launch_post_t<float>(pb, t, x, w, lam, z, diag, sigma2, sd, status, ckpt, den, st);
}

}  // namespace ws
