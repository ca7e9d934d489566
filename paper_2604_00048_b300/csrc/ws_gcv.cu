// Generalized cross-validation over a grid of scalar lambda values, per series.
//
// The paper lists ways of choosing lambda but defines none; the score here is the
// Craven-Wahba GCV: for each grid value, z = Omega^{-1} W x (Eq. 2), RSS = sum_t w_t (x_t -
// z_t)^2, tr H = sum_t w_t (Omega^{-1})_tt with H = Omega^{-1} W, n = sum_t w_t, and
// V = n RSS / (n - tr H)^2. The smallest V wins; ties go to the smaller lambda.
//
// diag(Omega^{-1}) comes from the banded selected-inverse recursion (Takahashi, Fagan and
// Chin, 1973) on the same factor the solve uses: with Omega = U^T diag(1/invD) U, U unit
// upper with U[t][t+j] = rho_{t,j}, the entries Sigma = Omega^{-1} within the band obey,
// backwards in t,
//     Sigma[t][t+m] = - sum_{j=1..d} rho_{t,j} Sigma[t+j][t+m]       (m = 1..d)
//     Sigma[t][t]   = invD_t - sum_{j=1..d} rho_{t,j} Sigma[t][t+j],
// so a d x d window of Sigma rides along the back substitution. For d >= 3 the window is
// carried in double-word arithmetic: for large lambda rho approaches the difference
// coefficients and rho^T Sigma rho is a d-th difference of a smooth function, so FP32 loses
// up to ~1e-2 of tr H at d = 3 (errors grow like t^(d-1) through the recursion). At d <= 2
// FP32 keeps tr H to ~4e-4 at lambda = 1e5, which moves V by ~3e-5 (tr H << n there), so
// the window stays FP32; rho and invD are FP32 in both cases.
//
// Mapping: one thread per (series, grid value). A CTA holds 16 series x 16 grid values;
// the 16 lanes of a half-warp share a series, whose x and w chunks are staged once into
// shared memory (LDGSTS) and read by broadcast, so HBM sees x and w once per sweep for all
// 16 values. Pass 1 runs the factor and forward substitution with a checkpoint per chunk;
// pass 2 goes back over the chunks, recomputes each chunk's factor rows into registers
// (chunk length a compile-time 16) and does the back substitution, the selected inverse,
// RSS and tr H. The argmin is a shuffle over the half-warp.
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

constexpr int kGcvPix = 16;                    // series per CTA
constexpr int kGcvG = 16;                      // grid values per series (one per lane)
constexpr int kGcvThreads = kGcvPix * kGcvG;   // 256
constexpr int kGcvC = 16;                      // days per chunk

struct GcvArgs {
  int T, P, n_groups, nch, n_grid;
  float grid[kGcvG];
  const float* x;   // [T][P] (tile layout, one band)
  const float* w;   // [T][P]
  float* lam_best;  // [P]
  float* scores;    // [n_grid][P] or null
  float* ckpt;      // per CTA: nch * fields * 256
  const float* t;   // sample times [T][P] (the uneven-spacing operator) or null (daily grid)
};

// DT: the rows of D come from each series' sample times (staged like w).
template <int D, bool DT>
__global__ void __launch_bounds__(kGcvThreads, 2) k_gcv(const GcvArgs a) {
  using SW = Sweep<float, D, 1>;
  constexpr int kF = SW::kFields;
  __shared__ float sx[2][kGcvC][kGcvPix];
  __shared__ float sw[2][kGcvC + D][kGcvPix];
  __shared__ float stt[2][DT ? kGcvC + D : 1][kGcvPix];
  const int tid = threadIdx.x, g = tid & (kGcvG - 1), pl = tid / kGcvG;
  const float lam = a.grid[g < a.n_grid ? g : 0];
  const int T = a.T, P = a.P, nch = a.nch;
  float* ck = a.ckpt + (size_t)blockIdx.x * nch * kF * kGcvThreads + tid;

  for (int grp = blockIdx.x; grp < a.n_groups; grp += gridDim.x) {
    const int p0 = grp * kGcvPix, p = p0 + pl;
    const bool live = p < P;
    // stage chunk c: C x-rows and C + D w-rows of the CTA's 16 series (zero outside)
    auto issue = [&](int c, int st) {
      const int t0 = c * kGcvC;
      constexpr int kRows = 2 * kGcvC + D + (DT ? kGcvC + D : 0);
      for (int e = tid; e < kRows * kGcvPix; e += kGcvThreads) {
        const int row = e / kGcvPix, col = e % kGcvPix, pp = p0 + col;
        if (row < kGcvC) {
          const int t = t0 + row;
          const bool v = t < T && pp < P;
          cp_async_elem<4>(&sx[st][row][col], a.x + (v ? (size_t)t * P + pp : 0), v);
        } else if (row < 2 * kGcvC + D) {
          const int t = t0 + row - kGcvC;
          const bool v = t < T && pp < P;
          cp_async_elem<4>(&sw[st][row - kGcvC][col], a.w + (v ? (size_t)t * P + pp : 0), v);
        } else if constexpr (DT) {
          const int t = t0 + row - 2 * kGcvC - D;
          const bool v = t < T && pp < P;
          cp_async_elem<4>(&stt[st][row - 2 * kGcvC - D][col], a.t + (v ? (size_t)t * P + pp : 0), v);
        }
      }
      cp_async_commit();
    };
    // rotation step of day i = c * C + k from the staged chunk (daily binomial rows, or the
    // rows formed from the series' dates)
    auto fstep = [&](SW& sv, int st, int k, int i, float wa, float (&rho)[D], float& invD) {
      if constexpr (DT) {
        float tw[D + 1], cf[D + 1];
#pragma unroll
        for (int j = 0; j <= D; ++j) tw[j] = stt[st][k + j][pl];
        if (i < T - D) dates_coef<float, D>(tw, cf);
        dates_factor_step(sv, i < T - D, lam, wa, cf, rho, invD);
      } else {
        sv.factor_step(i < T - D, lam, wa, rho, invD);
      }
    };

    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    float n = 0.f;
    issue(0, 0);
    if (nch > 1) issue(1, 1);
    for (int c = 0; c < nch; ++c) {
      if (c + 1 < nch) cp_async_wait<1>(); else cp_async_wait<0>();
      __syncthreads();
      const int st = c & 1;
      if (c == 0)
        for (int m = 0; m < D; ++m)
          if (m < T) s.init_weight(m, sw[0][m][pl]);
      s.save(ck + (size_t)c * kF * kGcvThreads, kGcvThreads);
      const int nd = min(kGcvC, T - c * kGcvC);
#pragma unroll 2
      for (int k = 0; k < nd; ++k) {
        const int i = c * kGcvC + k;
        const float wi = sw[st][k][pl], wa = sw[st][k + D][pl], xi = sx[st][k][pl];
        bad |= !(wi >= 0.f && wi <= 3.4028235e38f);  // negative, NaN or infinite
        if constexpr (DT) {
          bad |= !isfinite(stt[st][k][pl]);
          if (i + 1 < T) bad |= !(stt[st][k + 1][pl] > stt[st][k][pl]);
        }
        npos += wi > 0.f;
        n += wi;
        float bv[1] = {wi > 0.f ? wi * xi : 0.f};
        float rho[D], yh[1], invD;
        fstep(s, st, k, i, wa, rho, invD);
        s.subst_step(rho, invD, bv, yh);
      }
      __syncthreads();
      if (c + 2 < nch) issue(c + 2, st);
    }
    const bool okser = live && !bad && npos >= (D < T ? D : T);

    using DWf = DW<float>;
    constexpr bool kDWin = D >= 3;
    float zc[D];
    DWf Sg[D][D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      zc[j] = 0.f;
#pragma unroll
      for (int m = 0; m < D; ++m) Sg[j][m] = DWf{0.f, 0.f};
    }
    float rss = 0.f, trh = 0.f;
    for (int c = nch - 1; c >= 0; --c) {
      const int st = c & 1;
      if (c < nch - 2) {
        if (c >= 1) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();
      }
      s.load(ck + (size_t)c * kF * kGcvThreads, kGcvThreads);
      const int nd = min(kGcvC, T - c * kGcvC);
      float yk[kGcvC], ik[kGcvC], rk[kGcvC][D];
#pragma unroll
      for (int k = 0; k < kGcvC; ++k) {
        if (k < nd) {
          const int i = c * kGcvC + k;
          const float wi = sw[st][k][pl], wa = sw[st][k + D][pl], xi = sx[st][k][pl];
          float bv[1] = {wi > 0.f ? wi * xi : 0.f};
          float rho[D], yh[1], invD;
          fstep(s, st, k, i, wa, rho, invD);
          s.subst_step(rho, invD, bv, yh);
          yk[k] = yh[0];
          ik[k] = invD;
#pragma unroll
          for (int j = 0; j < D; ++j) rk[k][j] = rho[j];
        }
      }
#pragma unroll
      for (int k = kGcvC - 1; k >= 0; --k) {
        if (k < nd) {
          // back substitution: z_t = yhat_t - sum_j rho_{t,j} z_{t+j}
          float z = yk[k];
#pragma unroll
          for (int j = 0; j < D; ++j) z = fmaf(-rk[k][j], zc[j], z);
#pragma unroll
          for (int j = D - 1; j > 0; --j) zc[j] = zc[j - 1];
          zc[0] = z;
          // selected inverse: Sg[a][b] = Sigma[t+1+a][t+1+b] on entry
          DWf sm[D];
          DWf s0 = {ik[k], 0.f};
          if (kDWin) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
              DWf acc = {0.f, 0.f};
#pragma unroll
              for (int j = 0; j < D; ++j) acc = dw_fma(acc, rk[k][j], Sg[j][m]);
              sm[m] = DWf{-acc.hi, -acc.lo};  // Sigma[t][t+1+m]
            }
#pragma unroll
            for (int j = 0; j < D; ++j) s0 = dw_fma(s0, -rk[k][j], sm[j]);
          } else {  // FP32 window (the lo parts stay zero)
#pragma unroll
            for (int m = 0; m < D; ++m) {
              float acc = 0.f;
#pragma unroll
              for (int j = 0; j < D; ++j) acc = fmaf(rk[k][j], Sg[j][m].hi, acc);
              sm[m] = DWf{-acc, 0.f};
            }
            float s0h = ik[k];
#pragma unroll
            for (int j = 0; j < D; ++j) s0h = fmaf(-rk[k][j], sm[j].hi, s0h);
            s0 = DWf{s0h, 0.f};
          }
#pragma unroll
          for (int aa = D - 1; aa > 0; --aa)
#pragma unroll
            for (int bb = D - 1; bb > 0; --bb) Sg[aa][bb] = Sg[aa - 1][bb - 1];
          Sg[0][0] = s0;
#pragma unroll
          for (int m = 1; m < D; ++m) Sg[0][m] = Sg[m][0] = sm[m - 1];
          const float wi = sw[st][k][pl], xi = sx[st][k][pl];
          if (wi > 0.f) {
            const float r = xi - z;
            rss = fmaf(wi * r, r, rss);
            trh = fmaf(wi, s0.hi + s0.lo, trh);
          }
        }
      }
      __syncthreads();
      if (c >= 2) issue(c - 2, st);
    }

    // score and argmin over the half-warp (NaN and unused slots count as +inf)
    const float den = n - trh;
    float V = n * rss / (den * den);
    if (!(V == V) || g >= a.n_grid || !okser) V = INFINITY;
    if (a.scores != nullptr && live && g < a.n_grid) a.scores[(size_t)g * P + p] = okser ? V : NAN;
    float bvv = V;
    int bi = g;
#pragma unroll
    for (int off = kGcvG / 2; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bvv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov < bvv || (ov == bvv && oi < bi)) {
        bvv = ov;
        bi = oi;
      }
    }
    if (g == 0 && live) a.lam_best[p] = a.grid[bi];
  }
}

template <int D, bool DT = false>
static int gcv_grid_t(int n_groups, int& grid) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gcv<D, DT>, kGcvThreads, 0) != cudaSuccess || occ < 1)
    return set_error(WS_ECUDA, "gcv: occupancy query");
  grid = std::min(n_groups, di.sm_count * occ);
  if (grid < 1) grid = 1;
  return WS_OK;
}

template <bool DT>
static int gcv_plan_t(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  const int n_groups = (int)((pb.n_series + kGcvPix - 1) / kGcvPix);
  int rc = WS_EINVAL;
  switch (pb.d) {
    case 1: rc = gcv_grid_t<1, DT>(n_groups, grid); break;
    case 2: rc = gcv_grid_t<2, DT>(n_groups, grid); break;
    case 3: rc = gcv_grid_t<3, DT>(n_groups, grid); break;
    case 4: rc = gcv_grid_t<4, DT>(n_groups, grid); break;
    default: return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
  }
  if (rc != WS_OK) return rc;
  nch = (pb.T + kGcvC - 1) / kGcvC;
  const int fields = pb.d * (pb.d + 1) + pb.d;
  ck_bytes = (size_t)grid * nch * fields * kGcvThreads * sizeof(float);
  return WS_OK;
}

int gcv_plan(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  return gcv_plan_t<false>(pb, grid, nch, ck_bytes);
}
int gcv_plan_dates(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes) {
  return gcv_plan_t<true>(pb, grid, nch, ck_bytes);
}

int launch_gcv_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const float* grid_vals,
                     int n_grid, float* lam_best, float* scores, void* ckpt, cudaStream_t st);

int launch_gcv(const ws_problem& pb, const void* x, const void* w, const float* grid_vals, int n_grid,
               float* lam_best, float* scores, void* ckpt, cudaStream_t st) {
  return launch_gcv_dates(pb, nullptr, x, w, grid_vals, n_grid, lam_best, scores, ckpt, st);
}

int launch_gcv_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const float* grid_vals,
                     int n_grid, float* lam_best, float* scores, void* ckpt, cudaStream_t st) {
  GcvArgs a;
  memset(&a, 0, sizeof(a));
  int grid = 0, nch = 0;
  size_t ckb = 0;
  const bool dt = t != nullptr;
  int rc = dt ? gcv_plan_t<true>(pb, grid, nch, ckb) : gcv_plan_t<false>(pb, grid, nch, ckb);
  if (rc != WS_OK) return rc;
  a.T = pb.T;
  a.P = (int)pb.n_series;
  a.n_groups = (int)((pb.n_series + kGcvPix - 1) / kGcvPix);
  a.nch = nch;
  a.n_grid = n_grid;
  for (int g = 0; g < n_grid; ++g) a.grid[g] = grid_vals[g];
  a.x = static_cast<const float*>(x);
  a.w = static_cast<const float*>(w);
  a.lam_best = lam_best;
  a.scores = scores;
  a.ckpt = static_cast<float*>(ckpt);
  a.t = static_cast<const float*>(t);
  if (dt) {
    switch (pb.d) {
      case 1: k_gcv<1, true><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 2: k_gcv<2, true><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 3: k_gcv<3, true><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 4: k_gcv<4, true><<<grid, kGcvThreads, 0, st>>>(a); break;
    }
  } else {
    switch (pb.d) {
      case 1: k_gcv<1, false><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 2: k_gcv<2, false><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 3: k_gcv<3, false><<<grid, kGcvThreads, 0, st>>>(a); break;
      case 4: k_gcv<4, false><<<grid, kGcvThreads, 0, st>>>(a); break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "gcv kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

}  // namespace ws
