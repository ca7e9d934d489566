// Smoothing on unevenly spaced sample times (Section 2): the series are kept on their
// acquisition dates t_0 < ... < t_{T-1} instead of a padded daily grid, and the order-d
// difference operator is the discrete derivative for uneven spacing that the paper adopts
// from the divided-difference literature it cites: row k is d! times the weights of the
// divided difference f[t_k, ..., t_{k+d}],
//     c_{k,j} = d! / prod_{m != j} (t_{k+j} - t_{k+m}),   j = 0..d,
// which on t = 0, 1, 2, ... is the binomial difference of the daily grid. Omega = W +
// D^T Lambda D keeps bandwidth d, so the solve is the same two-sweep rotation recurrence as
// on the daily grid (ws_sweep.cuh) with these per-row coefficients in place of the binomial
// ones; each thread forms its rows from a window of d + 1 dates.
//
// Layout: tile, time-major; t [T][P] (each series its own dates, e.g. a different
// acquisition phase), x, z [T][B][P], w, lambda [T][P] (entry k weights row k) or [P].
// One series per thread (128 per CTA in FP32, 64 in FP64), each thread staging its own
// column of x, w, t and lambda (chunks of 4 days, two LDGSTS stages, no block barrier).
// Pass 1: rotations + forward substitution, state checkpointed per chunk. Pass 2, chunks in
// reverse: the chunk is recomputed from its checkpoint (rho into registers, yhat written in
// place over the staged x), then back-substituted, z stored with coalesced plain stores.
// Bands beyond the per-thread group (up to 5 in FP32, 2 in FP64) run as further groups.
//
// Adjoint (ADJ, Section 2.3 on sample times): the same sweeps solve Omega g = dL/dz (the
// right-hand side unweighted); the backward pass then writes gx = W g and
// dL/dlambda_k = -sum_b (D g_b)_k (D z_b)_k [* lambda_k], with (D f)_k formed as nested
// divided differences (level q at day k: (level q-1 at k+1 - level q-1 at k) * q / (t_{k+q}
// - t_k), the recursive discrete derivative): on smooth sequences each subtraction is
// exact, where the expanded weights would cancel digits in FP32. z is staged with the
// backward pass's chunks (plain loads for the two chunks still resident from pass 1).
//
// Correction solve (RAW, the refinement step): the same sweeps with the residual as an
// unweighted right-hand side, the result added onto z0 (staged like z above) in place;
// k_dates_resid forms the residual beforehand.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"
#include "ws_dates.cuh"

namespace ws {

template <typename F>
constexpr int dates_np() { return sizeof(F) == 8 ? 64 : 128; }
constexpr int kDatesC = 4;

template <typename F>
struct DatesArgs {
  int T, P, B, b0, nch, n_tiles, lam_scalar, write_status;
  const F* t;      // [T][P]
  const F* x;      // [T][B][P]
  const F* w;      // [T][P]
  const F* lam;    // [T][P] or [P]
  F* z;            // [T][B][P]: z, or gx (ADJ)
  const F* zin;    // ADJ: the forward output z [T][B][P]
  F* glam;         // ADJ: dL/dlambda [T][P] or [P] (may be null)
  int loglam;      // ADJ: glam multiplied by lambda (the derivative in log lambda)
  uint8_t* status; // [P] or null
  F* ckpt;         // per CTA: nch * kFields * NP
};

// Shared memory of one stage, in rows of NP elements: x (C * NB), w (C + D), t (C + D), lambda
// (C), and for the adjoint and the correction solve z (C * NB: the forward output or z0, staged
// with the chunks of the backward pass).
__host__ __device__ constexpr int dates_stage_rows(int NB, int D, bool z) {
  return kDatesC * NB + 2 * (kDatesC + D) + kDatesC + (z ? kDatesC * NB : 0);
}

template <typename F, int D, int NB, int MODE>
__global__ void __launch_bounds__(dates_np<F>(), sizeof(F) == 4 ? 4 : 1) k_dates(const DatesArgs<F> a) {
  constexpr bool ADJ = MODE == 1, RAW = MODE == 2;
  constexpr int NP = dates_np<F>(), C = kDatesC;
  using SW = Sweep<F, D, NB>;
  constexpr int kF = SW::kFields;
  constexpr bool HZ = ADJ || RAW;
  constexpr int SR = dates_stage_rows(NB, D, HZ);
  constexpr int rW = C * NB, rT = rW + C + D, rL = rT + C + D, rZ = rL + C;
  extern __shared__ __align__(16) unsigned char dates_smem[];
  F* const sm = reinterpret_cast<F*>(dates_smem);
  const int tid = threadIdx.x;
  const int T = a.T, P = a.P, nch = a.nch;
  F* const ck = a.ckpt + (size_t)blockIdx.x * nch * kF * NP + tid;
  auto row = [&](int st, int r) -> F* { return sm + ((size_t)st * SR + r) * NP + tid; };

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int p = tile * NP + tid;
    const bool act = p < P;
    const size_t sBP = (size_t)a.B * P;
    const F* const xcol = a.x + (size_t)a.b0 * P + (act ? p : 0);  // this thread's column
    const size_t ocol = act ? (size_t)p : 0;
    const F* const zcol = HZ ? a.zin + (size_t)a.b0 * P + (act ? p : 0) : nullptr;
    auto issue = [&](int c, int st, bool withz) {
      const int t0 = c * C;
      const F* xr = xcol + (size_t)t0 * sBP;
      const F* lr = a.lam + (size_t)t0 * P + ocol;
      const F* wr = a.w + (size_t)t0 * P + ocol;
      const F* tr = a.t + (size_t)t0 * P + ocol;
#pragma unroll
      for (int k = 0; k < C; ++k) {
        const bool v = act && t0 + k < T;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          cp_async_elem<sizeof(F)>(row(st, k * NB + b), v ? xr + (size_t)k * sBP + (size_t)b * P : a.x, v);
        if (!a.lam_scalar) cp_async_elem<sizeof(F)>(row(st, rL + k), v ? lr + (size_t)k * P : a.lam, v);
      }
#pragma unroll
      for (int k = 0; k < C + D; ++k) {
        const bool v = act && t0 + k < T;
        cp_async_elem<sizeof(F)>(row(st, rW + k), v ? wr + (size_t)k * P : a.w, v);
        cp_async_elem<sizeof(F)>(row(st, rT + k), v ? tr + (size_t)k * P : a.t, v);
      }
      if (HZ && withz) {
        const F* zr = zcol + (size_t)t0 * sBP;
#pragma unroll
        for (int k = 0; k < C; ++k) {
          const bool v = act && t0 + k < T;
#pragma unroll
          for (int b = 0; b < NB; ++b)
            cp_async_elem<sizeof(F)>(row(st, rZ + k * NB + b), v ? zr + (size_t)k * sBP + (size_t)b * P : a.zin, v);
        }
      }
      cp_async_commit();
    };

    // ---- pass 1: rotations + forward substitution, checkpoints ----
    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    const F lam_s = (a.lam_scalar && act) ? a.lam[p] : F(0);
    issue(0, 0, false);
    if (nch > 1) issue(1, 1, false);
    for (int c = 0; c < nch; ++c) {
      if (c + 1 < nch) cp_async_wait<1>(); else cp_async_wait<0>();
      const int st = c & 1;
      if (c == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m)
          if (m < T) s.init_weight(m, *row(0, rW + m));
      }
      s.save(ck + (size_t)c * kF * NP, NP);
      const int nd = min(C, T - c * C);
      for (int k = 0; k < nd; ++k) {
        const int i = c * C + k;
        const F wi = *row(st, rW + k), wa = *row(st, rW + k + D);
        const F li = a.lam_scalar ? lam_s : *row(st, rL + k);
        const bool has_row = i < T - D;
        F tw[D + 1], cf[D + 1];
#pragma unroll
        for (int j = 0; j <= D; ++j) tw[j] = *row(st, rT + k + j);
        bad |= !(wi >= F(0)) || !finite_(wi) || !finite_(tw[0]);
        if (i + 1 < T) bad |= !(tw[1] > tw[0]);
        if (has_row) bad |= !(li > F(0)) || !finite_(li);
        npos += wi > F(0);
        if (has_row) dates_coef<F, D>(tw, cf);
        F bv[NB], rho[D], yh[NB], invD;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const F xv = *row(st, k * NB + b);
          bv[b] = (ADJ || RAW) ? xv : (wi > F(0) ? wi * xv : F(0));
        }
        dates_factor_step(s, has_row, li, wa, cf, rho, invD);
        s.subst_step(rho, invD, bv, yh);
      }
      if (c + 2 < nch) issue(c + 2, st, false);
    }
    const int dmin = D < T ? D : T;
    const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
    const bool okser = act && code == WS_SERIES_OK;

    // ---- pass 2: chunk recompute, back substitution ----
    F zc[NB][D];
    F lg[NB][D], lz[NB][D];  // ADJ: levels 0..D-1 of the divided differences of g, z at day i+1
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < D; ++q) {
        zc[b][q] = F(0);
        lg[b][q] = F(0);
        lz[b][q] = F(0);
      }
    F nanacc = F(0);
    F glam_sum = F(0);
    for (int c = nch - 1; c >= 0; --c) {
      const int st = c & 1;
      if (c < nch - 2) {
        if (c >= 1) cp_async_wait<1>(); else cp_async_wait<0>();
      }
      s.load(ck + (size_t)c * kF * NP, NP);
      const int nd = min(C, T - c * C);
      const bool zstaged = HZ && c < nch - 2;
      F rk[C][D];
#pragma unroll
      for (int k = 0; k < C; ++k) {
        if (k < nd) {
          const int i = c * C + k;
          const F wi = *row(st, rW + k), wa = *row(st, rW + k + D);
          const F li = a.lam_scalar ? lam_s : *row(st, rL + k);
          const bool has_row = i < T - D;
          F tw[D + 1], cf[D + 1];
#pragma unroll
          for (int j = 0; j <= D; ++j) tw[j] = *row(st, rT + k + j);
          if (has_row) dates_coef<F, D>(tw, cf);
          F bv[NB], rho[D], yh[NB], invD;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const F xv = *row(st, k * NB + b);
            bv[b] = (ADJ || RAW) ? xv : (wi > F(0) ? wi * xv : F(0));
          }
          dates_factor_step(s, has_row, li, wa, cf, rho, invD);
          s.subst_step(rho, invD, bv, yh);
#pragma unroll
          for (int b = 0; b < NB; ++b) *row(st, k * NB + b) = yh[b];
#pragma unroll
          for (int j = 0; j < D; ++j) rk[k][j] = rho[j];
        }
      }
#pragma unroll
      for (int k = C - 1; k >= 0; --k) {
        if (k < nd) {
          const int i = c * C + k;
          F sq[D + 1];  // ADJ: q / (t_{i+q} - t_i), 0 where day i+q is past the end
          F wk = F(0);
          if (ADJ) {
            wk = *row(st, rW + k);
            const F t0 = *row(st, rT + k);
#pragma unroll
            for (int q = 1; q <= D; ++q) sq[q] = i + q < T ? F(q) / (*row(st, rT + k + q) - t0) : F(0);
          }
          F dl = F(0);
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            F acc = *row(st, k * NB + b);
#pragma unroll
            for (int q = 0; q < D; ++q) acc = fma(-rk[k][q], zc[b][q], acc);
#pragma unroll
            for (int q = D - 1; q > 0; --q) zc[b][q] = zc[b][q - 1];
            zc[b][0] = acc;
            F out = okser ? acc : F(0);
            if (ADJ) {
              // z staged with the chunk, except for the two chunks still resident from pass 1
              const F zv = zstaged ? *row(st, rZ + k * NB + b) : (act ? a.zin[((size_t)i * a.B + a.b0 + b) * P + p] : F(0));
              F cg = out, cz = zv;
#pragma unroll
              for (int q = 1; q <= D; ++q) {
                const F ng = (lg[b][q - 1] - cg) * sq[q], nz = (lz[b][q - 1] - cz) * sq[q];
                lg[b][q - 1] = cg;
                lz[b][q - 1] = cz;
                cg = ng;
                cz = nz;
              }
              dl = fma(cg, cz, dl);
              out = wk * out;
            }
            if (RAW && act)  // z0 + correction
              out += zstaged ? *row(st, rZ + k * NB + b) : a.zin[((size_t)i * a.B + a.b0 + b) * P + p];
            nanacc = fma(out, F(0), nanacc);
            if (act) a.z[((size_t)i * a.B + a.b0 + b) * P + p] = out;
          }
          if (ADJ && a.glam != nullptr && act) {
            F gl_i = (okser && i < T - D) ? -dl : F(0);
            if (a.loglam) gl_i *= a.lam_scalar ? lam_s : *row(st, rL + k);
            if (a.lam_scalar) {
              glam_sum += gl_i;
            } else {
              F* dst = a.glam + (size_t)i * P + p;
              *dst = a.b0 == 0 ? gl_i : *dst + gl_i;
            }
          }
        }
      }
      if (c >= 2) issue(c - 2, st, true);
    }
    if (ADJ && a.glam != nullptr && a.lam_scalar && act) a.glam[p] = a.b0 == 0 ? glam_sum : a.glam[p] + glam_sum;
    if (act && a.status != nullptr) {
      const bool nonfin = !(nanacc == F(0));
      if (a.write_status)
        a.status[p] = code != WS_SERIES_OK ? code : (nonfin ? WS_SERIES_NONFINITE : WS_SERIES_OK);
      else if (nonfin && a.status[p] == WS_SERIES_OK)
        a.status[p] = WS_SERIES_NONFINITE;
    }
  }
}

template <typename F, int D, int NB, int MODE>
static int dates_cfg_t(int n_tiles, int& grid, size_t& smem) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  constexpr int NP = dates_np<F>();
  smem = (size_t)2 * dates_stage_rows(NB, D, MODE != 0) * NP * sizeof(F);
  auto kern = k_dates<F, D, NB, MODE>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return set_error(WS_ECUDA, "dates: shared memory attribute");
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NP, smem) != cudaSuccess || occ < 1)
    return set_error(WS_ECUDA, "dates: occupancy query");
  grid = std::max(1, std::min(n_tiles, di.sm_count * occ));
  return WS_OK;
}

// Bands per thread of a group: FP32 1, 2, 4 or 5 (the adjoint, with its difference
// triangles, at most 4); FP64 1 or 2.
static int dates_group(const ws_problem& pb, int left, int mode) {
  if (pb.dtype == WS_F64) return left >= 2 ? 2 : 1;
  if (left >= 5 && mode != 1) return left == 8 ? 4 : 5;
  if (left >= 4) return 4;
  return left >= 2 ? 2 : 1;
}

template <typename T>
struct type_tag {
  using type = T;
};

// Runs `fn` (a generic lambda taking the kernel's compile-time parameters as
// integral_constant arguments) for the instantiation of (dtype, d, nb, mode).
template <typename Fn>
static int dates_dispatch(const ws_problem& pb, int nb, int mode, Fn&& fn) {
  using std::integral_constant;
  auto by_nb = [&](auto ft, auto dd, auto aj) -> int {
    using FT = typename decltype(ft)::type;
    if constexpr (sizeof(FT) == 8) {
      if (nb == 2) return fn(ft, dd, integral_constant<int, 2>{}, aj);
      return fn(ft, dd, integral_constant<int, 1>{}, aj);
    } else {
      switch (nb) {
        case 1: return fn(ft, dd, integral_constant<int, 1>{}, aj);
        case 2: return fn(ft, dd, integral_constant<int, 2>{}, aj);
        case 4: return fn(ft, dd, integral_constant<int, 4>{}, aj);
        case 5:
          if constexpr (decltype(aj)::value != 1) return fn(ft, dd, integral_constant<int, 5>{}, aj);
          break;
      }
      return set_error(WS_EUNSUPPORTED, "dates: band group of %d", nb);
    }
  };
  auto by_d = [&](auto ft, auto aj) -> int {
    switch (pb.d) {
      case 1: return by_nb(ft, integral_constant<int, 1>{}, aj);
      case 2: return by_nb(ft, integral_constant<int, 2>{}, aj);
      case 3: return by_nb(ft, integral_constant<int, 3>{}, aj);
      case 4: return by_nb(ft, integral_constant<int, 4>{}, aj);
    }
    return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
  };
  auto by_adj = [&](auto ft) -> int {
    if (mode == 1) return by_d(ft, integral_constant<int, 1>{});
    if (mode == 2) return by_d(ft, integral_constant<int, 2>{});
    return by_d(ft, integral_constant<int, 0>{});
  };
  if (pb.dtype == WS_F64) return by_adj(type_tag<double>{});
  return by_adj(type_tag<float>{});
}

// Checkpoint bytes (the largest over the problem's band groups; groups run in turn).
static int dates_plan_mode(const ws_problem& pb, int mode, size_t& ck_bytes) {
  ck_bytes = 0;
  const bool f64 = pb.dtype == WS_F64;
  const int np = f64 ? dates_np<double>() : dates_np<float>();
  const int n_tiles = (int)((pb.n_series + np - 1) / np);
  const int nch = (pb.T + kDatesC - 1) / kDatesC;
  for (int b0 = 0; b0 < pb.n_bands;) {
    const int nb = dates_group(pb, pb.n_bands - b0, mode);
    int grid = 0;
    size_t smem = 0;
    int rc = dates_dispatch(pb, nb, mode, [&](auto ft, auto dd, auto nbb, auto aj) -> int {
      return dates_cfg_t<typename decltype(ft)::type, decltype(dd)::value, decltype(nbb)::value,
                         decltype(aj)::value>(n_tiles, grid, smem);
    });
    if (rc != WS_OK) return rc;
    const int fields = pb.d * (pb.d + 1) + nb * pb.d;
    ck_bytes = std::max(ck_bytes, (size_t)grid * nch * fields * np * (f64 ? 8 : 4));
    b0 += nb;
  }
  return WS_OK;
}

int dates_plan(const ws_problem& pb, bool adj, size_t& ck_bytes) {
  size_t a = 0, b = 0;
  int rc = dates_plan_mode(pb, adj ? 1 : 0, a);
  if (rc == WS_OK && !adj) rc = dates_plan_mode(pb, 2, b);
  ck_bytes = std::max(a, b);
  return rc;
}

template <typename F>
static int dates_run_t(const ws_problem& pb, int mode, const void* t, const void* x, const void* w,
                       const void* lam, void* out, const void* zin, void* glam, int loglam, uint8_t* status,
                       void* ckpt, cudaStream_t st) {
  DatesArgs<F> a;
  memset(&a, 0, sizeof(a));
  constexpr int np = dates_np<F>();
  a.T = pb.T;
  a.P = (int)pb.n_series;
  a.B = pb.n_bands;
  a.nch = (pb.T + kDatesC - 1) / kDatesC;
  a.n_tiles = (int)((pb.n_series + np - 1) / np);
  a.lam_scalar = pb.lam_mode == WS_LAM_SCALAR;
  a.t = static_cast<const F*>(t);
  a.x = static_cast<const F*>(x);
  a.w = static_cast<const F*>(w);
  a.lam = static_cast<const F*>(lam);
  a.z = static_cast<F*>(out);
  a.zin = static_cast<const F*>(zin);
  a.glam = static_cast<F*>(glam);
  a.loglam = loglam;
  a.status = status;
  a.ckpt = static_cast<F*>(ckpt);
  for (int b0 = 0; b0 < pb.n_bands;) {
    const int nb = dates_group(pb, pb.n_bands - b0, mode);
    a.b0 = b0;
    a.write_status = b0 == 0 && mode != 2;
    int rc = dates_dispatch(pb, nb, mode, [&](auto ft, auto dd, auto nbb, auto aj) -> int {
      using FT = typename decltype(ft)::type;
      constexpr int DD = decltype(dd)::value, NBB = decltype(nbb)::value;
      constexpr int AJ = decltype(aj)::value;
      if constexpr (!std::is_same_v<FT, F>) {
        return set_error(WS_EINVAL, "dates: dtype mismatch");
      } else {
        int grid = 0;
        size_t smem = 0;
        int rc2 = dates_cfg_t<F, DD, NBB, AJ>(a.n_tiles, grid, smem);
        if (rc2 != WS_OK) return rc2;
        k_dates<F, DD, NBB, AJ><<<grid, np, smem, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_error(WS_ECUDA, "dates kernel launch: %s", cudaGetErrorString(e));
        return WS_OK;
      }
    });
    if (rc != WS_OK) return rc;
    b0 += nb;
  }
  return WS_OK;
}

int launch_dates(const ws_problem& pb, bool adj, const void* t, const void* x, const void* w, const void* lam,
                 void* out, const void* zin, void* glam, int loglam, uint8_t* status, void* ckpt, cudaStream_t st) {
  const int mode = adj ? 1 : 0;
  if (pb.dtype == WS_F64) return dates_run_t<double>(pb, mode, t, x, w, lam, out, zin, glam, loglam, status, ckpt, st);
  return dates_run_t<float>(pb, mode, t, x, w, lam, out, zin, glam, loglam, status, ckpt, st);
}

// ---- refinement on dates: residual r = W x - Omega z0, then Omega d = r, z = z0 + d ----

// One thread per (series, band); CTA index = series block * B + b (the bands of a block of
// series are adjacent, so w, lambda and t reach them through L2). Streaming over the days
// with delay lines of d + 1 values:
//   (D z0)_k as nested divided differences (level l at day k from level l - 1 at days k,
//     k + 1, times l / (t_{k+l} - t_k)), available when day k + d is read;
//   q_k = lambda_k (D z0)_k;
//   (D^T q)_k by the transposed recursion: v = u * l / (t_{k+l} - t_k) for l = d .. 1 (0 past
//     the level's last row), u <- v_{k-1} - v_k (a backward difference);
//   r_k = w_k (x_k - z0_k) - (D^T q)_k, with x - z0 split exactly by TwoSum and the
//     combination rounded once (FMA): the result is small against its terms.
template <typename F, int D>
__global__ void __launch_bounds__(128) k_dates_resid(int T, int B, int P, const F* __restrict__ t,
                                                     const F* __restrict__ x, const F* __restrict__ w,
                                                     const F* __restrict__ lam, int lam_scalar,
                                                     const F* __restrict__ z0, F* __restrict__ r) {
  const int b = blockIdx.x % B;
  const int p = (blockIdx.x / B) * 128 + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P, sBP = (size_t)B * P, ob = (size_t)b * P + p;
  const F lam_s = lam_scalar ? lam[p] : F(0);
  F tw[D + 1];               // t_{s}, t_{s-1}, ..., t_{s-D}
  F fl[D];                   // forward levels 0..D-1 at the previous step
  F zq[D + 1], xq[D + 1], wq[D + 1], lq[D + 1];  // delay lines (index j: day s - j)
  F vv[D + 1];               // transposed levels 1..D at the previous column
#pragma unroll
  for (int j = 0; j <= D; ++j) {
    tw[j] = F(0);
    zq[j] = xq[j] = wq[j] = lq[j] = vv[j] = F(0);
  }
#pragma unroll
  for (int j = 0; j < D; ++j) fl[j] = F(0);
#pragma unroll 4
  for (int s = 0; s < T + D; ++s) {
    const bool in = s < T;
    const F ts = in ? t[(size_t)s * sP + p] : tw[0];
    const F zs = in ? z0[(size_t)s * sBP + ob] : F(0);
    const F ws = in ? w[(size_t)s * sP + p] : F(0);
    const F xs = (in && ws > F(0)) ? x[(size_t)s * sBP + ob] : zs;  // gaps: x - z0 = 0
    const F ls = in ? (lam_scalar ? lam_s : lam[(size_t)s * sP + p]) : F(0);
#pragma unroll
    for (int j = D; j > 0; --j) {
      tw[j] = tw[j - 1];
      zq[j] = zq[j - 1];
      xq[j] = xq[j - 1];
      wq[j] = wq[j - 1];
      lq[j] = lq[j - 1];
    }
    tw[0] = ts;
    zq[0] = zs;
    xq[0] = xs;
    wq[0] = ws;
    lq[0] = ls;
    // forward: levels of day s - l, the last one (D z0)_{s-D}
    F cur = zs;
    if (in) {
#pragma unroll
      for (int l = 1; l <= D; ++l) {
        const F nw = s >= l ? (cur - fl[l - 1]) * (F(l) / (ts - tw[l])) : F(0);
        fl[l - 1] = cur;
        cur = nw;
      }
    }
    const int k = s - D;  // the column finished at this step
    if (k < 0) continue;
    const F q = (in && k <= T - D - 1) ? lq[D] * cur : F(0);
    // transposed recursion down to level 0
    F u = q;
#pragma unroll
    for (int l = D; l >= 1; --l) {
      const F v = (k <= T - l - 1) ? u * (F(l) / (tw[D - l] - tw[D])) : F(0);
      const F un = vv[l] - v;
      vv[l] = v;
      u = un;
    }
    // r_k = w_k (x_k - z0_k) - (D^T q)_k
    const DW<F> e = two_sum(xq[D], -zq[D]);
    r[(size_t)k * sBP + ob] = fma(wq[D], e.lo, fma(wq[D], e.hi, -u));
  }
}

int launch_dates_refine(const ws_problem& pb, const void* t, const void* x, const void* w, const void* lam, void* z,
                        void* r, void* ckpt, cudaStream_t st) {
  const int B = pb.n_bands, P = (int)pb.n_series;
  const long long blocks = ((pb.n_series + 127) / 128) * (long long)B;
  if (blocks > 0x7fffffffLL) return set_error(WS_EINVAL, "dates refinement: too many series x bands");
  const int ls = pb.lam_mode == WS_LAM_SCALAR;
  const bool f64 = pb.dtype == WS_F64;
#define WS_DR(FT, DD)                                                                                        \
  k_dates_resid<FT, DD><<<(unsigned)blocks, 128, 0, st>>>(pb.T, B, P, (const FT*)t, (const FT*)x, (const FT*)w, \
                                                         (const FT*)lam, ls, (const FT*)z, (FT*)r)
  switch (pb.d) {
    case 1: if (f64) WS_DR(double, 1); else WS_DR(float, 1); break;
    case 2: if (f64) WS_DR(double, 2); else WS_DR(float, 2); break;
    case 3: if (f64) WS_DR(double, 3); else WS_DR(float, 3); break;
    case 4: if (f64) WS_DR(double, 4); else WS_DR(float, 4); break;
    default: return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
  }
#undef WS_DR
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "dates residual launch: %s", cudaGetErrorString(e));
  // correction: Omega d = r with the same rotations, accumulated onto z in place
  if (f64) return dates_run_t<double>(pb, 2, t, r, w, lam, z, z, nullptr, 0, nullptr, ckpt, st);
  return dates_run_t<float>(pb, 2, t, r, w, lam, z, z, nullptr, 0, nullptr, ckpt, st);
}

}  // namespace ws
