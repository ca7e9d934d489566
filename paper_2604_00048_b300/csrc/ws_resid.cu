// Residual of the smoothing system for one step of iterative refinement:
//     r = W x - Omega z0 = W (x - z0) - D^T (Lambda (D z0))        (Omega from Eq. 3)
// or, for a right-hand side taken as given (the adjoint solve Omega g = gz),
//     r = x - Omega z0 = x - W z0 - D^T (Lambda (D z0)).
// At a good z0 the two terms cancel to a few parts in 1e5. D z0 and D^T q are taken
// as nested first differences (exact on smooth sequences, where the binomial sums
// would cancel digits), and the final combination is a double word (ws_df.cuh).
// Every band streams through rings of the last d+1 values of z0 and of
// q_k = lambda_k (D z0)_k: pushing z0_u completes the difference row k = u - d, and with
// it the residual of day t = u - d.
//
// Two kernels over the pixel-fastest tile layout:
//   k_residual_tma  CTA = 128 pixels x up to 10 bands x a block of kResidDaysTma days.
//                   Chunks of C days of z0, x, w and lambda are staged in shared memory
//                   by TMA (cp.async.bulk.tensor) through a ring of NS stages with
//                   mbarrier completion, so the loads in flight per SM do not depend on
//                   the registers of the arithmetic; each thread owns one pixel and up to
//                   5 bands (two threads per pixel above 5 bands).
//   k_residual      thread = one pixel x a block of kResidDays days x up to 5 bands, plain
//                   coalesced loads (used when TMA cannot describe the arrays: row pitch
//                   not a multiple of 16 bytes or a base not 16-byte aligned).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

namespace ws {

constexpr int kResidDays = 64;       // k_residual: days per thread
constexpr int kResidDaysTma = 256;   // k_residual_tma: days per CTA
constexpr int kResidNP = 128;        // k_residual_tma: pixels per CTA
constexpr int kResidNBT = 5;         // bands per thread (both kernels)
#ifndef WS_RESID_CHUNK
#define WS_RESID_CHUNK 2             // days per stage (FP32; FP64 takes half, rounded up)
#endif
#ifndef WS_RESID_STAGES
#define WS_RESID_STAGES 2            // stages in the ring
#endif

// Push z0_u into the band's rings: zr holds z0_{u-d..u}, qb gets q_k for the row
// k = u - d (zero where the row does not exist).
template <typename F, int D>
__device__ __forceinline__ void resid_push(F (&zr)[D + 1], F (&qb)[D + 1], F zu, bool row, F lk) {
#pragma unroll
  for (int n = 0; n < D; ++n) zr[n] = zr[n + 1];
  zr[D] = zu;
#pragma unroll
  for (int n = 0; n < D; ++n) qb[n] = qb[n + 1];
  F q = F(0);
  if (row) {
    F lv[D + 1];
#pragma unroll
    for (int n = 0; n <= D; ++n) lv[n] = zr[n];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int n = 0; n < D - i; ++n) lv[n] = lv[n + 1] - lv[n];
    q = lk * lv[0];
  }
  qb[D] = q;
}

// Residual of day t = u - d after resid_push of day u: zr[0] = z0_t, qb = q_{t-d..t}.
// The data term and D^T q cancel to a few parts in 1e5 of either, so the combination keeps
// what plain rounding would lose: with s + e = x - z0 exactly (two_sum),
//   W (x - z0) - D^T q = fma(w, e, fma(w, s, -D^T q))     (w s - D^T q rounded once),
// and with p + pe = w z0 exactly (two_prod), s + e = x - p,
//   x - W z0 - D^T q   = (s - D^T q) + (e - pe);
// either is within about one rounding of the (small) result.
template <typename F, int D>
__device__ __forceinline__ F resid_emit(const F (&zr)[D + 1], const F (&qb)[D + 1], F xt, F wt, int raw) {
  // (D^T q)_t = sum_n c_n q_{t-n} = (-1)^D * (D-th backward difference of q at t)
  F lv[D + 1];
#pragma unroll
  for (int n = 0; n <= D; ++n) lv[n] = qb[n];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int n = D; n > i; --n) lv[n] = lv[n] - lv[n - 1];
  const F dtq = (D % 2) ? -lv[D] : lv[D];
  if (raw) {
    const DW<F> wz = two_prod(wt, zr[0]);
    const DW<F> se = two_sum(xt, -wz.hi);
    return (se.hi - dtq) + (se.lo - wz.lo);
  }
  // a day without an observation contributes no data term (x may hold anything there)
  const DW<F> se = two_sum(wt > F(0) ? xt : zr[0], -zr[0]);
  return fma(wt, se.lo, fma(wt, se.hi, -dtq));
}

// ---------------------------------------------------------------------------------------
// TMA-staged form.
struct ResidArgs {
  const void* lam;  // scalar lambda (one per pixel) when lam_scalar
  void* r;
  unsigned* err;
  int T, B, P, NS, nbx, lam_scalar, raw;
};

// Shared memory of one stage, in rows of kResidNP elements:
//   Z [C*nbx]  z0 of days u = u0 .. u0+C-1, band-minor
//   X [C*nbx]  x of days t = u - d
//   W [C]      w of days t = u - d
//   L [C]      lambda of rows k = u - d (per-day lambda)
// then NS mbarriers after the last stage.
__host__ __device__ inline size_t resid_stage_rows(int C, int nbx) { return (size_t)C * (2 * nbx + 2); }

template <typename F, int D, int S, int C>
__global__ void __launch_bounds__(kResidNP* S) k_residual_tma(const __grid_constant__ CUtensorMap tm_x,
                                                             const __grid_constant__ CUtensorMap tm_z,
                                                             const __grid_constant__ CUtensorMap tm_w,
                                                             const __grid_constant__ CUtensorMap tm_l,
                                                             const ResidArgs a) {
  constexpr int NBT = kResidNBT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  F* const smem = reinterpret_cast<F*>(smem_raw);
  const int tid = threadIdx.x;
  const int pl = tid % kResidNP, h = tid / kResidNP;
  const int p0 = blockIdx.x * kResidNP, p = p0 + pl;
  const int T = a.T, NS = a.NS, nbx = a.nbx;
  const int t0 = blockIdx.y * kResidDaysTma, t1 = min(T, t0 + kResidDaysTma);
  const int b0 = blockIdx.z * nbx;
  const int us = t0 - D, ue = t1 + D;  // steps u = us .. ue-1
  const int nck = (ue - us + C - 1) / C;
  const size_t srows = resid_stage_rows(C, nbx);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)NS * srows * kResidNP);
  const uint32_t z_bytes = static_cast<uint32_t>(C * nbx * kResidNP * sizeof(F));
  const uint32_t x_bytes = static_cast<uint32_t>((C * nbx + C + (a.lam_scalar ? 0 : C)) * kResidNP * sizeof(F));

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
    prefetch_tmap(&tm_x);
    prefetch_tmap(&tm_z);
    prefetch_tmap(&tm_w);
    if (!a.lam_scalar) prefetch_tmap(&tm_l);
  }
  __syncthreads();

  // Chunk c (steps u0 = us + c C ...) into stage c % NS; thread 0 only. A box that runs
  // past either end of the series reads zeros there; a box with no day inside the series
  // is not loaded (its rows are never used: z0 outside the series is taken as 0, and x,
  // w, lambda are read only on the series' own days).
  auto issue = [&](int c) {
    const int st = c % NS;
    F* Sg = smem + (size_t)st * srows * kResidNP;
    const int u0 = us + c * C, ux = u0 - D;
    const bool lz = u0 < T && u0 + C > 0;
    const bool lx = ux < T && ux + C > 0;
    mbar_arrive_expect_tx(&bar[st], (lz ? z_bytes : 0u) + (lx ? x_bytes : 0u));
    if (lz) tma_load_3d(Sg, &tm_z, &bar[st], p0, b0, u0);
    if (lx) {
      tma_load_3d(Sg + (size_t)C * nbx * kResidNP, &tm_x, &bar[st], p0, b0, ux);
      tma_load_2d(Sg + (size_t)2 * C * nbx * kResidNP, &tm_w, &bar[st], p0, ux);
      if (!a.lam_scalar) tma_load_2d(Sg + (size_t)(2 * C * nbx + C) * kResidNP, &tm_l, &bar[st], p0, ux);
    }
  };
  uint32_t phase = 0u;  // thread 0: bit i = parity of the next completion of stage i
  if (tid == 0)
    for (int c = 0; c < NS && c < nck; ++c) issue(c);

  const bool pv = p < a.P;
  const F ls = (a.lam_scalar && pv) ? static_cast<const F*>(a.lam)[p] : F(0);
  const size_t sP = (size_t)a.P, sBP = (size_t)a.B * a.P;
  // this thread's first band of day 0 (only dereferenced on emitted days and bands)
  F* const rp = static_cast<F*>(a.r) + (size_t)(b0 + h * NBT) * sP + p;
  F zr[NBT][D + 1], qb[NBT][D + 1];
#pragma unroll
  for (int j = 0; j < NBT; ++j)
#pragma unroll
    for (int n = 0; n <= D; ++n) zr[j][n] = qb[j][n] = F(0);

  for (int c = 0; c < nck; ++c) {
    const int st = c % NS;
    bool ok = true;
    if (tid == 0) {
      ok = mbar_wait_bounded(&bar[st], (phase >> st) & 1u);
      if (ok) phase ^= 1u << st;
    }
    if (__syncthreads_or(!ok)) {
      // a wait gave up: flag it, let the copies in flight land (bounded), return
      if (tid == 0) {
        atomicOr(a.err, kDevErrTimeout);
        for (int i = c; i < nck && i < c + NS; ++i)
          (void)mbar_wait_bounded(&bar[i % NS], (phase >> (i % NS)) & 1u);
      }
      return;
    }
    const F* Sg = smem + (size_t)st * srows * kResidNP;
    const F* Sz = Sg + h * NBT * kResidNP + pl;
    const F* Sx = Sz + C * nbx * kResidNP;
    const F* Sw = Sg + (size_t)2 * C * nbx * kResidNP + pl;
    const F* Sl = Sw + (size_t)C * kResidNP;
    const int u0 = us + c * C;
    const int nu = min(C, ue - u0);
#pragma unroll
    for (int i = 0; i < C; ++i) {
      if (i >= nu) break;
      const int u = u0 + i;
      const int t = u - D;  // row k = t, residual day t
      const bool row = t >= 0 && t <= T - D - 1;
      const bool emit = pv && t >= t0 && t < t1;
      const bool zin = u >= 0 && u < T;
      const F lk = a.lam_scalar ? ls : Sl[i * kResidNP];
      const F wt = Sw[i * kResidNP];
      F* const rt = rp + (size_t)t * sBP;
#pragma unroll
      for (int j = 0; j < NBT; ++j) {
        const int bl = h * NBT + j;
        if (bl >= nbx) break;
        const int o = (i * nbx + j) * kResidNP;
        resid_push<F, D>(zr[j], qb[j], zin ? Sz[o] : F(0), row, lk);
        if (emit && b0 + bl < a.B) rt[(size_t)j * sP] = resid_emit<F, D>(zr[j], qb[j], Sx[o], wt, a.raw);
      }
    }
    __syncthreads();
    if (tid == 0 && c + NS < nck) issue(c + NS);
  }
}

// ---------------------------------------------------------------------------------------
// Plain-load form.
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
  F zr[NBR][D + 1];
  F qb[NBR][D + 1];
#pragma unroll
  for (int j = 0; j < NBR; ++j)
#pragma unroll
    for (int n = 0; n <= D; ++n) zr[j][n] = qb[j][n] = F(0);
  // Days are taken in groups of G: every load of a group (z0 and x of each band, w, lambda)
  // is issued before any of them is used, so G days of reads are in flight per thread.
  constexpr int G = 4;
  for (int ug = t0 - D; ug < t1 + D; ug += G) {
    F zl[G][NBR], xl[G][NBR], wl[G], ll[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int u = ug + g;
      const int t = u - D;
      const bool live_u = u < t1 + D;
      const bool row = live_u && t >= 0 && t <= T - D - 1;
      const bool emit = live_u && t >= t0 && t < t1;
      ll[g] = row ? (lam_scalar ? ls : lam[(size_t)t * sP + p]) : F(0);
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
      const int t = u - D;
      const bool row = t >= 0 && t <= T - D - 1;
      const bool emit = t >= t0 && t < t1;
#pragma unroll
      for (int j = 0; j < NBR; ++j) {
        if (j >= nb) break;
        resid_push<F, D>(zr[j], qb[j], zl[g][j], row, ll[g]);
        if (emit) r[(size_t)t * sBP + (size_t)(b0 + j) * sP + p] = resid_emit<F, D>(zr[j], qb[j], xl[g][j], wl[g], raw);
      }
    }
  }
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename F, int D, int S, int C>
static int launch_resid_tma(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0,
                            void* r, int raw, unsigned* err, int nbx, cudaStream_t st) {
  const int es = sizeof(F);
  const int NS = WS_RESID_STAGES;
  const bool per_day = pb.lam_mode == WS_LAM_PER_DAY;
  CUtensorMap maps[4];
  memset(maps, 0, sizeof(maps));
  const uint64_t Pn = (uint64_t)pb.n_series, B = (uint64_t)pb.n_bands, T = (uint64_t)pb.T;
  const uint64_t dx[3] = {Pn, B, T}, sx[2] = {Pn * es, B * Pn * es};
  const uint32_t bx[3] = {(uint32_t)kResidNP, (uint32_t)nbx, (uint32_t)C};
  const uint64_t d2[2] = {Pn, T}, s2[1] = {Pn * es};
  const uint32_t b2[2] = {(uint32_t)kResidNP, (uint32_t)C};
  if (make_tmap(&maps[0], pb.dtype, 3, x, dx, sx, bx) != WS_OK ||
      make_tmap(&maps[1], pb.dtype, 3, z0, dx, sx, bx) != WS_OK ||
      make_tmap(&maps[2], pb.dtype, 2, w, d2, s2, b2) != WS_OK ||
      (per_day && make_tmap(&maps[3], pb.dtype, 2, lam, d2, s2, b2) != WS_OK))
    return WS_EUNSUPPORTED;
  if (!per_day) maps[3] = maps[2];  // unused
  const size_t smem = (size_t)NS * resid_stage_rows(C, nbx) * kResidNP * es + 8 * NS;
  auto kern = k_residual_tma<F, D, S, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  ResidArgs a;
  a.lam = lam;
  a.r = r;
  a.err = err;
  a.T = pb.T;
  a.B = pb.n_bands;
  a.P = (int)pb.n_series;
  a.NS = NS;
  a.nbx = nbx;
  a.lam_scalar = per_day ? 0 : 1;
  a.raw = raw;
  dim3 grid((unsigned)((pb.n_series + kResidNP - 1) / kResidNP), (unsigned)((pb.T + kResidDaysTma - 1) / kResidDaysTma),
            (unsigned)((pb.n_bands + nbx - 1) / nbx));
  kern<<<grid, kResidNP * S, smem, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "residual kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

template <typename F, int D>
static int launch_resid_t(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0,
                          void* r, int raw, unsigned* err, cudaStream_t st) {
  const bool per_day = pb.lam_mode == WS_LAM_PER_DAY;
  const bool tma_ok = ((size_t)pb.n_series * sizeof(F)) % 16 == 0 && aligned16(x) && aligned16(z0) &&
                      aligned16(w) && (!per_day || aligned16(lam));
  if (tma_ok) {
    // bands per CTA: all of them up to 2 x kResidNBT (two threads per pixel above kResidNBT),
    // else groups of 2 x kResidNBT (the last group's box runs past B and reads zeros)
    const int nbx = pb.n_bands < 2 * kResidNBT ? pb.n_bands : 2 * kResidNBT;
    constexpr int C = sizeof(F) == 8 ? (WS_RESID_CHUNK + 1) / 2 : WS_RESID_CHUNK;  // days per stage
    const int rc = nbx > kResidNBT ? launch_resid_tma<F, D, 2, C>(pb, x, w, lam, z0, r, raw, err, nbx, st)
                                   : launch_resid_tma<F, D, 1, C>(pb, x, w, lam, z0, r, raw, err, nbx, st);
    if (rc != WS_EUNSUPPORTED) return rc;
  }
  constexpr int NBR = kResidNBT;
  dim3 grid((unsigned)((pb.n_series + 127) / 128), (unsigned)((pb.T + kResidDays - 1) / kResidDays),
            (unsigned)((pb.n_bands + NBR - 1) / NBR));
  k_residual<F, D, NBR><<<grid, 128, 0, st>>>(static_cast<const F*>(x), static_cast<const F*>(w),
                                              static_cast<const F*>(lam), static_cast<const F*>(z0),
                                              static_cast<F*>(r), pb.T, pb.n_bands, (int)pb.n_series,
                                              pb.lam_mode == WS_LAM_SCALAR, raw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "residual kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int launch_residual(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0, void* r,
                    int raw, unsigned* err, cudaStream_t st) {
  if (pb.dtype == WS_F32) {
    switch (pb.d) {
      case 1: return launch_resid_t<float, 1>(pb, x, w, lam, z0, r, raw, err, st);
      case 2: return launch_resid_t<float, 2>(pb, x, w, lam, z0, r, raw, err, st);
      case 3: return launch_resid_t<float, 3>(pb, x, w, lam, z0, r, raw, err, st);
      case 4: return launch_resid_t<float, 4>(pb, x, w, lam, z0, r, raw, err, st);
    }
  } else {
    switch (pb.d) {
      case 1: return launch_resid_t<double, 1>(pb, x, w, lam, z0, r, raw, err, st);
      case 2: return launch_resid_t<double, 2>(pb, x, w, lam, z0, r, raw, err, st);
      case 3: return launch_resid_t<double, 3>(pb, x, w, lam, z0, r, raw, err, st);
      case 4: return launch_resid_t<double, 4>(pb, x, w, lam, z0, r, raw, err, st);
    }
  }
  return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
}

}  // namespace ws
