// Tile-layout banded-solve kernel, one series per thread, NB right-hand sides.
//
//   MODE_SMOOTH: z = Omega^{-1} W x                       (Eq. 3; Eq. 2 for scalar lambda)
//   MODE_RAW:    out = [out +] Omega^{-1} x               (correction solve of the iterative
//                                                          refinement: x is the residual)
//   MODE_ADJ:    g = Omega^{-1} gz, gx = W g,             (Section 2.3, Eqs. 4-5)
//                glam_k = -sum_b (D g_b)_k (D z_b)_k [* lambda_k]
//
// Data flow per tile of NP pixels (persistent CTAs loop over tiles):
//   pass 1 (forward in time): chunks of C days of the right-hand sides (NB bands),
//     w (C+d days: the rotation of day i needs w_{i+d}) and lambda are staged in shared
//     memory by TMA (cp.async.bulk.tensor, two stages, mbarrier completion). Each thread
//     runs the rotation factor + forward substitution (ws_sweep.cuh) and stores its state
//     at every chunk boundary to a checkpoint area in global memory.
//   pass 2 (backward in time): for each chunk, last to first, the state is reloaded from
//     its checkpoint and the chunk is recomputed from the staged inputs, writing yhat and
//     rho in place; back substitution then runs over the chunk in reverse, writing the
//     output in place over yhat, and TMA stores the output box. The last two chunks of
//     pass 1 are still resident and are reused.
// Inputs are read twice and the output written once, plus d(d+1)+NB*d checkpoint words
// per pixel per chunk, instead of spilling the factor and y for every day.
//
// Shared-memory stage (rows of NP elements):
//   X [C*NB rows]  right-hand sides (pass 2: yhat, then the output)
//   W [C+d rows]   w       (SMOOTH/RAW pass 2: rho_2 over the first C rows)
//   L [C rows]     lambda  (SMOOTH/RAW pass 2: rho_1)
//   E [extra rows] SMOOTH/RAW: rho_3..rho_d ((d-2)*C rows); ADJ: rho_1..rho_d (d*C rows),
//                  keeping w and lambda for the epilogue
// When TMA cannot describe the arrays (row pitch not a multiple of 16 bytes, base not
// 16-byte aligned) every thread copies its own column with LDGSTS instead and stores its
// outputs directly; the arithmetic is the same.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

namespace ws {

template <int MODE, int D>
__host__ __device__ constexpr int extra_rows_per_day() {
  return MODE == MODE_ADJ ? D : (D > 2 ? D - 2 : 0);
}

template <typename F, int D, int NB, int MODE>
__global__ void __launch_bounds__(256) k_tile(const __grid_constant__ CUtensorMap tm_x,
                                              const __grid_constant__ CUtensorMap tm_w,
                                              const __grid_constant__ CUtensorMap tm_l,
                                              const __grid_constant__ CUtensorMap tm_z, const TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  using SW = Sweep<F, D, NB>;
  const int tid = threadIdx.x;
  const int NP = a.NP, C = a.C, T = a.T;
  F* const stage0 = reinterpret_cast<F*>(smem_raw);
  auto stage = [&](int st) -> F* { return stage0 + (size_t)st * a.stage_elems; };
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<F*>(smem_raw) + 2 * a.stage_elems);
  const int rowX = 0, rowW = NB * C, rowL = NB * C + C + D, rowE = rowL + C;
  const uint32_t tx_bytes = static_cast<uint32_t>((NB * C + C + D + (a.lam_scalar ? 0 : C)) * NP * sizeof(F));
  const F* gx_in = static_cast<const F*>(a.x);
  const F* gw = static_cast<const F*>(a.w);
  const F* gl = static_cast<const F*>(a.lam);
  const F* gzin = static_cast<const F*>(a.zin);
  const F* gg0 = static_cast<const F*>(a.g0);
  F* gout = static_cast<F*>(a.out);
  F* gout2 = static_cast<F*>(a.out2);
  F* gf = static_cast<F*>(a.factor);
  const bool want_out = gout != nullptr;

  auto rho_row = [&](int j, int k) -> int {  // j = 1..D
    if (MODE == MODE_ADJ) return rowE + (j - 1) * C + k;
    if (j == 1) return rowL + k;
    if (j == 2) return rowW + k;
    return rowE + (j - 3) * C + k;
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if (a.tma) {
      prefetch_tmap(&tm_x);
      prefetch_tmap(&tm_w);
      if (!a.lam_scalar) prefetch_tmap(&tm_l);
      if (want_out) prefetch_tmap(&tm_z);
    }
  }
  __syncthreads();
  uint32_t phase = 0u;    // bit st: parity of the next completion of stage st
  uint32_t pending = 0u;  // bit st: a load into stage st has not been waited for

  auto issue = [&](int c, int st, int p0) {
    F* S = stage(st);
    if (a.tma) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&bar[st], tx_bytes);
        tma_load_3d(S + rowX * NP, &tm_x, &bar[st], p0, a.b0, c * C);
        tma_load_2d(S + rowW * NP, &tm_w, &bar[st], p0, c * C);
        if (!a.lam_scalar) tma_load_2d(S + rowL * NP, &tm_l, &bar[st], p0, c * C);
      }
    } else {
      const int p = p0 + tid;
      const bool act = p < a.P;
      for (int k = 0; k < C; ++k) {
        const int t = c * C + k;
        const bool v = act && t < T;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          cp_async_elem<sizeof(F)>(S + (rowX + k * NB + b) * NP + tid,
                                   v ? gx_in + ((size_t)t * a.B + a.b0 + b) * a.P + p : gx_in, v);
        if (!a.lam_scalar)
          cp_async_elem<sizeof(F)>(S + (rowL + k) * NP + tid, v ? gl + (size_t)t * a.P + p : gl, v);
      }
      for (int k = 0; k < C + D; ++k) {
        const int t = c * C + k;
        const bool v = act && t < T;
        cp_async_elem<sizeof(F)>(S + (rowW + k) * NP + tid, v ? gw + (size_t)t * a.P + p : gw, v);
      }
      cp_async_commit();
    }
    pending |= 1u << st;
  };

  auto wait_stage = [&](int st, bool newer_pending) -> bool {
    bool ok = true;
    if (a.tma) {
      ok = mbar_wait_bounded(&bar[st], (phase >> st) & 1u);
      if (ok) phase ^= 1u << st;
    } else {
      if (newer_pending)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
    }
    if (ok) pending &= ~(1u << st);
    return ok;
  };

  // A wait gave up: flag it, let this CTA's copies in flight drain (bounded), return.
  auto abort_all = [&]() {
    if (tid == 0) {
      atomicOr(a.err, kDevErrTimeout);
      if (a.tma) {
        for (int st = 0; st < 2; ++st)
          if ((pending >> st) & 1u) (void)mbar_wait_bounded(&bar[st], (phase >> st) & 1u);
        bulk_wait_all();
      }
    }
    if (!a.tma) cp_async_wait<0>();
  };

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int p0 = tile * NP;
    const int p = p0 + tid;
    const bool act = p < a.P;
    F* ck = static_cast<F*>(a.ckpt) + (size_t)blockIdx.x * a.nch * SW::kFields * NP + tid;

    // ---------------- pass 1: forward sweep, checkpoints ----------------
    issue(0, 0, p0);
    if (a.nch > 1) issue(1, 1, p0);
    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    F lam_s = F(0);
    if (a.lam_scalar && act) lam_s = gl[p];
    for (int c = 0; c < a.nch; ++c) {
      const int st = c & 1;
      const bool ok = wait_stage(st, c + 1 < a.nch);
      if (__syncthreads_or(!ok)) {
        abort_all();
        return;
      }
      const F* S = stage(st);
      if (c == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m)
          if (m < T) s.init_weight(m, S[(rowW + m) * NP + tid]);
      }
      s.save(ck + (size_t)c * SW::kFields * NP, NP);
      const int nd = min(C, T - c * C);
      for (int k = 0; k < nd; ++k) {
        const int i = c * C + k;
        const F wi = S[(rowW + k) * NP + tid];
        const F wa = S[(rowW + k + D) * NP + tid];
        const F li = a.lam_scalar ? lam_s : S[(rowL + k) * NP + tid];
        const bool has_row = i < T - D;
        bad |= !(wi >= F(0)) || !finite_(wi);
        npos += wi > F(0);
        if (has_row) bad |= !(li > F(0)) || !finite_(li);
        F bv[NB], rho[D], yh[NB], invD;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const F xv = S[(rowX + k * NB + b) * NP + tid];
          bv[b] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
        }
        s.factor_step(has_row, li, wa, rho, invD);
        s.subst_step(rho, invD, bv, yh);
      }
      __syncthreads();
      if (c + 2 < a.nch) issue(c + 2, st, p0);
    }

    // ---------------- pass 2: backward sweep, chunk recompute ----------------
    const int dmin = D < T ? D : T;
    const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
    const bool okser = code == WS_SERIES_OK;
    // zc: solution of the next D days (back substitution), per band.
    // ADJ: difference triangles of g and z at day t+1, for (D g)_t and (D z)_t taken as
    //      nested first differences (the recursive definition of the order-D forward
    //      difference): on smooth sequences each subtraction is exact (Sterbenz), where
    //      the binomial form would cancel ~3 digits in FP32.
    //      gt[b][j-1] = Delta^j g_{t+1} (j = 1..D-1); zt[b][0] = z_{t+1}, zt[b][j] = Delta^j z_{t+1}.
    constexpr int DT = D > 1 ? D - 1 : 1;
    F zc[NB][D];
    F gt[NB][DT];
    F zt[NB][D];
    F gn[NB];  // ADJ: g_{t+1} (differs from zc[b][0] when accumulating a correction)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        zc[b][j] = F(0);
        zt[b][j] = F(0);
      }
#pragma unroll
      for (int j = 0; j < DT; ++j) gt[b][j] = F(0);
      gn[b] = F(0);
    }
    F glam_sum = F(0);  // ADJ with scalar lambda
    bool nonfin = false;
    for (int c = a.nch - 1; c >= 0; --c) {
      const int st = c & 1;
      if (c < a.nch - 2) {
        const bool ok = wait_stage(st, c >= 1);
        if (__syncthreads_or(!ok)) {
          abort_all();
          return;
        }
      }
      F* S = stage(st);
      s.load(ck + (size_t)c * SW::kFields * NP, NP);
      const int nd = min(C, T - c * C);
      for (int k = 0; k < nd; ++k) {
        const int i = c * C + k;
        const F wi = S[(rowW + k) * NP + tid];
        const F wa = S[(rowW + k + D) * NP + tid];
        const F li = a.lam_scalar ? lam_s : S[(rowL + k) * NP + tid];
        const bool has_row = i < T - D;
        F bv[NB], rho[D], yh[NB], invD;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const F xv = S[(rowX + k * NB + b) * NP + tid];
          bv[b] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
        }
        s.factor_step(has_row, li, wa, rho, invD);
        s.subst_step(rho, invD, bv, yh);
#pragma unroll
        for (int b = 0; b < NB; ++b) S[(rowX + k * NB + b) * NP + tid] = yh[b];
#pragma unroll
        for (int j = 1; j <= D; ++j) S[rho_row(j, k) * NP + tid] = rho[j - 1];
        if (MODE == MODE_SMOOTH && gf != nullptr && a.write_status && act) {
          gf[((size_t)i * (D + 1)) * a.P + p] = okser ? invD : F(0);
#pragma unroll
          for (int j = 1; j <= D; ++j) gf[((size_t)i * (D + 1) + j) * a.P + p] = okser ? rho[j - 1] : F(0);
        }
      }
      for (int k = nd - 1; k >= 0; --k) {
        const int i = c * C + k;
        F rho[D];
#pragma unroll
        for (int j = 1; j <= D; ++j) rho[j - 1] = S[rho_row(j, k) * NP + tid];
        F wk = F(0), lk = F(0);
        if (MODE == MODE_ADJ) {
          wk = S[(rowW + k) * NP + tid];
          lk = a.lam_scalar ? lam_s : S[(rowL + k) * NP + tid];
        }
        F dl = F(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          F acc = S[(rowX + k * NB + b) * NP + tid];
#pragma unroll
          for (int j = 1; j <= D; ++j) acc = fma(-rho[j - 1], zc[b][j - 1], acc);
          nonfin |= !finite_(acc);
          F out = okser ? acc : F(0);
          if (MODE == MODE_ADJ) {
            const size_t gi = ((size_t)i * a.B + a.b0 + b) * a.P + p;
            const F zv = (act && gzin != nullptr) ? gzin[gi] : F(0);
            if (a.accum && act && okser && gg0 != nullptr) out += gg0[gi];   // g = g0 + correction
            F cg = out, cz = zv;                 // level j at day t
            F pg = gn[b], pz = zt[b][0];         // level j-1 at day t+1 (j = 1: the values)
            zt[b][0] = zv;
            gn[b] = out;
#pragma unroll
            for (int j = 1; j <= D; ++j) {
              const F ng = pg - cg, nz = pz - cz;  // Delta^j at day t
              if (j < D) {
                pg = gt[b][j - 1];
                pz = zt[b][j];
                gt[b][j - 1] = ng;
                zt[b][j] = nz;
              }
              cg = ng;
              cz = nz;
            }
            if (i < T - D) dl = fma(cg, cz, dl);
          }
#pragma unroll
          for (int j = D - 1; j > 0; --j) zc[b][j] = zc[b][j - 1];
          zc[b][0] = acc;
          if (MODE == MODE_ADJ) out = wk * out;
          if (MODE == MODE_RAW && a.accum && act && want_out) out += gout[((size_t)i * a.B + a.b0 + b) * a.P + p];
          if (a.tma)
            S[(rowX + k * NB + b) * NP + tid] = out;
          else if (act && want_out)
            gout[((size_t)i * a.B + a.b0 + b) * a.P + p] = out;
        }
        if (MODE == MODE_ADJ && gout2 != nullptr) {
          F gl_t = okser ? -dl : F(0);
          if (a.grad_loglam) gl_t *= lk;
          if (a.lam_scalar) {
            glam_sum += gl_t;
          } else if (act) {
            F* dst = gout2 + (size_t)i * a.P + p;
            *dst = a.b0 == 0 ? gl_t : *dst + gl_t;
          }
        }
      }
      if (a.tma) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          if (want_out) {
            tma_store_3d(&tm_z, S + rowX * NP, p0, a.b0, c * C);
            bulk_commit();
          }
          if (c >= 2) {
            bulk_wait_read_all();
            issue(c - 2, st, p0);
          }
        }
      } else if (c >= 2) {
        issue(c - 2, st, p0);
      }
    }
    if (MODE == MODE_ADJ && gout2 != nullptr && a.lam_scalar && act)
      gout2[p] = a.b0 == 0 ? glam_sum : gout2[p] + glam_sum;
    if (act && a.status != nullptr) {
      if (a.write_status)
        a.status[p] = code != WS_SERIES_OK ? code : (nonfin ? WS_SERIES_NONFINITE : WS_SERIES_OK);
      else if (nonfin && a.status[p] == WS_SERIES_OK)
        a.status[p] = WS_SERIES_NONFINITE;
    }
    if (a.tma && tid == 0) bulk_wait_read_all();
    __syncthreads();
  }
  if (a.tma && tid == 0) bulk_wait_all();
}

template <typename F, int D, int NB, int MODE>
int launch_tile_one(const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  auto kern = k_tile<F, D, NB, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem_bytes);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  kern<<<cfg.grid, cfg.NP, cfg.smem_bytes, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "tile kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

template <typename F, int D, int MODE>
int dispatch_tile_nb(int nb, const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  if (sizeof(F) == 8) {
    if (nb == 2 && D == 2) return launch_tile_one<F, D, 2, MODE>(cfg, a, maps, st);
    if (nb == 1) return launch_tile_one<F, D, 1, MODE>(cfg, a, maps, st);
    return set_error(WS_EUNSUPPORTED, "FP64 band group of %d bands not instantiated", nb);
  }
  switch (nb) {
    case 1: return launch_tile_one<F, D, 1, MODE>(cfg, a, maps, st);
    case 2: return launch_tile_one<F, D, 2, MODE>(cfg, a, maps, st);
    case 4: return launch_tile_one<F, D, 4, MODE>(cfg, a, maps, st);
#ifndef WS_FAST_BUILD
    case 3: return launch_tile_one<F, D, 3, MODE>(cfg, a, maps, st);
    case 5: return launch_tile_one<F, D, 5, MODE>(cfg, a, maps, st);
    case 6: return launch_tile_one<F, D, 6, MODE>(cfg, a, maps, st);
    case 7: return launch_tile_one<F, D, 7, MODE>(cfg, a, maps, st);
    case 8: return launch_tile_one<F, D, 8, MODE>(cfg, a, maps, st);
    case 9: return launch_tile_one<F, D, 9, MODE>(cfg, a, maps, st);
    case 10: return launch_tile_one<F, D, 10, MODE>(cfg, a, maps, st);
#endif
    default: return set_error(WS_EUNSUPPORTED, "band group of %d bands not instantiated", nb);
  }
}

template <int D>
int dispatch_tile_d(const ws_problem& pb, int mode, int nb, const TileCfg& cfg, const TileArgs& a,
                    const CUtensorMap* maps, cudaStream_t st) {
  if (pb.dtype == WS_F32) {
    switch (mode) {
      case MODE_SMOOTH: return dispatch_tile_nb<float, D, MODE_SMOOTH>(nb, cfg, a, maps, st);
      case MODE_RAW: return dispatch_tile_nb<float, D, MODE_RAW>(nb, cfg, a, maps, st);
      case MODE_ADJ: return dispatch_tile_nb<float, D, MODE_ADJ>(nb, cfg, a, maps, st);
    }
  } else {
    switch (mode) {
      case MODE_SMOOTH: return dispatch_tile_nb<double, D, MODE_SMOOTH>(nb, cfg, a, maps, st);
      case MODE_RAW: return dispatch_tile_nb<double, D, MODE_RAW>(nb, cfg, a, maps, st);
      case MODE_ADJ: return dispatch_tile_nb<double, D, MODE_ADJ>(nb, cfg, a, maps, st);
    }
  }
  return set_error(WS_EINVAL, "unknown kernel mode %d", mode);
}

}  // namespace ws
