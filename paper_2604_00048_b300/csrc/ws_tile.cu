// Tile-layout smoothing kernel: z = (W + D^T Lambda D)^{-1} W x (Eq. 3) for NP pixel
// series per CTA, one series per thread, B bands as right-hand sides.
//
// Data flow per tile of NP pixels (persistent CTAs loop over tiles):
//   pass 1 (forward in time): chunks of C days of x (NB bands), w (C+d days, the
//     rotation of day i needs w_{i+d}) and lambda are staged in shared memory by TMA
//     (cp.async.bulk.tensor, two stages, mbarrier completion). Each thread runs the
//     rotation factor + forward substitution (ws_sweep.cuh) and stores its state at
//     every chunk boundary to a checkpoint area in global memory.
//   pass 2 (backward in time): for each chunk, last to first, the state is reloaded
//     from its checkpoint and the chunk is recomputed from the staged inputs,
//     writing yhat and rho in place over x, w and lambda; back substitution then
//     runs over the chunk in reverse, writing z in place over yhat, and TMA stores
//     the z box. The last two chunks of pass 1 are still resident and are reused.
// Inputs are read twice and z written once (plus d(d+1)+B*d checkpoint words per
// pixel per chunk), instead of spilling the factor and y for every day.
//
// Shared-memory stage (rows of NP elements):
//   X [C*NB rows]  x[t][b] (pass 2: yhat, then z)
//   W [C+d rows]   w       (pass 2: rho_2 over the first C rows)
//   L [C rows]     lambda  (pass 2: rho_1)
//   E [(d-2)*C]    pass 2: rho_3..rho_d (d > 2)
// When TMA cannot describe the arrays (row pitch not a multiple of 16 bytes, base
// not 16-byte aligned) every thread copies its own column with LDGSTS instead and
// stores z directly; the arithmetic is the same.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

namespace ws {

template <typename F, int D, int NB>
__global__ void __launch_bounds__(256) k_smooth_tile(const __grid_constant__ CUtensorMap tm_x,
                                                     const __grid_constant__ CUtensorMap tm_w,
                                                     const __grid_constant__ CUtensorMap tm_l,
                                                     const __grid_constant__ CUtensorMap tm_z,
                                                     const TileArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  using SW = Sweep<F, D, NB>;
  const int tid = threadIdx.x;
  const int NP = a.NP, C = a.C, T = a.T;
  F* const stage0 = reinterpret_cast<F*>(smem_raw);
  auto stage = [&](int st) -> F* { return stage0 + (size_t)st * a.stage_elems; };
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<F*>(smem_raw) + 2 * a.stage_elems);
  const int rowX = 0, rowW = NB * C, rowL = NB * C + C + D, rowE = rowL + C;
  const uint32_t tx_bytes = static_cast<uint32_t>((NB * C + C + D + (a.lam_scalar ? 0 : C)) * NP * sizeof(F));
  const F* gx = static_cast<const F*>(a.x);
  const F* gw = static_cast<const F*>(a.w);
  const F* gl = static_cast<const F*>(a.lam);
  F* gz = static_cast<F*>(a.out);
  F* gf = static_cast<F*>(a.factor);

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if (a.tma) {
      prefetch_tmap(&tm_x);
      prefetch_tmap(&tm_w);
      if (!a.lam_scalar) prefetch_tmap(&tm_l);
      prefetch_tmap(&tm_z);
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
                                   v ? gx + ((size_t)t * a.B + a.b0 + b) * a.P + p : gx, v);
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
          bv[b] = wi > F(0) ? wi * xv : F(0);
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
    F zc[NB][D];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int j = 0; j < D; ++j) zc[b][j] = F(0);
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
          bv[b] = wi > F(0) ? wi * xv : F(0);
        }
        s.factor_step(has_row, li, wa, rho, invD);
        s.subst_step(rho, invD, bv, yh);
#pragma unroll
        for (int b = 0; b < NB; ++b) S[(rowX + k * NB + b) * NP + tid] = yh[b];
        S[(rowL + k) * NP + tid] = rho[0];
        if (D >= 2) S[(rowW + k) * NP + tid] = rho[D >= 2 ? 1 : 0];
#pragma unroll
        for (int j = 3; j <= D; ++j) S[(rowE + (j - 3) * C + k) * NP + tid] = rho[j - 1];
        if (gf != nullptr && a.write_status && act) {
          const bool ok = code == WS_SERIES_OK;
          gf[((size_t)i * (D + 1)) * a.P + p] = ok ? invD : F(0);
#pragma unroll
          for (int j = 1; j <= D; ++j) gf[((size_t)i * (D + 1) + j) * a.P + p] = ok ? rho[j - 1] : F(0);
        }
      }
      for (int k = nd - 1; k >= 0; --k) {
        const int i = c * C + k;
        F rho[D];
        rho[0] = S[(rowL + k) * NP + tid];
        if (D >= 2) rho[D >= 2 ? 1 : 0] = S[(rowW + k) * NP + tid];
#pragma unroll
        for (int j = 3; j <= D; ++j) rho[j - 1] = S[(rowE + (j - 3) * C + k) * NP + tid];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          F acc = S[(rowX + k * NB + b) * NP + tid];
#pragma unroll
          for (int j = 1; j <= D; ++j) acc = fma(-rho[j - 1], zc[b][j - 1], acc);
#pragma unroll
          for (int j = D - 1; j > 0; --j) zc[b][j] = zc[b][j - 1];
          zc[b][0] = acc;
          nonfin |= !finite_(acc);
          const F out = code == WS_SERIES_OK ? acc : F(0);
          if (a.tma)
            S[(rowX + k * NB + b) * NP + tid] = out;
          else if (act)
            gz[((size_t)i * a.B + a.b0 + b) * a.P + p] = out;
        }
      }
      if (a.tma) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
          tma_store_3d(&tm_z, S + rowX * NP, p0, a.b0, c * C);
          bulk_commit();
          if (c >= 2) {
            bulk_wait_read_all();
            issue(c - 2, st, p0);
          }
        }
      } else if (c >= 2) {
        issue(c - 2, st, p0);
      }
    }
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

// ----------------------------------------------------------------------------------
// host side

int g_tune_np = 0, g_tune_chunk = 0;

int plan_tile(const ws_problem& pb, int nb, int D, int extra_planes, TileCfg& cfg) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  const int es = pb.dtype == WS_F64 ? 8 : 4;
  cfg.NP = g_tune_np > 0 ? g_tune_np : 128;
  cfg.stages = 2;
  const int T = pb.T;
  // rows per stage = C * (nb + 2 + extra_planes) + D; two stages in the opt-in shared memory
  const long budget = (long)di.smem_optin - 1024;
  const long rows_max = budget / (2L * cfg.NP * es);
  long C = (rows_max - D) / (nb + 2 + extra_planes);
  if (C > 256 - D) C = 256 - D;
  if (g_tune_chunk > 0 && g_tune_chunk < C) C = g_tune_chunk;
  if (C > T) C = T > 0 ? T : 1;
  if (C < 1) C = 1;
  cfg.C = (int)C;
  cfg.nch = T > 0 ? (T + cfg.C - 1) / cfg.C : 0;
  cfg.n_tiles = (int)((pb.n_series + cfg.NP - 1) / cfg.NP);
  const size_t rows = (size_t)cfg.C * (nb + 2 + extra_planes) + D;
  cfg.stage_elems = rows * cfg.NP;
  cfg.smem_bytes = 2 * cfg.stage_elems * es + 64;
  int per_sm = (int)((long)(di.smem_optin + 1024) / (long)(cfg.smem_bytes + 1024));
  if (per_sm < 1) per_sm = 1;
  const long cap = (long)di.sm_count * per_sm;
  cfg.grid = (int)(cfg.n_tiles < cap ? cfg.n_tiles : cap);
  cfg.fields = D * (D + 1) + nb * D;
  return WS_OK;
}

template <typename F, int D, int NB>
static int launch_one(const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  auto kern = k_smooth_tile<F, D, NB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem_bytes);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  kern<<<cfg.grid, cfg.NP, cfg.smem_bytes, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "smooth kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

template <typename F, int D>
static int dispatch_nb(int nb, const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps,
                       cudaStream_t st) {
  switch (nb) {
    case 1: return launch_one<F, D, 1>(cfg, a, maps, st);
    case 2: return launch_one<F, D, 2>(cfg, a, maps, st);
    case 4: return launch_one<F, D, 4>(cfg, a, maps, st);
#ifndef WS_FAST_BUILD
    case 3: return launch_one<F, D, 3>(cfg, a, maps, st);
    case 5: return launch_one<F, D, 5>(cfg, a, maps, st);
    case 6: return launch_one<F, D, 6>(cfg, a, maps, st);
    case 7: return launch_one<F, D, 7>(cfg, a, maps, st);
    case 8: return launch_one<F, D, 8>(cfg, a, maps, st);
    case 9: return launch_one<F, D, 9>(cfg, a, maps, st);
    case 10: return launch_one<F, D, 10>(cfg, a, maps, st);
#endif
    default: return set_error(WS_EUNSUPPORTED, "band group of %d bands not instantiated", nb);
  }
}

int launch_smooth_tile(const ws_problem& pb, int nb, const TileCfg& cfg, const TileArgs& a,
                       const CUtensorMap* maps, cudaStream_t st) {
  if (pb.dtype == WS_F32) {
    switch (pb.d) {
      case 1: return dispatch_nb<float, 1>(nb, cfg, a, maps, st);
      case 2: return dispatch_nb<float, 2>(nb, cfg, a, maps, st);
      case 3: return dispatch_nb<float, 3>(nb, cfg, a, maps, st);
      case 4: return dispatch_nb<float, 4>(nb, cfg, a, maps, st);
    }
  } else {
    switch (pb.d) {
      case 1: return launch_one<double, 1, 1>(cfg, a, maps, st);
      case 2: return nb == 2 ? launch_one<double, 2, 2>(cfg, a, maps, st) : launch_one<double, 2, 1>(cfg, a, maps, st);
      case 3: return launch_one<double, 3, 1>(cfg, a, maps, st);
      case 4: return launch_one<double, 4, 1>(cfg, a, maps, st);
    }
  }
  return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
}

}  // namespace ws
