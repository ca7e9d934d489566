// Tile-layout banded-solve kernel: kNP = 128 pixel series per CTA, one series per
// thread for up to 5 bands; for 6, 8 or 10 bands two threads share a pixel (S = 2),
// each owning NBT = NB / S bands and both running the (cheap, per-pixel) rotation
// factor, which halves the registers per thread and doubles the warps that hide the
// latency of the sequential time recurrence.
//
//   MODE_SMOOTH: z = Omega^{-1} W x                       (Eq. 3; Eq. 2 for scalar lambda)
//   MODE_RAW:    out = [z0 +] Omega^{-1} x                (correction solve of the iterative
//                                                          refinement: x is the residual)
//   MODE_ADJ:    g = [g0 +] Omega^{-1} gz, gx = W g,      (Section 2.3, Eqs. 4-5)
//                glam_k = -sum_b (D g_b)_k (D z_b)_k [* lambda_k]
//                (raw_g: the output is g itself, for the gradient in the weights)
//
// Data flow per tile (persistent CTAs loop over tiles):
//   pass 1 (forward in time): chunks of C days of the right-hand sides, w (C+d days: the
//     rotation of day i needs w_{i+d}) and lambda are staged in shared memory by TMA
//     (cp.async.bulk.tensor, two stages, mbarrier completion). Each thread runs the
//     rotation factor + forward substitution (ws_sweep.cuh) and stores its state at every
//     chunk boundary to a checkpoint area in global memory.
//   pass 2 (backward in time): for each chunk, last to first, the state is reloaded from
//     its checkpoint and the chunk is recomputed from the staged inputs, writing yhat and
//     rho in place; back substitution then runs over the chunk in reverse, writing the
//     output in place over yhat, and TMA stores the output box. The last two chunks of
//     pass 1 are still resident and are reused. RAW/ADJ also need a per-day array in
//     pass 2 (z0 or the forward output z): a single-buffered Z region loaded by TMA at the
//     start of the chunk's recompute and waited for before its back substitution.
// Inputs are read twice and the output written once, plus d(d+1) + B*d checkpoint words
// per pixel per chunk, instead of spilling the factor and y for every day.
//
// Shared memory (rows of kNP elements):
//   stage s (s = 0, 1):
//     X [C*NB rows]  right-hand sides, band-minor (pass 2: yhat, then the output)
//     W [C+d rows]   w       (SMOOTH/RAW with S = 1, pass 2: rho_2 over the first C rows)
//     L [C rows]     lambda  (SMOOTH/RAW with S = 1, pass 2: rho_1)
//     E [extra rows] SMOOTH/RAW with S = 1: rho_3..rho_d ((d-2)*C rows); otherwise
//                    rho_1..rho_d (d*C rows): ADJ keeps w and lambda for its epilogue, and
//                    with S = 2 the other band half still reads them
//   Z [C*NB rows]    RAW/ADJ: z0 or z of the chunk in pass 2
//   G [S*C rows]     ADJ: per-thread partial sums of (D g)(D z) before the band-split combine
//   then 3 mbarriers and kNP status words.
// When TMA cannot describe the arrays (row pitch not a multiple of 16 bytes, base not
// 16-byte aligned) every thread copies its own columns with LDGSTS instead and stores its
// outputs with plain coalesced stores; the arithmetic is the same.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

namespace ws {

template <typename F, int D, int NBT, int S, int MODE>
__global__ void __launch_bounds__(kNP* S, S > 1 ? 2 : 4) k_tile(const __grid_constant__ CUtensorMap tm_x,
                                                 const __grid_constant__ CUtensorMap tm_w,
                                                 const __grid_constant__ CUtensorMap tm_l,
                                                 const __grid_constant__ CUtensorMap tm_o,
                                                 const __grid_constant__ CUtensorMap tm_z, const TileArgs a) {
  constexpr int NB = NBT * S;
  constexpr int EXTRA = MODE == MODE_ADJ || S > 1 ? D : (D > 2 ? D - 2 : 0);
  constexpr bool HAS_Z = MODE == MODE_RAW || MODE == MODE_ADJ;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  using SW = Sweep<F, D, NBT>;
  const int tid = threadIdx.x;
  const int pl = tid % kNP;  // pixel lane within the tile
  const int h = tid / kNP;   // band half (S = 2) or 0
  const int C = a.C, T = a.T;
  constexpr int kFF = SW::kFactorFields;
  constexpr int kFields = kFF + NB * D;
  const size_t stage_rows = (size_t)C * NB + C + D + C + (size_t)EXTRA * C + kFields;
  F* const smem = reinterpret_cast<F*>(smem_raw);
  F* const zbuf = smem + 2 * stage_rows * kNP;                  // Z region
  F* const gbuf = zbuf + (HAS_Z ? (size_t)C * NB * kNP : 0);     // G region
  const size_t rows_total = tile_smem_rows(MODE, C, NB, D, S);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + rows_total * kNP);
  unsigned* nflag = reinterpret_cast<unsigned*>(bar + 4);
  const int rowW = NB * C, rowL = rowW + C + D, rowE = rowL + C, rowK = rowE + EXTRA * C;
  const uint32_t tx_bytes = static_cast<uint32_t>((NB * C + C + D + (a.lam_scalar ? 0 : C)) * kNP * sizeof(F));
  const uint32_t tz_bytes = static_cast<uint32_t>(NB * C * kNP * sizeof(F));
  const uint32_t tk_bytes = static_cast<uint32_t>(kFields * kNP * sizeof(F));
  const F* gx_in = static_cast<const F*>(a.x);
  const F* gw = static_cast<const F*>(a.w);
  const F* gl = static_cast<const F*>(a.lam);
  const F* gzin = static_cast<const F*>(a.zin);
  const F* gg0 = static_cast<const F*>(a.g0);
  F* gout = static_cast<F*>(a.out);
  F* gout2 = static_cast<F*>(a.out2);
  F* gf = static_cast<F*>(a.factor);
  const bool want_out = gout != nullptr;
  const bool want_z = HAS_Z && gzin != nullptr;  // RAW without accumulation reads no Z
  auto stage = [&](int st) -> F* { return smem + (size_t)st * stage_rows * kNP; };
  auto rho_row = [&](int j, int k) -> int {  // j = 1..D
    if (MODE == MODE_ADJ || S > 1) return rowE + (j - 1) * C + k;
    if (j == 1) return rowL + k;
    if (j == 2) return rowW + k;
    return rowE + (j - 3) * C + k;
  };

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
    if (a.tma) {
      prefetch_tmap(&tm_x);
      prefetch_tmap(&tm_w);
      if (!a.lam_scalar) prefetch_tmap(&tm_l);
      if (want_out) prefetch_tmap(&tm_o);
      if (want_z) prefetch_tmap(&tm_z);
    }
  }
  __syncthreads();
  uint32_t phase = 0u;    // bit i: parity of the next completion of barrier i
  uint32_t pending = 0u;  // bit i: a load on barrier i has not been waited for

  // Stage load of chunk c: every thread calls it (TMA: thread 0 issues; LDGSTS: each
  // thread copies its own columns). ckg: the chunk's checkpoint to prefetch (pass 2, TMA).
  auto issue = [&](int c, int st, int p0, const F* ckg) {
    F* Sg = stage(st);
    if (a.tma) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&bar[st], tx_bytes + (ckg != nullptr ? tk_bytes : 0u));
        if (ckg != nullptr) bulk_load_1d(Sg + (size_t)rowK * kNP, ckg, tk_bytes, &bar[st]);
        tma_load_3d(Sg, &tm_x, &bar[st], p0, a.b0, c * C);
        tma_load_2d(Sg + (size_t)rowW * kNP, &tm_w, &bar[st], p0, c * C);
        if (!a.lam_scalar) tma_load_2d(Sg + (size_t)rowL * kNP, &tm_l, &bar[st], p0, c * C);
      }
    } else {
      const int p = p0 + pl;
      const bool act = p < a.P;
      for (int k = 0; k < C; ++k) {
        const int t = c * C + k;
        const bool v = act && t < T;
#pragma unroll
        for (int j = 0; j < NBT; ++j) {
          const int b = h * NBT + j;
          cp_async_elem<sizeof(F)>(Sg + (size_t)(k * NB + b) * kNP + pl,
                                   v ? gx_in + ((size_t)t * a.B + a.b0 + b) * a.P + p : gx_in, v);
        }
        if (h == 0 && !a.lam_scalar)
          cp_async_elem<sizeof(F)>(Sg + (size_t)(rowL + k) * kNP + pl, v ? gl + (size_t)t * a.P + p : gl, v);
      }
      if (h == 0)
        for (int k = 0; k < C + D; ++k) {
          const int t = c * C + k;
          const bool v = act && t < T;
          cp_async_elem<sizeof(F)>(Sg + (size_t)(rowW + k) * kNP + pl, v ? gw + (size_t)t * a.P + p : gw, v);
        }
      cp_async_commit();
    }
    pending |= 1u << st;
  };

  auto issue_z = [&](int c, int p0) {
    if (a.tma) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&bar[2], tz_bytes);
        tma_load_3d(zbuf, &tm_z, &bar[2], p0, a.b0, c * C);
      }
    } else {
      const int p = p0 + pl;
      const bool act = p < a.P;
      for (int k = 0; k < C; ++k) {
        const int t = c * C + k;
        const bool v = act && t < T;
#pragma unroll
        for (int j = 0; j < NBT; ++j) {
          const int b = h * NBT + j;
          cp_async_elem<sizeof(F)>(zbuf + (size_t)(k * NB + b) * kNP + pl,
                                   v ? gzin + ((size_t)t * a.B + a.b0 + b) * a.P + p : gzin, v);
        }
      }
      cp_async_commit();
    }
    pending |= 4u;
  };

  // Wait for barrier i. LDGSTS path: `newer` groups were committed after the awaited one
  // (waiting for the Z group drains every group, which is correct and only costs overlap).
  // TMA path: thread 0 alone polls the barrier (the others wait at the block barrier
  // that always follows, which orders the copied data for them).
  auto wait_bar = [&](int i, int newer) -> bool {
    bool ok = true;
    if (a.tma) {
      if (tid == 0) ok = mbar_wait_bounded(&bar[i], (phase >> i) & 1u);
      if (ok) phase ^= 1u << i;  // thread 0 keeps the parity it gave up on, for abort_all
    } else {
      if (newer >= 1)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
      __syncthreads();
    }
    if (ok) pending &= ~(1u << i);
    return ok;
  };

  // A wait gave up: flag it, let this CTA's copies in flight drain (bounded), return.
  auto abort_all = [&]() {
    if (tid == 0) {
      atomicOr(a.err, kDevErrTimeout);
      if (a.tma) {
        for (int i = 0; i < 3; ++i)
          if ((pending >> i) & 1u) (void)mbar_wait_bounded(&bar[i], (phase >> i) & 1u);
        bulk_wait_all();
      }
    }
    if (!a.tma) cp_async_wait<0>();
  };

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int p0 = tile * kNP;
    const int p = p0 + pl;
    const bool act = p < a.P;
    F* ck = static_cast<F*>(a.ckpt) + (size_t)blockIdx.x * a.nch * kFields * kNP + pl;  // this thread's column

    // ---------------- pass 1: forward sweep, checkpoints ----------------
    issue(0, 0, p0, nullptr);
    if (a.nch > 1) issue(1, 1, p0, nullptr);
    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    F lam_s = F(0);
    if (a.lam_scalar && act) lam_s = gl[p];
    for (int c = 0; c < a.nch; ++c) {
      const int st = c & 1;
      const bool ok = wait_bar(st, c + 1 < a.nch ? 1 : 0);
      if (__syncthreads_or(!ok)) {
        abort_all();
        return;
      }
      const F* Sg = stage(st);
      if (c == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m)
          if (m < T) s.init_weight(m, Sg[(size_t)(rowW + m) * kNP + pl]);
      }
      F* ckc = ck + (size_t)c * kFields * kNP;
      if (h == 0) s.save_factor(ckc, kNP);
      s.save_y(ckc + (size_t)(kFF + h * NBT * D) * kNP, kNP);
      const int nd = min(C, T - c * C);
      const F* Sx = Sg + (size_t)h * NBT * kNP + pl;
      const F* Sw = Sg + (size_t)rowW * kNP + pl;
      const F* Sl = Sg + (size_t)rowL * kNP + pl;
      for (int k = 0; k < nd; ++k, Sx += NB * kNP, Sw += kNP, Sl += kNP) {
        const int i = c * C + k;
        const F wi = Sw[0];
        const F wa = Sw[D * kNP];
        const F li = a.lam_scalar ? lam_s : Sl[0];
        const bool has_row = i < T - D;
        bad |= !(wi >= F(0)) || !finite_(wi);
        npos += wi > F(0);
        if (has_row) bad |= !(li > F(0)) || !finite_(li);
        F bv[NBT], rho[D], yh[NBT], invD;
#pragma unroll
        for (int j = 0; j < NBT; ++j) {
          const F xv = Sx[j * kNP];
          bv[j] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
        }
        s.factor_step(has_row, li, wa, rho, invD);
        s.subst_step(rho, invD, bv, yh);
      }
      if (c + 2 >= a.nch) fence_proxy_async_global();  // checkpoints are read back by bulk copies
      __syncthreads();
      if (c + 2 < a.nch) issue(c + 2, st, p0, nullptr);
    }

    // ---------------- pass 2: backward sweep, chunk recompute ----------------
    const int dmin = D < T ? D : T;
    const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
    const bool okser = code == WS_SERIES_OK;
    // zc: solution of the next D days (back substitution), per own band.
    // ADJ: difference triangles of g and z at day t+1, for (D g)_t and (D z)_t taken as
    //      nested first differences (the recursive definition of the order-D forward
    //      difference): on smooth sequences each subtraction is exact (Sterbenz), where
    //      the binomial form would cancel ~3 digits in FP32.
    //      gt[j][k-1] = Delta^k g_{t+1} (k = 1..D-1); zt[j][0] = z_{t+1}, zt[j][k] = Delta^k z_{t+1};
    //      gn[j] = g_{t+1} (differs from zc when a correction is accumulated onto g0).
    constexpr int DT = D > 1 ? D - 1 : 1;
    F zc[NBT][D];
    F gt[NBT][DT];
    F zt[NBT][D];
    F gn[NBT];
#pragma unroll
    for (int j = 0; j < NBT; ++j) {
#pragma unroll
      for (int q = 0; q < D; ++q) {
        zc[j][q] = F(0);
        zt[j][q] = F(0);
      }
#pragma unroll
      for (int q = 0; q < DT; ++q) gt[j][q] = F(0);
      gn[j] = F(0);
    }
    F glam_sum = F(0);  // ADJ with scalar lambda
    F nanacc = F(0);    // becomes NaN if any output is not finite
    // ADJ with accumulation (refinement correction): largest |correction|, |g| and |D^d g|
    // of this thread's bands, for the settle test of the double-float re-solve
    F dmx = F(0), gmx = F(0), dgmx = F(0);
    for (int c = a.nch - 1; c >= 0; --c) {
      const int st = c & 1;
      if (c < a.nch - 2) {
        const bool ok = wait_bar(st, c >= 1 ? 1 : 0);
        if (__syncthreads_or(!ok)) {
          abort_all();
          return;
        }
      }
      if (want_z) issue_z(c, p0);
      F* Sg = stage(st);
      // the chunk's checkpoint: prefetched into the stage by the bulk copy, except for the
      // two chunks still resident from pass 1 (and on the LDGSTS path)
      const F* ckc = (a.tma && c < a.nch - 2) ? Sg + (size_t)rowK * kNP + pl : ck + (size_t)c * kFields * kNP;
      s.load_factor(ckc, kNP);
      s.load_y(ckc + (size_t)(kFF + h * NBT * D) * kNP, kNP);
      const int nd = min(C, T - c * C);
      {
        F* Sx = Sg + (size_t)h * NBT * kNP + pl;
        const F* Sw = Sg + (size_t)rowW * kNP + pl;
        const F* Sl = Sg + (size_t)rowL * kNP + pl;
        for (int k = 0; k < nd; ++k, Sx += NB * kNP, Sw += kNP, Sl += kNP) {
          const int i = c * C + k;
          const F wi = Sw[0];
          const F wa = Sw[D * kNP];
          const F li = a.lam_scalar ? lam_s : Sl[0];
          const bool has_row = i < T - D;
          F bv[NBT], rho[D], yh[NBT], invD;
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            const F xv = Sx[j * kNP];
            bv[j] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
          }
          s.factor_step(has_row, li, wa, rho, invD);
          s.subst_step(rho, invD, bv, yh);
#pragma unroll
          for (int j = 0; j < NBT; ++j) Sx[j * kNP] = yh[j];
          if (h == 0) {
#pragma unroll
            for (int j = 1; j <= D; ++j) Sg[(size_t)rho_row(j, k) * kNP + pl] = rho[j - 1];
            if (MODE == MODE_SMOOTH && gf != nullptr && a.write_status && act) {
              gf[((size_t)i * (D + 1)) * a.P + p] = okser ? invD : F(0);
#pragma unroll
              for (int j = 1; j <= D; ++j) gf[((size_t)i * (D + 1) + j) * a.P + p] = okser ? rho[j - 1] : F(0);
            }
          }
        }
      }
      if (S > 1) __syncthreads();  // rho rows written by the h = 0 threads; w/lambda reads done
      if (want_z) {
        const bool ok = wait_bar(2, 0);
        if (__syncthreads_or(!ok)) {
          abort_all();
          return;
        }
      }
      {
        F* Sx = Sg + (size_t)((nd - 1) * NB + h * NBT) * kNP + pl;
        const F* Sz = zbuf + (size_t)((nd - 1) * NB + h * NBT) * kNP + pl;
        for (int k = nd - 1; k >= 0; --k, Sx -= NB * kNP, Sz -= NB * kNP) {
          const int i = c * C + k;
          F rho[D];
#pragma unroll
          for (int j = 1; j <= D; ++j) rho[j - 1] = Sg[(size_t)rho_row(j, k) * kNP + pl];
          F wk = F(0);
          if (MODE == MODE_ADJ) wk = Sg[(size_t)(rowW + k) * kNP + pl];
          F dl = F(0);
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            F acc = Sx[j * kNP];
#pragma unroll
            for (int q = 1; q <= D; ++q) acc = fma(-rho[q - 1], zc[j][q - 1], acc);
#pragma unroll
            for (int q = D - 1; q > 0; --q) zc[j][q] = zc[j][q - 1];
            zc[j][0] = acc;
            F out = okser ? acc : F(0);
            if (MODE == MODE_RAW && want_z) out += Sz[j * kNP];  // z0 + correction
            if (MODE == MODE_ADJ) {
              const F zv = Sz[j * kNP];
              if (a.accum && okser && act)  // g = g0 + correction
                out += gg0[((size_t)i * a.B + a.b0 + h * NBT + j) * a.P + p];
              F cg = out, cz = zv;           // level q at day t
              F pg = gn[j], pz = zt[j][0];   // level q-1 at day t+1 (q = 1: the values)
              zt[j][0] = zv;
              gn[j] = out;
              if (a.accum) {
                dmx = fmax(dmx, fabs(acc));
                gmx = fmax(gmx, fabs(out));
              }
#pragma unroll
              for (int q = 1; q <= D; ++q) {
                const F ng = pg - cg, nz = pz - cz;  // Delta^q at day t
                if (q < D) {
                  pg = gt[j][q - 1];
                  pz = zt[j][q];
                  gt[j][q - 1] = ng;
                  zt[j][q] = nz;
                }
                cg = ng;
                cz = nz;
              }
              dl = fma(cg, cz, dl);
              if (a.accum && i < T - D) dgmx = fmax(dgmx, fabs(cg));
              if (!a.raw_g) out = wk * out;
            }
            nanacc = fma(out, F(0), nanacc);
            Sx[j * kNP] = out;
          }
          if (MODE == MODE_ADJ) gbuf[(size_t)(h * C + k) * kNP + pl] = i < T - D ? dl : F(0);
        }
      }
      if (a.tma) fence_proxy_async_smem();
      __syncthreads();
      if (MODE == MODE_ADJ && gout2 != nullptr && h == 0) {
        const F* Sl = Sg + (size_t)rowL * kNP + pl;
        for (int k = 0; k < nd; ++k) {
          F dl = gbuf[(size_t)k * kNP + pl];
#pragma unroll
          for (int q = 1; q < S; ++q) dl += gbuf[(size_t)(q * C + k) * kNP + pl];
          F gl_t = okser ? -dl : F(0);
          if (a.grad_loglam) gl_t *= a.lam_scalar ? lam_s : Sl[(size_t)k * kNP];
          if (a.lam_scalar) {
            glam_sum += gl_t;
          } else if (act) {
            F* dst = gout2 + (size_t)(c * C + k) * a.P + p;
            *dst = a.b0 == 0 ? gl_t : *dst + gl_t;
          }
        }
      }
      if (!a.tma && want_out && act)
        for (int k = 0; k < nd; ++k)
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            const int b = h * NBT + j;
            gout[((size_t)(c * C + k) * a.B + a.b0 + b) * a.P + p] = Sg[(size_t)(k * NB + b) * kNP + pl];
          }
      if (MODE == MODE_ADJ || !a.tma) __syncthreads();  // stage reads done before it is refilled
      if (a.tma) {
        if (tid == 0) {
          if (want_out) {
            tma_store_3d(&tm_o, Sg, p0, a.b0, c * C);
            bulk_commit();
          }
          if (c >= 2) {
            bulk_wait_read_all();
            issue(c - 2, st, p0, static_cast<const F*>(a.ckpt) + ((size_t)blockIdx.x * a.nch + (c - 2)) * kFields * kNP);
          }
        }
      } else if (c >= 2) {
        issue(c - 2, st, p0, nullptr);
      }
    }
    // per-series status; the band halves combine their non-finite flags
    bool nonfin = !(nanacc == F(0));
    // settle test of the refined adjoint: the error left after the step, |delta|^2 / |g|
    // (the step squares a contracting relative error) plus g's own rounding, differenced
    // d times (at most 2^d), against 1e-4 of |D^d g|
    bool unsettled = false;
    if (MODE == MODE_ADJ && a.df_list != nullptr && gmx > F(0)) {
      const F e1 = dmx * (dmx / gmx) + F(1.2e-7) * gmx;
      unsettled = F(1 << D) * e1 > F(1e-4) * dgmx;
    }
    if (S > 1) {
      if (h == 1) nflag[pl] = (nonfin ? 1u : 0u) | (unsettled ? 2u : 0u);
      __syncthreads();
      if (h == 0) {
        nonfin = nonfin || (nflag[pl] & 1u) != 0u;
        unsettled = unsettled || (nflag[pl] & 2u) != 0u;
      }
    }
    if (MODE == MODE_ADJ && unsettled && okser && act && h == 0 && atomicExch(a.df_mark + p, 1u) == 0u)
      a.df_list[atomicAdd(a.df_count, 1u)] = p;
    if (MODE == MODE_ADJ && gout2 != nullptr && a.lam_scalar && act && h == 0)
      gout2[p] = a.b0 == 0 ? glam_sum : gout2[p] + glam_sum;
    if (act && a.status != nullptr && h == 0) {
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

template <typename F, int D, int NBT, int S, int MODE>
int launch_tile_one(const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  auto kern = k_tile<F, D, NBT, S, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem_bytes);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  kern<<<cfg.grid, kNP * S, cfg.smem_bytes, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "tile kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

template <typename F, int D, int MODE>
int dispatch_tile_nb(int nb, const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  if (sizeof(F) == 8) {
    if (nb == 2 && D == 2) return launch_tile_one<F, D, 2, 1, MODE>(cfg, a, maps, st);
    if (nb == 1) return launch_tile_one<F, D, 1, 1, MODE>(cfg, a, maps, st);
    return set_error(WS_EUNSUPPORTED, "FP64 band group of %d bands not instantiated", nb);
  }
  switch (nb) {
    case 1: return launch_tile_one<F, D, 1, 1, MODE>(cfg, a, maps, st);
    case 2: return launch_tile_one<F, D, 2, 1, MODE>(cfg, a, maps, st);
    case 4: return launch_tile_one<F, D, 4, 1, MODE>(cfg, a, maps, st);
#ifndef WS_FAST_BUILD
    case 3: return launch_tile_one<F, D, 3, 1, MODE>(cfg, a, maps, st);
    case 5: return launch_tile_one<F, D, 5, 1, MODE>(cfg, a, maps, st);
    case 6: return launch_tile_one<F, D, 3, 2, MODE>(cfg, a, maps, st);
    case 7: return launch_tile_one<F, D, 7, 1, MODE>(cfg, a, maps, st);
    case 8: return launch_tile_one<F, D, 4, 2, MODE>(cfg, a, maps, st);
    case 9: return launch_tile_one<F, D, 9, 1, MODE>(cfg, a, maps, st);
    case 10: return launch_tile_one<F, D, 5, 2, MODE>(cfg, a, maps, st);
#endif
    default: return set_error(WS_EUNSUPPORTED, "band group of %d bands not instantiated", nb);
  }
}

template <typename F, int D, int MODE>
const void* kernel_ptr_nb(int nb) {
  if (sizeof(F) == 8) {
    if (nb == 2 && D == 2) return (const void*)k_tile<F, D, 2, 1, MODE>;
    if (nb == 1) return (const void*)k_tile<F, D, 1, 1, MODE>;
    return nullptr;
  }
  switch (nb) {
    case 1: return (const void*)k_tile<F, D, 1, 1, MODE>;
    case 2: return (const void*)k_tile<F, D, 2, 1, MODE>;
    case 4: return (const void*)k_tile<F, D, 4, 1, MODE>;
#ifndef WS_FAST_BUILD
    case 3: return (const void*)k_tile<F, D, 3, 1, MODE>;
    case 5: return (const void*)k_tile<F, D, 5, 1, MODE>;
    case 6: return (const void*)k_tile<F, D, 3, 2, MODE>;
    case 7: return (const void*)k_tile<F, D, 7, 1, MODE>;
    case 8: return (const void*)k_tile<F, D, 4, 2, MODE>;
    case 9: return (const void*)k_tile<F, D, 9, 1, MODE>;
    case 10: return (const void*)k_tile<F, D, 5, 2, MODE>;
#endif
  }
  return nullptr;
}

template <int D>
const void* tile_kernel_ptr_t(const ws_problem& pb, int mode, int nb) {
  if (pb.dtype == WS_F32) {
    switch (mode) {
      case MODE_SMOOTH: return kernel_ptr_nb<float, D, MODE_SMOOTH>(nb);
      case MODE_RAW: return kernel_ptr_nb<float, D, MODE_RAW>(nb);
      case MODE_ADJ: return kernel_ptr_nb<float, D, MODE_ADJ>(nb);
    }
  } else {
    switch (mode) {
      case MODE_SMOOTH: return kernel_ptr_nb<double, D, MODE_SMOOTH>(nb);
      case MODE_RAW: return kernel_ptr_nb<double, D, MODE_RAW>(nb);
      case MODE_ADJ: return kernel_ptr_nb<double, D, MODE_ADJ>(nb);
    }
  }
  return nullptr;
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
