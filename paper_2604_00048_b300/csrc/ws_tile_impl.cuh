// Tile-layout banded-solve kernel: NP (128 or 64) pixel series per CTA, one series per
// thread for up to 5 bands; for 6, 8 or 10 bands two threads share a pixel (S = 2),
// each owning NBT = NB / S bands and both running the (cheap, per-pixel) rotation
// factor, which halves the registers per thread and doubles the warps that hide the
// latency of the sequential time recurrence. 64-pixel CTAs give each pixel twice the
// shared memory of 128-pixel ones at the same CTAs per SM: chunks twice as deep, half the
// checkpoint traffic.
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
//     rotation factor + forward substitution (ws_sweep.cuh) and stores its state at the
//     start of every group of G chunks (G = 2 by default) to a checkpoint area in global
//     memory.
//   pass 2 (backward in time): group by group, last to first, the state is reloaded from
//     the group's checkpoint (loaded into registers one group ahead) and the group's chunks,
//     both resident in the two stages, are recomputed from the staged inputs, writing yhat
//     and rho in place; back substitution then runs over each chunk in reverse, writing the
//     output in place over yhat, and TMA stores the output box. The last two chunks of pass
//     1 are still resident and are reused. RAW with accumulation and ADJ also need a per-day
//     array in pass 2 (z0 or the forward output z): it is staged with the chunk's inputs (the
//     two chunks resident from pass 1 get theirs when pass 1 ends).
// Inputs are read twice and the output written once, plus d(d+1) + B*d checkpoint words
// per pixel per group of chunks, instead of spilling the factor and y for every day.
//
// Shared memory (rows of NP elements):
//   stage s (s = 0, 1):
//     X [C*NB rows]  right-hand sides, band-minor (pass 2: yhat, then the output)
//     Z [C*NB rows]  RAW/ADJ: z0 or z of the chunk in pass 2
//     W [C+d rows]   w       (SMOOTH/RAW with S = 1, pass 2: rho_2 over the first C rows)
//     L [C rows]     lambda  (SMOOTH/RAW with S = 1, pass 2: rho_1)
//     E [extra rows] SMOOTH/RAW with S = 1: rho_3..rho_d ((d-2)*C rows); otherwise
//                    rho_1..rho_d (d*C rows): ADJ keeps w and lambda for its epilogue, and
//                    with S = 2 the other band half still reads them
//   G [S*C rows]     ADJ: per-thread partial sums of (D g)(D z) before the band-split combine
//   then 3 mbarriers and NP status words.
// When TMA cannot describe the arrays (row pitch not a multiple of 16 bytes, base not
// 16-byte aligned) every thread copies its own columns with LDGSTS instead and stores its
// outputs with plain coalesced stores; the arithmetic is the same.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <limits>
#include <type_traits>

#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

// Unroll factor of the per-day loops (the rotating per-day state then needs no copies
// between iterations).
#ifndef WS_TILE_UNROLL
#define WS_TILE_UNROLL 2
#endif
#define WS_PRAGMA_(x) _Pragma(#x)
#define WS_UNROLL_N(n) WS_PRAGMA_(unroll n)

namespace ws {

template <typename F, int D, int NBT, int S, int MODE, int NP>
__global__ void __launch_bounds__(NP* S, (S > 1 ? 2 : 4) * (128 / NP))
    k_tile(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_w,
           const __grid_constant__ CUtensorMap tm_l, const __grid_constant__ CUtensorMap tm_o,
           const __grid_constant__ CUtensorMap tm_z, const __grid_constant__ CUtensorMap tm_m,
           const TileArgs a) {
  constexpr int NB = NBT * S;
  constexpr int EXTRA = MODE == MODE_ADJ || S > 1 ? D : (D > 2 ? D - 2 : 0);
  constexpr bool HAS_Z = MODE == MODE_RAW || MODE == MODE_ADJ;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  using SW = Sweep<F, D, NBT>;
  const int tid = threadIdx.x;
  const int pl = tid % NP;  // pixel lane within the tile
  const int h = tid / NP;   // band half (S = 2) or 0
  const int C = a.C, T = a.T;
  constexpr int kFF = SW::kFactorFields;
  constexpr int kFields = kFF + NB * D;
  constexpr int kYT = NBT * D;  // this thread's forward-substitution words in a checkpoint
  constexpr F kFMax = std::numeric_limits<F>::max();
  // ADJ with the masked-MSE loss fused in: x is the target, the right-hand side
  // gz = scale * m_t * (z - target) is formed per day from the staged z, target and m
  const bool mse = MODE == MODE_ADJ && a.mse;
  const bool has_m = mse && a.mask != nullptr;
  const F mscale = static_cast<F>(a.mse_scale);
  const int stage_rows = (int)tile_stage_rows(MODE, C, NB, D, S, mse ? 1 : 0);
  F* const smem = reinterpret_cast<F*>(smem_raw);
  F* const gbuf = smem + 2 * stage_rows * NP;  // G region (ADJ)
  const size_t rows_total = tile_smem_rows(MODE, C, NB, D, S, mse ? 1 : 0);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + rows_total * NP);
  unsigned* nflag = reinterpret_cast<unsigned*>(bar + 4);
  const int rowZ = NB * C;                                   // HAS_Z: pass 2's z / z0 of the chunk
  const int rowW = NB * C * (HAS_Z ? 2 : 1), rowL = rowW + C + D, rowE = rowL + C;
  const int rowM = rowE + EXTRA * C;  // ADJ with the MSE loss: day weights m of the chunk
  const uint32_t tx_bytes = static_cast<uint32_t>((NB * C + C + D + (a.lam_scalar ? 0 : C)) * NP * sizeof(F));
  const uint32_t tz_bytes = static_cast<uint32_t>(NB * C * NP * sizeof(F));
  const uint32_t tm_bytes = static_cast<uint32_t>(has_m ? C * NP * sizeof(F) : 0);
  const F* gm = static_cast<const F*>(a.mask);
  const F* gx_in = static_cast<const F*>(a.x);
  const F* gw = static_cast<const F*>(a.w);
  const F* gl = static_cast<const F*>(a.lam);
  const F* gzin = static_cast<const F*>(a.zin);
  const F* gg0 = static_cast<const F*>(a.g0);
  F* gout = static_cast<F*>(a.out);
  F* gout2 = static_cast<F*>(a.out2);
  F* gf = static_cast<F*>(a.factor);
  const bool want_out = gout != nullptr;
  const bool want_z = HAS_Z && gzin != nullptr;  // RAW without accumulation reads no z
  auto stage = [&](int st) -> F* { return smem + st * stage_rows * NP; };
  // chunks per checkpoint (1 or 2) and the ring stage of chunk q in pass 2. Pass 1 puts
  // chunk q in stage q & 1. With G = 2, pass 2 handles chunks in groups {2m, 2m + 1}; the
  // next group's earlier chunk goes into the stage freed first (the later chunk's, back-
  // substituted first), so the roles of the two stages alternate from group to group,
  // counted from the last complete group (a last chunk alone keeps stage 0).
  const int G = a.ck_group == 2 ? 2 : 1;
  auto pstage = [&](int q) -> int {
    if (G == 1) return q & 1;
    if ((a.nch & 1) && q == a.nch - 1) return 0;
    const int mlf = ((a.nch - 1) >> 1) - (a.nch & 1);
    const int es = (mlf - (q >> 1)) & 1;
    return (q & 1) ? es ^ 1 : es;
  };
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
      if (has_m) prefetch_tmap(&tm_m);
    }
  }
  __syncthreads();
  uint32_t phase = 0u;    // bit i: parity of the next completion of barrier i
  uint32_t pending = 0u;  // bit i: a load on barrier i has not been waited for

  // z of chunk c (pass 2) into stage st: TMA on barrier `b`, or LDGSTS (own columns).
  auto copy_z = [&](int c, int st, int p0, uint64_t* b) {
    F* Sz = stage(st) + rowZ * NP;
    if (a.tma) {
      if (tid == 0) tma_load_3d(Sz, &tm_z, b, p0, a.b0, c * C);
    } else {
      const int p = p0 + pl;
      const bool act = p < a.P;
      for (int k = 0; k < C; ++k) {
        const int t = c * C + k;
        const bool v = act && t < T;
#pragma unroll
        for (int j = 0; j < NBT; ++j) {
          const int b2 = h * NBT + j;
          cp_async_elem<sizeof(F)>(Sz + (k * NB + b2) * NP + pl,
                                   v ? gzin + ((size_t)t * a.B + a.b0 + b2) * a.P + p : gzin, v);
        }
      }
    }
  };

  // Stage load of chunk c: every thread calls it (TMA: thread 0 issues; LDGSTS: each
  // thread copies its own columns). with_z: pass 2 of RAW/ADJ also stages z of the chunk.
  auto issue = [&](int c, int st, int p0, bool with_z) {
    F* Sg = stage(st);
    if (a.tma) {
      if (tid == 0) {
        mbar_arrive_expect_tx(&bar[st], tx_bytes + (with_z ? tz_bytes : 0u) + tm_bytes);
        tma_load_3d(Sg, &tm_x, &bar[st], p0, a.b0, c * C);
        tma_load_2d(Sg + rowW * NP, &tm_w, &bar[st], p0, c * C);
        if (!a.lam_scalar) tma_load_2d(Sg + rowL * NP, &tm_l, &bar[st], p0, c * C);
        if (with_z) copy_z(c, st, p0, &bar[st]);
        if (has_m) tma_load_2d(Sg + rowM * NP, &tm_m, &bar[st], p0, c * C);
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
          cp_async_elem<sizeof(F)>(Sg + (k * NB + b) * NP + pl,
                                   v ? gx_in + ((size_t)t * a.B + a.b0 + b) * a.P + p : gx_in, v);
        }
        if (h == 0 && !a.lam_scalar)
          cp_async_elem<sizeof(F)>(Sg + (size_t)(rowL + k) * NP + pl, v ? gl + (size_t)t * a.P + p : gl, v);
        if (h == 0 && has_m)
          cp_async_elem<sizeof(F)>(Sg + (size_t)(rowM + k) * NP + pl, v ? gm + (size_t)t * a.P + p : gm, v);
      }
      if (h == 0)
        for (int k = 0; k < C + D; ++k) {
          const int t = c * C + k;
          const bool v = act && t < T;
          cp_async_elem<sizeof(F)>(Sg + (size_t)(rowW + k) * NP + pl, v ? gw + (size_t)t * a.P + p : gw, v);
        }
      if (with_z) copy_z(c, st, p0, nullptr);
      cp_async_commit();
    }
    pending |= 1u << st;
  };

  // Wait for barrier i. LDGSTS path: `newer` groups were committed after the awaited one.
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
    const int p0 = tile * NP;
    const int p = p0 + pl;
    const bool act = p < a.P;
    // checkpoints: field f of checkpoint j (chunk j * G) of this CTA's tile at ck[(j * kFields + f) * NP]
    F* ck = static_cast<F*>(a.ckpt) + (size_t)blockIdx.x * a.nch * kFields * NP + pl;

    // ---------------- pass 1: forward sweep, checkpoints ----------------
    issue(0, 0, p0, mse);
    if (a.nch > 1) issue(1, 1, p0, mse);
    SW s;
    s.reset();
    int npos = 0;
    bool bad = false;
    F lam_s = F(0);
    if (a.lam_scalar && act) lam_s = gl[p];
    F lsum = F(0);  // MSE loss: sum of m (z - target)^2 over this thread's bands
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
          if (m < T) s.init_weight(m, Sg[(rowW + m) * NP + pl]);
      }
      if (G == 1 || (c & 1) == 0) {  // the checkpoint of chunk c (groups of G chunks)
        F* ckc = ck + (size_t)(c >> (G - 1)) * kFields * NP;
        if (h == 0) s.save_factor(ckc, NP);
        s.save_y(ckc + (size_t)(kFF + h * kYT) * NP, NP);
      }
      const int nd = min(C, T - c * C);
      const F* Sx = Sg + h * NBT * NP + pl;
      const F* Sw = Sg + rowW * NP + pl;
      const F* Sl = Sg + rowL * NP + pl;
      // the day loop; MSE (ADJ with the loss fused in) is a compile-time branch
      auto p1days = [&](auto mse_tag) {
        constexpr bool MSE = MODE == MODE_ADJ && decltype(mse_tag)::value;
WS_UNROLL_N(WS_TILE_UNROLL)
        for (int k = 0; k < nd; ++k, Sx += NB * NP, Sw += NP, Sl += NP) {
          const int i = c * C + k;
          const F wi = Sw[0];
          const F wa = Sw[D * NP];
          const F li = a.lam_scalar ? lam_s : Sl[0];
          const bool has_row = i < T - D;
          bad |= !(wi >= F(0) && wi <= kFMax);  // negative, NaN or infinite
          npos += wi > F(0);
          if (has_row) bad |= !(li > F(0) && li <= kFMax);
          F bv[NBT], rho[D], yh[NBT], invD;
          const F mk = MSE && has_m ? Sg[(rowM + k) * NP + pl] : F(1);
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            const F xv = Sx[j * NP];
            bv[j] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
            if (MSE) {  // gz = scale m (z - target); masked days are inert whatever the target
              const F e = mk > F(0) ? Sx[rowZ * NP + j * NP] - xv : F(0);
              bv[j] = mscale * mk * e;
              lsum = fma(mk * e, e, lsum);
            }
          }
          s.factor_step(has_row, li, wa, rho, invD);
          s.subst_step(rho, invD, bv, yh);
        }
      };
      if (mse)
        p1days(std::true_type{});
      else
        p1days(std::false_type{});
      __syncthreads();
      if (c + 2 < a.nch) issue(c + 2, st, p0, mse);
    }

    // The last two chunks of pass 1 stay resident for pass 2: stage their z now (one
    // barrier for both), waited for before the first back substitution.
    if (want_z && !mse) {  // (with the MSE loss pass 1 staged z already)
      if (a.tma) {
        if (tid == 0) {
          mbar_arrive_expect_tx(&bar[2], tz_bytes * (a.nch > 1 ? 2u : 1u));
          copy_z(a.nch - 1, (a.nch - 1) & 1, p0, &bar[2]);
          if (a.nch > 1) copy_z(a.nch - 2, (a.nch - 2) & 1, p0, &bar[2]);
        }
        pending |= 4u;
      } else {
        copy_z(a.nch - 1, (a.nch - 1) & 1, p0, nullptr);
        if (a.nch > 1) copy_z(a.nch - 2, (a.nch - 2) & 1, p0, nullptr);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
      }
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
    // the next chunk's checkpoint (factor state + this thread's substitution state), loaded
    // into registers one chunk ahead so that its latency hides behind a chunk of work
    F pf[kFF + kYT];
    {
      const F* ckc = ck + (size_t)((a.nch - 1) >> (G - 1)) * kFields * NP;
#pragma unroll
      for (int f = 0; f < kFF; ++f) pf[f] = ckc[(size_t)f * NP];
#pragma unroll
      for (int f = 0; f < kYT; ++f) pf[kFF + f] = ckc[(size_t)(kFF + h * kYT + f) * NP];
    }
    for (int c = a.nch - 1; c >= 0; --c) {
      const int st = pstage(c);
      // G = 2: the later chunk of a group (or a last chunk alone) leads: it recomputes the
      // whole group from the group's checkpoint; the earlier chunk then back-substitutes
      // from what the lead left in its stage.
      const int c0 = G == 2 ? (c & ~1) : c;
      const bool lead = G == 1 || (c & 1) || c == a.nch - 1;
      F* Sg = stage(st);
      if (lead) {
        if (G == 1) {
          if (c < a.nch - 2) {
            const bool ok = wait_bar(st, c >= 1 ? 1 : 0);
            if (__syncthreads_or(!ok)) {
              abort_all();
              return;
            }
          }
        }
        s.load_factor(pf, 1);
        s.load_y(pf + kFF, 1);
        if (c0 > 0) {
          const F* ckc = ck + (size_t)((c0 - 1) >> (G - 1)) * kFields * NP;
#pragma unroll
          for (int f = 0; f < kFF; ++f) pf[f] = ckc[(size_t)f * NP];
#pragma unroll
          for (int f = 0; f < kYT; ++f) pf[kFF + f] = ckc[(size_t)(kFF + h * kYT + f) * NP];
        }
        for (int q = c0; q <= c; ++q) {
          // G = 2: wait for each chunk of the group just before recomputing it (the later
          // chunk, loaded last, lands while the earlier one is recomputed)
          const int sq = pstage(q);
          if (G == 2 && ((pending >> sq) & 1u)) {
            const bool later_pending = q < c && ((pending >> pstage(c)) & 1u);
            const bool ok = wait_bar(sq, later_pending ? 1 : 0);
            if (__syncthreads_or(!ok)) {
              abort_all();
              return;
            }
          }
          F* Sq = stage(sq);
          const int ndq = min(C, T - q * C);
          F* Sx = Sq + h * NBT * NP + pl;
          const F* Sw = Sq + rowW * NP + pl;
          const F* Sl = Sq + rowL * NP + pl;
          // the day loop; MSE (ADJ) and the factor output (SMOOTH) are compile-time branches
          auto p2days = [&](auto xtra_tag) {
            constexpr bool MSE = MODE == MODE_ADJ && decltype(xtra_tag)::value;
            constexpr bool FAC = MODE == MODE_SMOOTH && decltype(xtra_tag)::value;
WS_UNROLL_N(WS_TILE_UNROLL)
            for (int k = 0; k < ndq; ++k, Sx += NB * NP, Sw += NP, Sl += NP) {
              const int i = q * C + k;
              const F wi = Sw[0];
              const F wa = Sw[D * NP];
              const F li = a.lam_scalar ? lam_s : Sl[0];
              const bool has_row = i < T - D;
              F bv[NBT], rho[D], yh[NBT], invD;
              const F mk = MSE && has_m ? Sq[(rowM + k) * NP + pl] : F(1);
#pragma unroll
              for (int j = 0; j < NBT; ++j) {
                const F xv = Sx[j * NP];
                bv[j] = MODE == MODE_SMOOTH ? (wi > F(0) ? wi * xv : F(0)) : xv;
                if (MSE) bv[j] = mscale * mk * (mk > F(0) ? Sx[rowZ * NP + j * NP] - xv : F(0));
              }
              s.factor_step(has_row, li, wa, rho, invD);
              s.subst_step(rho, invD, bv, yh);
#pragma unroll
              for (int j = 0; j < NBT; ++j) Sx[j * NP] = yh[j];
              if (h == 0) {
#pragma unroll
                for (int j = 1; j <= D; ++j) Sq[rho_row(j, k) * NP + pl] = rho[j - 1];
                if (FAC && act) {
                  gf[((size_t)i * (D + 1)) * a.P + p] = okser ? invD : F(0);
#pragma unroll
                  for (int j = 1; j <= D; ++j) gf[((size_t)i * (D + 1) + j) * a.P + p] = okser ? rho[j - 1] : F(0);
                }
              }
            }
          };
          if (MODE == MODE_ADJ ? mse : (MODE == MODE_SMOOTH && gf != nullptr && a.write_status))
            p2days(std::true_type{});
          else
            p2days(std::false_type{});
        }
      }
      const int nd = min(C, T - c * C);
      if (want_z && !mse && c == a.nch - 1 && a.tma) {  // z of the two chunks resident from pass 1
        const bool ok = wait_bar(2, 0);
        if (__syncthreads_or(!ok)) {
          abort_all();
          return;
        }
      } else if (S > 1 && lead) {
        __syncthreads();  // rho rows written by the h = 0 threads; w/lambda reads done
      }
      // back substitution over the chunk; ACC (ADJ with accumulation onto g0, the refined
      // adjoint) is a compile-time branch so that the plain adjoint carries none of its
      // loads and settle statistics
      auto bsub = [&](auto acc_tag) {
        constexpr bool ACC = MODE == MODE_ADJ && decltype(acc_tag)::value;
        F* Sx = Sg + ((nd - 1) * NB + h * NBT) * NP + pl;
        const F* Sz = Sg + (rowZ + (nd - 1) * NB + h * NBT) * NP + pl;
WS_UNROLL_N(WS_TILE_UNROLL)
        for (int k = nd - 1; k >= 0; --k, Sx -= NB * NP, Sz -= NB * NP) {
          const int i = c * C + k;
          F rho[D];
#pragma unroll
          for (int j = 1; j <= D; ++j) rho[j - 1] = Sg[rho_row(j, k) * NP + pl];
          F wk = F(0);
          if (MODE == MODE_ADJ) wk = Sg[(rowW + k) * NP + pl];
          F dl = F(0);
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            F acc = Sx[j * NP];
#pragma unroll
            for (int q = 1; q <= D; ++q) acc = fma(-rho[q - 1], zc[j][q - 1], acc);
#pragma unroll
            for (int q = D - 1; q > 0; --q) zc[j][q] = zc[j][q - 1];
            zc[j][0] = acc;
            F out = okser ? acc : F(0);
            if (MODE == MODE_RAW && want_z) out += Sz[j * NP];  // z0 + correction
            if (MODE == MODE_ADJ) {
              const F zv = Sz[j * NP];
              if (ACC && okser && act)  // g = g0 + correction
                out += gg0[((size_t)i * a.B + a.b0 + h * NBT + j) * a.P + p];
              F cg = out, cz = zv;           // level q at day t
              F pg = gn[j], pz = zt[j][0];   // level q-1 at day t+1 (q = 1: the values)
              zt[j][0] = zv;
              gn[j] = out;
              if (ACC) {
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
              if (ACC && i < T - D) dgmx = fmax(dgmx, fabs(cg));
              if (!a.raw_g) out = wk * out;
            }
            // a non-finite g or z reaches every earlier day through the back substitution,
            // so the plain solves test day 0 once at the end; outputs that add a stored
            // array (z0, g0) are tested day by day
            if (ACC || MODE == MODE_RAW) nanacc = fma(out, F(0), nanacc);
            Sx[j * NP] = out;
          }
          if (MODE == MODE_ADJ) gbuf[(h * C + k) * NP + pl] = i < T - D ? dl : F(0);
        }
      };
      if (MODE == MODE_ADJ && a.accum)
        bsub(std::true_type{});
      else
        bsub(std::false_type{});
      if (a.tma) fence_proxy_async_smem();
      __syncthreads();
      // dL/dlambda of the chunk's days: per-day lambda splits the days over the band halves
      // (day k by half k mod S, so neither waits for the other at the next barrier); scalar
      // lambda sums over all days in half 0
      if (MODE == MODE_ADJ && gout2 != nullptr && (!a.lam_scalar || h == 0)) {
        const int k0 = a.lam_scalar ? 0 : h, ks = a.lam_scalar ? 1 : S;
        const F* Sl = Sg + rowL * NP + pl;
        F* dst = gout2 + (size_t)(c * C + k0) * a.P + p;
        const bool first_group = a.b0 == 0;  // later band groups add onto the first's sums
        for (int k = k0; k < nd; k += ks, dst += (size_t)ks * a.P) {
          F dl = gbuf[k * NP + pl];
#pragma unroll
          for (int q = 1; q < S; ++q) dl += gbuf[(q * C + k) * NP + pl];
          F gl_t = okser ? -dl : F(0);
          if (a.grad_loglam) gl_t *= a.lam_scalar ? lam_s : Sl[k * NP];
          if (a.lam_scalar) {
            glam_sum += gl_t;
          } else if (act) {
            if (first_group)
              *dst = gl_t;
            else
              *dst += gl_t;
          }
        }
      }
      if (!a.tma && want_out && act)
        for (int k = 0; k < nd; ++k)
#pragma unroll
          for (int j = 0; j < NBT; ++j) {
            const int b = h * NBT + j;
            gout[((size_t)(c * C + k) * a.B + a.b0 + b) * a.P + p] = Sg[(size_t)(k * NB + b) * NP + pl];
          }
      if (MODE == MODE_ADJ || !a.tma) __syncthreads();  // stage reads done before it is refilled
      // refill the stage just freed: G = 1, chunk c - 2; G = 2, the next group's earlier
      // chunk after a lead (it is recomputed first), its later chunk after the earlier one
      const int nxt = G == 1 ? c - 2 : (lead ? ((c & 1) ? c - 3 : c - 2) : c - 1);
      if (a.tma) {
        if (tid == 0) {
          if (want_out) {
            tma_store_3d(&tm_o, Sg, p0, a.b0, c * C);
            bulk_commit();
          }
          if (nxt >= 0) {
            bulk_wait_read_all();
            issue(nxt, st, p0, want_z);
          }
        }
        if (nxt >= 0) pending |= 1u << st;
      } else if (nxt >= 0) {
        issue(nxt, st, p0, want_z);
      }
    }
    // per-series status; the band halves combine their non-finite flags
    if (MODE == MODE_SMOOTH || (MODE == MODE_ADJ && !a.accum)) {
#pragma unroll
      for (int j = 0; j < NBT; ++j) nanacc = fma(zc[j][0], F(0), nanacc);
    }
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
      if (h == 1) {
        nflag[pl] = (nonfin ? 1u : 0u) | (unsettled ? 2u : 0u);
        if (mse) gbuf[pl] = lsum;  // (the G region is free once the last chunk is done)
      }
      __syncthreads();
      if (h == 0) {
        nonfin = nonfin || (nflag[pl] & 1u) != 0u;
        unsettled = unsettled || (nflag[pl] & 2u) != 0u;
        if (mse) lsum += gbuf[pl];
      }
    }
    if (mse && a.loss != nullptr && act && h == 0) {
      F* lp = static_cast<F*>(a.loss) + p;
      const F v = F(0.5) * mscale * lsum;
      *lp = a.b0 == 0 ? v : *lp + v;
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

template <typename F, int D, int NBT, int S, int MODE, int NP>
int launch_tile_one(const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  auto kern = k_tile<F, D, NBT, S, MODE, NP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem_bytes);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  kern<<<cfg.grid, NP * S, cfg.smem_bytes, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "tile kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

// Kernel of a band group: FP32 groups of 1..10 bands (6, 8, 10 with two threads per pixel)
// at 128 or 64 pixels per CTA; FP64 groups of 1 band (2 for d = 2) at 128 pixels.
template <typename F, int D, int MODE, int NP>
const void* kernel_ptr_np(int nb) {
  if constexpr (sizeof(F) == 8) {
    if constexpr (NP != 128) {
      return nullptr;
    } else {
      if (nb == 2 && D == 2) return (const void*)k_tile<F, D, 2, 1, MODE, NP>;
      if (nb == 1) return (const void*)k_tile<F, D, 1, 1, MODE, NP>;
      return nullptr;
    }
  } else {
  switch (nb) {
    case 1: return (const void*)k_tile<F, D, 1, 1, MODE, NP>;
    case 2: return (const void*)k_tile<F, D, 2, 1, MODE, NP>;
    case 4: return (const void*)k_tile<F, D, 4, 1, MODE, NP>;
#ifndef WS_FAST_BUILD
    case 3: return (const void*)k_tile<F, D, 3, 1, MODE, NP>;
    case 5: return (const void*)k_tile<F, D, 5, 1, MODE, NP>;
    case 6: return (const void*)k_tile<F, D, 3, 2, MODE, NP>;
    case 7: return (const void*)k_tile<F, D, 7, 1, MODE, NP>;
    case 8: return (const void*)k_tile<F, D, 4, 2, MODE, NP>;
    case 9: return (const void*)k_tile<F, D, 9, 1, MODE, NP>;
    case 10: return (const void*)k_tile<F, D, 5, 2, MODE, NP>;
#endif
  }
  return nullptr;
  }
}

template <typename F, int D, int MODE, int NP>
int dispatch_tile_np(int nb, const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  if constexpr (sizeof(F) == 8) {
    if constexpr (NP == 128) {
      if (nb == 2 && D == 2) return launch_tile_one<F, D, 2, 1, MODE, NP>(cfg, a, maps, st);
      if (nb == 1) return launch_tile_one<F, D, 1, 1, MODE, NP>(cfg, a, maps, st);
    }
    return set_error(WS_EUNSUPPORTED, "FP64 band group of %d bands at %d pixels per CTA not instantiated", nb, NP);
  } else {
  switch (nb) {
    case 1: return launch_tile_one<F, D, 1, 1, MODE, NP>(cfg, a, maps, st);
    case 2: return launch_tile_one<F, D, 2, 1, MODE, NP>(cfg, a, maps, st);
    case 4: return launch_tile_one<F, D, 4, 1, MODE, NP>(cfg, a, maps, st);
#ifndef WS_FAST_BUILD
    case 3: return launch_tile_one<F, D, 3, 1, MODE, NP>(cfg, a, maps, st);
    case 5: return launch_tile_one<F, D, 5, 1, MODE, NP>(cfg, a, maps, st);
    case 6: return launch_tile_one<F, D, 3, 2, MODE, NP>(cfg, a, maps, st);
    case 7: return launch_tile_one<F, D, 7, 1, MODE, NP>(cfg, a, maps, st);
    case 8: return launch_tile_one<F, D, 4, 2, MODE, NP>(cfg, a, maps, st);
    case 9: return launch_tile_one<F, D, 9, 1, MODE, NP>(cfg, a, maps, st);
    case 10: return launch_tile_one<F, D, 5, 2, MODE, NP>(cfg, a, maps, st);
#endif
    default: return set_error(WS_EUNSUPPORTED, "band group of %d bands not instantiated", nb);
  }
  }
}

template <typename F, int D, int MODE>
const void* kernel_ptr_nb(int nb, int np) {
  return np == 64 ? kernel_ptr_np<F, D, MODE, 64>(nb) : kernel_ptr_np<F, D, MODE, 128>(nb);
}

template <typename F, int D, int MODE>
int dispatch_tile_nb(int nb, const TileCfg& cfg, const TileArgs& a, const CUtensorMap* maps, cudaStream_t st) {
  return cfg.NP == 64 ? dispatch_tile_np<F, D, MODE, 64>(nb, cfg, a, maps, st)
                      : dispatch_tile_np<F, D, MODE, 128>(nb, cfg, a, maps, st);
}

template <int D>
const void* tile_kernel_ptr_t(const ws_problem& pb, int mode, int nb, int np) {
  if (pb.dtype == WS_F32) {
    switch (mode) {
      case MODE_SMOOTH: return kernel_ptr_nb<float, D, MODE_SMOOTH>(nb, np);
      case MODE_RAW: return kernel_ptr_nb<float, D, MODE_RAW>(nb, np);
      case MODE_ADJ: return kernel_ptr_nb<float, D, MODE_ADJ>(nb, np);
    }
  } else {
    switch (mode) {
      case MODE_SMOOTH: return kernel_ptr_nb<double, D, MODE_SMOOTH>(nb, np);
      case MODE_RAW: return kernel_ptr_nb<double, D, MODE_RAW>(nb, np);
      case MODE_ADJ: return kernel_ptr_nb<double, D, MODE_ADJ>(nb, np);
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
