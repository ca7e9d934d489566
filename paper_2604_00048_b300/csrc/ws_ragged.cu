// Ragged batches: series of different lengths T_i and orders d_i packed back to back,
// band b of series i at x[b*N + off[i] + t] (N = off[n]), w and lambda like one band.
//
// Host plan: series are sorted by (d, length descending) and cut into work items of 32
// (one per lane), so every warp runs one order and lanes of similar length; items are
// ordered largest first. A persistent grid of warps pulls items from an atomic counter.
// Per item, the warp runs the same two-pass recurrence as the tile kernels (ws_sweep.cuh):
// pass 1 forward over chunks of RC days with checkpoints, pass 2 backward recomputing each
// chunk from its checkpoint. Each lane owns one series; chunks are staged in shared memory
// by warp-cooperative LDGSTS copies that read each series contiguously (coalesced) and
// write a padded [day][lane] layout (conflict-free), and results leave the same way.
// The launch (counter reset + kernel) is captured in a CUDA graph and replayed; an
// autotuner picks the chunk length and warps per CTA on the plan's own data.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <vector>

#include "ws_internal.h"
#include "ws_df.cuh"
#include "ws_ptx.cuh"
#include "ws_sweep.cuh"

namespace ws {

constexpr int kPitch = 33;  // shared-memory row pitch: 32 lanes + 1 pad

struct RaggedArgs {
  const int64_t* off;     // n + 1
  const int32_t* order;   // n_items * 32 series ids (-1 = idle lane)
  const int8_t* item_d;   // order of each item
  const int32_t* item_t;  // longest series of each item
  int n_items;
  int64_t N;              // off[n]
  int B, band;            // band of this launch
  int lam_scalar;
  const float* x;
  const float* w;
  const float* lam;
  float* z;
  uint8_t* status;
  float* ckpt;            // per persistent warp: max_nch * kFieldsMax * 32
  int max_nch;
  int* counter;
  unsigned* err;
  int warp_rows;          // ragged_warp_rows(RC, largest order of the plan)
  // refinement (plan-owned; NULL without WS_PLAN_REFINE)
  float* resid;           // r = W x - Omega z, same packing as x
  uint8_t* active;        // per item: 1 while some series of the item has not settled
  uint8_t* conv;          // per series, after the last correction: bit 0 settled, bit 1 done
                          // (later steps leave the series out), bit 2 listed for the
                          // double-float re-solve by the first step
  float* zmax;            // per series: max |z| of the unrefined solution
  float* prevc;           // per series: max |correction| of the previous step (0 before the first)
  int32_t* list64;        // series re-solved in double-float
  int* count64;
  double* ck64;           // double-float re-solve: per thread, (yhat, rho_1..rho_d) of every day
                          // (8 bytes each), interleaved across the kernel's threads
  const int8_t* d_of;     // per series order
  float tau, tau_drop, tau_cond;
  const uint8_t* item_tiled;  // per item: 1 = its series are solved through the length-class tiles
};

constexpr int kFieldsMax = 4 * 5 + 4;  // d(d+1) + d for d <= 4, one band
constexpr int kHPBlocksPerSM = 5;    // double-float re-solve: 5 x 128 threads per SM (at most 102 registers each)

template <int RC>
struct RaggedSmem {
  // one stage, rows of kPitch floats: X [RC], W [RC + 4], L [RC]
  static constexpr int rowX = 0, rowW = RC, rowL = 2 * RC + 4, rows = 3 * RC + 4;
};
// Shared-memory rows of one warp: two stages, then E [(max_d - 2) * RC] rows holding rho_3..
// of the chunk being back-substituted (pass 2 only, so a single copy).
__host__ __device__ inline int ragged_warp_rows(int RC, int max_d) {
  return 2 * (3 * RC + 4) + (max_d > 2 ? max_d - 2 : 0) * RC;
}

// One item (32 series of order D) on one warp. RAW: the right-hand side is taken as given
// (the refinement residual) and the solution is added to z (z0 + correction).
template <int D, int RC, int MODE>
__device__ void ragged_item(const RaggedArgs& a, int item, float* sm, float* ck, int lane) {
  using L = RaggedSmem<RC>;
  using SW = Sweep<float, D, 1>;
  constexpr int kFF = SW::kFactorFields;
  constexpr int kF = kFF + D;
  const int sid = a.order[(size_t)item * 32 + lane];
  const bool live = sid >= 0;
  const int64_t off = live ? a.off[sid] : 0;
  const int T = live ? (int)(a.off[sid + 1] - off) : 0;
  const int nch = (a.item_t[item] + RC - 1) / RC;
  if (MODE == MODE_RAW && !a.active[item]) return;  // every series of the item has settled
  if (a.item_tiled != nullptr && a.item_tiled[item]) return;  // solved (or refined) as tiles
  const float* xb = MODE == MODE_RAW ? a.resid : a.x + (size_t)a.band * a.N;
  float* zb = a.z + (size_t)a.band * a.N;
  auto stg = [&](int st) -> float* { return sm + (size_t)st * L::rows * kPitch; };
  float* const E = sm + (size_t)2 * L::rows * kPitch;
  if (nch == 0) {  // every series of the item is empty
    if (live && a.status != nullptr && a.band == 0) a.status[sid] = WS_SERIES_OK;
    return;
  }

  // warp-cooperative staging of chunk c into stage st: for every series s of the item,
  // consecutive lanes copy consecutive days (coalesced), into row = day, column = s.
  auto issue = [&](int c, int st) {
    float* S = stg(st);
    const int t0 = c * RC;
    for (int s = 0; s < 32; ++s) {
      const int64_t os = __shfl_sync(0xffffffffu, off, s);
      const int Ts = __shfl_sync(0xffffffffu, T, s);
      for (int j = lane; j < RC + 4; j += 32) {
        const int t = t0 + j;
        const bool v = t < Ts;
        const int64_t g = os + (v ? t : 0);
        if (j < RC) {
          cp_async_elem<4>(S + (L::rowX + j) * kPitch + s, xb + g, v);
          if (!a.lam_scalar) cp_async_elem<4>(S + (L::rowL + j) * kPitch + s, a.lam + g, v);
        }
        cp_async_elem<4>(S + (L::rowW + j) * kPitch + s, a.w + g, v);
      }
    }
    cp_async_commit();
  };

  SW s;
  s.reset();
  int npos = 0;
  bool bad = false;
  const float ls = (live && a.lam_scalar) ? a.lam[sid] : 0.f;
  issue(0, 0);
  if (nch > 1) issue(1, 1);
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) cp_async_wait<1>(); else cp_async_wait<0>();
    __syncwarp();
    const float* S = stg(c & 1);
    if (c == 0)
      for (int m = 0; m < D; ++m)
        if (m < T) s.init_weight(m, S[(L::rowW + m) * kPitch + lane]);
    float* ckc = ck + (size_t)c * kF * 32 + lane;
    s.save_factor(ckc, 32);
    s.save_y(ckc + kFF * 32, 32);
    const int nd = min(RC, T - c * RC);
    for (int k = 0; k < nd; ++k) {
      const int i = c * RC + k;
      const float wi = S[(L::rowW + k) * kPitch + lane];
      const float wa = S[(L::rowW + k + D) * kPitch + lane];
      const float li = a.lam_scalar ? ls : S[(L::rowL + k) * kPitch + lane];
      const bool has_row = i < T - D;
      bad |= !(wi >= 0.f) || !isfinite(wi);
      npos += wi > 0.f;
      if (has_row) bad |= !(li > 0.f) || !isfinite(li);
      float bv[1] = {MODE == MODE_RAW ? S[(L::rowX + k) * kPitch + lane]
                                      : (wi > 0.f ? wi * S[(L::rowX + k) * kPitch + lane] : 0.f)};
      float rho[D], yh[1], invD;
      s.factor_step(has_row, li, wa, rho, invD);
      s.subst_step(rho, invD, bv, yh);
    }
    __syncwarp();
    if (c + 2 < nch) issue(c + 2, c & 1);
  }
  const int dmin = D < T ? D : T;
  const uint8_t code = bad ? WS_SERIES_BADARG : (npos < dmin ? WS_SERIES_NOT_PD : WS_SERIES_OK);
  const bool okser = code == WS_SERIES_OK;
  float zc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) zc[j] = 0.f;
  float nanacc = 0.f, amax = 0.f;
  for (int c = nch - 1; c >= 0; --c) {
    const int st = c & 1;
    if (c < nch - 2) {
      if (c >= 1) cp_async_wait<1>(); else cp_async_wait<0>();
      __syncwarp();
    }
    float* S = stg(st);
    const int t0 = c * RC;
    const float* ckc = ck + (size_t)c * kF * 32 + lane;
    s.load_factor(ckc, 32);
    s.load_y(ckc + kFF * 32, 32);
    const int nd = min(RC, T - c * RC);
    for (int k = 0; k < nd; ++k) {
      const int i = c * RC + k;
      const float wi = S[(L::rowW + k) * kPitch + lane];
      const float wa = S[(L::rowW + k + D) * kPitch + lane];
      const float li = a.lam_scalar ? ls : S[(L::rowL + k) * kPitch + lane];
      const bool has_row = i < T - D;
      float bv[1] = {MODE == MODE_RAW ? S[(L::rowX + k) * kPitch + lane]
                                      : (wi > 0.f ? wi * S[(L::rowX + k) * kPitch + lane] : 0.f)};
      float rho[D], yh[1], invD;
      s.factor_step(has_row, li, wa, rho, invD);
      s.subst_step(rho, invD, bv, yh);
      S[(L::rowX + k) * kPitch + lane] = yh[0];
      // rho_1 over lambda, rho_2 over w (both already consumed for day k), rho_3.. in E
      S[(L::rowL + k) * kPitch + lane] = rho[0];
      if (D >= 2) S[(L::rowW + k) * kPitch + lane] = rho[D >= 2 ? 1 : 0];
#pragma unroll
      for (int j = 3; j <= D; ++j) E[((j - 3) * RC + k) * kPitch + lane] = rho[j - 1];
    }
    for (int k = nd - 1; k >= 0; --k) {
      float rho[D];
      rho[0] = S[(L::rowL + k) * kPitch + lane];
      if (D >= 2) rho[D >= 2 ? 1 : 0] = S[(L::rowW + k) * kPitch + lane];
#pragma unroll
      for (int j = 3; j <= D; ++j) rho[j - 1] = E[((j - 3) * RC + k) * kPitch + lane];
      float acc = S[(L::rowX + k) * kPitch + lane];
#pragma unroll
      for (int j = 1; j <= D; ++j) acc = fmaf(-rho[j - 1], zc[j - 1], acc);
#pragma unroll
      for (int j = D - 1; j > 0; --j) zc[j] = zc[j - 1];
      zc[0] = acc;
      const float out = okser ? acc : 0.f;
      nanacc = fmaf(out, 0.f, nanacc);
      amax = fmaxf(amax, fabsf(out));
      S[(L::rowX + k) * kPitch + lane] = out;
    }
    __syncwarp();
    // transposed store of the chunk: consecutive lanes write consecutive days of series s
    // (RC <= 32: one day per lane). RAW adds the correction to z0, whose loads are issued
    // 8 series at a time ahead of the stores (they may alias as far as the compiler knows).
    static_assert(RC <= 32, "one day per lane in the transposed store");
    for (int s0 = 0; s0 < 32; s0 += 8) {
      int64_t gi[8];
      bool ok[8];
      float z0v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t os = __shfl_sync(0xffffffffu, off, s0 + q);
        const int Ts = __shfl_sync(0xffffffffu, T, s0 + q);
        gi[q] = os + t0 + lane;
        ok[q] = lane < RC && t0 + lane < Ts;
        z0v[q] = (MODE == MODE_RAW && ok[q]) ? zb[gi[q]] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (ok[q]) zb[gi[q]] = z0v[q] + S[(L::rowX + lane) * kPitch + s0 + q];  // RAW: z0 + correction
    }
    __syncwarp();
    if (c >= 2) issue(c - 2, st);
  }
  if (MODE == MODE_SMOOTH && live && a.zmax != nullptr) a.zmax[sid] = amax;
  if (MODE == MODE_RAW) {
    // Settle test. The first correction measures the FP32 solve's own error: above
    // tau_cond * max|z| the series is ill-conditioned for FP32 (eps32 * cond near 1), where
    // the corrections can shrink quickly towards a point still far from the solution (the
    // refinement's limit is set by the residual's rounding times cond(Omega)); such a series
    // leaves the FP32 steps and is listed for the double-float re-solve at once.
    // Otherwise a series has settled when its correction is below tau * max|z| (NaN never
    // settles) and the step contracts: the correction at most half the previous one, so the
    // error left (correction * ratio / (1 - ratio)) is below the correction; the first step
    // has no ratio and needs tau_drop. A series is done, and leaves the later steps, below
    // tau_drop * max|z|.
    if (!(nanacc == 0.f)) amax = __int_as_float(0x7fc00000);  // a non-finite correction (fmaxf drops NaN)
    const float zm = live ? a.zmax[sid] : 0.f;
    const float prev = live ? a.prevc[sid] : 0.f;
    const bool small = amax <= a.tau_drop * zm;
    const bool suspect = live && prev == 0.f && amax > a.tau_cond * zm;
    const bool done = !live || small || suspect;
    const bool settled = !live || (!suspect && (small || (amax <= a.tau * zm && amax <= 0.5f * prev)));
    if (live) {
      a.prevc[sid] = amax;
      a.conv[sid] = (settled ? 1 : 0) | (done ? 2 : 0) | (suspect ? 4 : 0);
      if (suspect) a.list64[atomicAdd(a.count64, 1)] = sid;
    }
    if (__all_sync(0xffffffffu, done) && lane == 0) a.active[item] = 0;
  }
  if (MODE == MODE_SMOOTH && live && a.status != nullptr) {
    const bool nonfin = !(nanacc == 0.f);
    if (a.band == 0)
      a.status[sid] = okser ? (nonfin ? WS_SERIES_NONFINITE : WS_SERIES_OK) : code;
    else if (nonfin && a.status[sid] == WS_SERIES_OK)
      a.status[sid] = WS_SERIES_NONFINITE;
  }
}

template <int RC, int MODE>
__global__ void __launch_bounds__(512, 1) k_ragged(const RaggedArgs a) {
  extern __shared__ __align__(16) float rsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* sm = rsm + (size_t)wid * a.warp_rows * kPitch;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wid;  // persistent warp id
  float* ck = a.ckpt + (size_t)gw * a.max_nch * kFieldsMax * 32;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    switch (a.item_d[item]) {
      case 1: ragged_item<1, RC, MODE>(a, item, sm, ck, lane); break;
      case 2: ragged_item<2, RC, MODE>(a, item, sm, ck, lane); break;
      case 3: ragged_item<3, RC, MODE>(a, item, sm, ck, lane); break;
      case 4: ragged_item<4, RC, MODE>(a, item, sm, ck, lane); break;
    }
  }
}

// Refinement residual of a ragged batch, r = W x - Omega z0, carried in double-word
// arithmetic from the first difference on: the series of this path reach cond(Omega) ~ 1e13
// (unsmoothed lambda up to 1e5, d = 3, sparse weights), where a working-precision residual
// would stall the refinement at the FP32 solution's own error. One warp per item, the lanes
// over 32 consecutive days of one series at a time (coalesced, no recurrence). Each lane forms
// its own row q_t = lambda_t (D z0)_t once; D^T q at day t is the d-th backward difference
// of q, built level by level from the previous lane's value (shuffle), lane 0 taking the last
// lane's value of the previous 32 days.
template <int D>
__device__ void ragged_resid_item(const RaggedArgs& a, int item, int lane) {
  using DWf = DW<float>;
  const float* xb = a.x + (size_t)a.band * a.N;
  const float* zb = a.z + (size_t)a.band * a.N;
  float* rb = a.resid;  // one band at a time
  for (int s = 0; s < 32; ++s) {
    const int sid = a.order[(size_t)item * 32 + s];
    if (sid < 0) continue;
    const int64_t os = a.off[sid];
    const int T = (int)(a.off[sid + 1] - os);
    const float ls = a.lam_scalar ? a.lam[sid] : 0.f;
    DWf carry[D];  // nabla^j q at the previous block's last day, j = 0..D-1
#pragma unroll
    for (int j = 0; j < D; ++j) carry[j] = DWf{0.f, 0.f};
    for (int t0 = 0; t0 < T; t0 += 32) {
      const int t = t0 + lane;
      // q_t = lambda_t (D^D z0)_t, the nested first differences exact from the first on
      DWf lv = {0.f, 0.f};
      if (t <= T - D - 1) {
        DWf dz[D];
#pragma unroll
        for (int m = 0; m < D; ++m) dz[m] = two_sum(zb[os + t + m + 1], -zb[os + t + m]);
#pragma unroll
        for (int i = 1; i < D; ++i)
#pragma unroll
          for (int m = 0; m < D - i; ++m) dz[m] = dw_add(dz[m + 1], DWf{-dz[m].hi, -dz[m].lo});
        lv = dw_scale(dz[0], a.lam_scalar ? ls : a.lam[os + t]);
      }
      // nabla^j q_t = nabla^{j-1} q_t - nabla^{j-1} q_{t-1}
#pragma unroll
      for (int j = 0; j < D; ++j) {
        DWf prev = {__shfl_up_sync(0xffffffffu, lv.hi, 1), __shfl_up_sync(0xffffffffu, lv.lo, 1)};
        if (lane == 0) prev = carry[j];
        carry[j] = DWf{__shfl_sync(0xffffffffu, lv.hi, 31), __shfl_sync(0xffffffffu, lv.lo, 31)};
        lv = dw_add(lv, DWf{-prev.hi, -prev.lo});
      }
      if (t < T) {
        const DWf v = (D % 2) ? DWf{-lv.hi, -lv.lo} : lv;  // (D^T q)_t
        const float wt = a.w[os + t], xt = xb[os + t], zt = zb[os + t];
        DWf acc = wt > 0.f ? dw_scale(two_sum(xt, -zt), wt) : DWf{0.f, 0.f};
        acc = dw_add(acc, DWf{-v.hi, -v.lo});
        rb[os + t] = acc.hi + acc.lo;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_ragged_resid(const RaggedArgs a) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items || !a.active[item]) return;
  if (a.item_tiled != nullptr && a.item_tiled[item]) return;  // refined as tiles
  switch (a.item_d[item]) {
    case 1: ragged_resid_item<1>(a, item, lane); break;
    case 2: ragged_resid_item<2>(a, item, lane); break;
    case 3: ragged_resid_item<3>(a, item, lane); break;
    case 4: ragged_resid_item<4>(a, item, lane); break;
  }
}

// Series whose FP32 refinement has not settled are listed for a double-float re-solve: one warp
// per item, one atomic per warp, so the list keeps the items' (order, length) grouping
// within each item and roughly across items.
__global__ void __launch_bounds__(256) k_ragged_collect(const RaggedArgs a) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items || !a.active[item]) return;
  const int sid = a.order[(size_t)item * 32 + lane];
  const bool need = sid >= 0 && !(a.conv[sid] & 1) && !(a.conv[sid] & 4);  // bit 2: listed already
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (m == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(a.count64, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (need) a.list64[base + __popc(m & ((1u << lane) - 1u))] = sid;
}

// Regrouping between refinement steps: the series not yet done after a step are listed
// per order (one region of the compacted list per order, sized for all of that order's
// series, in items of 32), so the next step runs those series only, in fresh items. One warp
// per item, one atomic per warp; appends follow the items' (order, length) grouping.
__global__ void __launch_bounds__(256) k_ragged_compact(const RaggedArgs a, int32_t* __restrict__ dst,
                                                        int* __restrict__ cnt, int4 reg) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items || !a.active[item]) return;
  const int sid = a.order[(size_t)item * 32 + lane];
  const bool need = sid >= 0 && !(a.conv[sid] & 2);
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (m == 0) return;
  const int d = a.item_d[item];
  int base = 0;
  if (lane == 0) base = atomicAdd(&cnt[d - 1], __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  const int r0 = d == 1 ? reg.x : (d == 2 ? reg.y : (d == 3 ? reg.z : reg.w));
  if (need) dst[r0 + base + __popc(m & ((1u << lane) - 1u))] = sid;
}

// Items of the compacted list: order and longest series of each, idle lanes marked -1,
// items past their region's count inactive. reg: first slot of each order's region.
__global__ void __launch_bounds__(256) k_ragged_regroup(const int64_t* __restrict__ off, int32_t* __restrict__ order,
                                                        const int* __restrict__ cnt, int4 reg, int n_items,
                                                        int8_t* __restrict__ item_d, int32_t* __restrict__ item_t,
                                                        uint8_t* __restrict__ active) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= n_items) return;
  const int slot = item * 32;
  const int d = slot < reg.y ? 1 : (slot < reg.z ? 2 : (slot < reg.w ? 3 : 4));
  const int r0 = d == 1 ? reg.x : (d == 2 ? reg.y : (d == 3 ? reg.z : reg.w));
  const bool live = slot - r0 + lane < cnt[d - 1];
  int T = 0;
  if (live) {
    const int sid = order[slot + lane];
    T = (int)(off[sid + 1] - off[sid]);
  } else {
    order[slot + lane] = -1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) T = max(T, __shfl_xor_sync(0xffffffffu, T, o));
  const unsigned m = __ballot_sync(0xffffffffu, live);
  if (lane == 0) {
    item_d[item] = (int8_t)d;
    item_t[item] = T;
    active[item] = m != 0u ? 1 : 0;
  }
}

// High-precision re-solve of one listed series by one thread: the rotation factor, forward
// and back substitution in double-float (HP = dwf, about 48 bits) instead of FP32, inputs
// read directly from global memory (a small share of the batch goes this way). The forward
// sweep stores each day's (yhat, rho_1..rho_d) in the thread's workspace column (word f of
// day i at st[(i * (1 + d) + f) * nt], nt = threads of the launch, so a warp's stores of one
// day are contiguous); the backward sweep reads them back four days ahead of their use
// instead of recomputing the factor. Overwrites z of the series.
using HP = dwf;
static_assert(sizeof(HP) == sizeof(double), "the per-day store holds 8-byte values");

template <int D>
__device__ void ragged64_series(const RaggedArgs& a, int sid, HP* st, size_t nt) {
  using SW = Sweep<HP, D, 1>;
  constexpr int kSF = 1 + D;  // words per day: yhat, rho_1..rho_D
  const int64_t os = a.off[sid];
  const int T = (int)(a.off[sid + 1] - os);
  const float* xs = a.x + (size_t)a.band * a.N + os;
  const float* ws = a.w + os;
  const float* lsr = a.lam + (a.lam_scalar ? (int64_t)sid : os);
  float* zs = a.z + (size_t)a.band * a.N + os;
  auto lam_at = [&](int i) -> HP { return HP(a.lam_scalar ? lsr[0] : lsr[i]); };
  auto w_at = [&](int i) -> HP { return HP(i < T ? ws[i] : 0.f); };
  const HP zero(0.f);
  SW s;
  s.reset();
  for (int m = 0; m < D && m < T; ++m) s.init_weight(m, w_at(m));
  for (int i = 0; i < T; ++i) {
    const HP wi = w_at(i);
    HP bv[1] = {wi > zero ? wi * HP(xs[i]) : zero};
    HP rho[D], yh[1], invD;
    s.factor_step(i < T - D, i < T - D ? lam_at(i) : zero, w_at(i + D), rho, invD);
    s.subst_step(rho, invD, bv, yh);
    HP* e = st + (size_t)i * kSF * nt;
    e[0] = yh[0];
#pragma unroll
    for (int j = 0; j < D; ++j) e[(size_t)(j + 1) * nt] = rho[j];
  }
  // back substitution, z_i = yhat_i - sum_j rho_{i,j} z_{i+j}; four register sets hold the
  // words of the next four days, each reloaded four days ahead of its use
  HP zc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) zc[j] = zero;
  auto load = [&](int i, HP (&v)[kSF]) {
    const HP* e = st + (size_t)i * kSF * nt;
#pragma unroll
    for (int f = 0; f < kSF; ++f) v[f] = e[(size_t)f * nt];
  };
  auto step = [&](int i, const HP (&v)[kSF]) {
    HP acc = v[0];
#pragma unroll
    for (int j = 1; j <= D; ++j) acc = fma(-v[j], zc[j - 1], acc);
#pragma unroll
    for (int j = D - 1; j > 0; --j) zc[j] = zc[j - 1];
    zc[0] = acc;
    zs[i] = acc.to_float();
  };
  HP b0[kSF], b1[kSF], b2[kSF], b3[kSF];
  int i = T - 1;
  if (i >= 0) load(i, b0);
  if (i >= 1) load(i - 1, b1);
  if (i >= 2) load(i - 2, b2);
  if (i >= 3) load(i - 3, b3);
  for (; i >= 3; i -= 4) {
    step(i, b0);
    if (i >= 4) load(i - 4, b0);
    step(i - 1, b1);
    if (i >= 5) load(i - 5, b1);
    step(i - 2, b2);
    if (i >= 6) load(i - 6, b2);
    step(i - 3, b3);
    if (i >= 7) load(i - 7, b3);
  }
  if (i >= 0) step(i, b0);
  if (i >= 1) step(i - 1, b1);
  if (i >= 2) step(i - 2, b2);
}

__global__ void __launch_bounds__(128, kHPBlocksPerSM) k_ragged64(const RaggedArgs a) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nt = (size_t)gridDim.x * blockDim.x;
  HP* st = reinterpret_cast<HP*>(a.ck64) + gt;
  const int n = *a.count64;
  for (int j = gt; j < n; j += (int)nt) {
    const int sid = a.list64[j];
    const int d = a.d_of[sid];
    if (d == 1) ragged64_series<1>(a, sid, st, nt);
    else if (d == 2) ragged64_series<2>(a, sid, st, nt);
    else if (d == 3) ragged64_series<3>(a, sid, st, nt);
    else ragged64_series<4>(a, sid, st, nt);
  }
}

// Length classes: series of one order whose lengths round up to the same T_c are solved as
// one [T_c][P_c] tile problem by the tile kernels (TMA staging, two CTAs per SM). A series
// of length T is padded to T_c with w = 0, x = 0 (lambda = 1 on padded rows): the padded
// problem's minimiser agrees with the original one on days 0..T-1, because z on the padded
// days can continue the last d values so that every added difference row is zero.
// Gather: packed series -> tile columns (a 32 x 32 transpose through shared memory, reads
// coalesced along days, writes along series). Scatter: back, with the status codes and the
// per-series max |z| the refinement's settle test needs.
constexpr int kTileMinT = 64;  // shorter series stay on the per-lane kernel
constexpr int kTileStreams = 32;  // a class fills only part of the GPU: run 32 at a time (8: 40.3 ms, 16: 29.1, 32: 28.3 for the 1,048,576-series solve)
constexpr int kClassRound = 32;

__global__ void __launch_bounds__(256) k_gather(const RaggedArgs a, const int32_t* __restrict__ sids, int Pc,
                                                int Tc, float* __restrict__ tx, float* __restrict__ tw,
                                                float* __restrict__ tl) {
  __shared__ float sx[32][33], sw[32][33], sl[32][33];
  const int p0 = blockIdx.x * 32, t0 = blockIdx.y * 32, lx = threadIdx.x, ly = threadIdx.y;
  for (int j = ly; j < 32; j += 8) {
    const int p = p0 + j, t = t0 + lx;
    const int sid = p < Pc ? sids[p] : -1;
    float xv = 0.f, wv = 0.f, lv = 1.f;
    if (sid >= 0) {
      const int64_t os = a.off[sid];
      const int T = (int)(a.off[sid + 1] - os);
      if (t < T) {
        xv = a.x[os + t];
        wv = a.w[os + t];
        lv = a.lam_scalar ? a.lam[sid] : a.lam[os + t];
      }
    }
    sx[j][lx] = xv;
    sw[j][lx] = wv;
    sl[j][lx] = lv;
  }
  __syncthreads();
  for (int j = ly; j < 32; j += 8) {
    const int t = t0 + j, p = p0 + lx;
    if (t < Tc && p < Pc) {
      const size_t o = (size_t)t * Pc + p;
      tx[o] = sx[lx][j];
      tw[o] = sw[lx][j];
      tl[o] = sl[lx][j];
    }
  }
}

__global__ void __launch_bounds__(256) k_scatter(const RaggedArgs a, const int32_t* __restrict__ sids, int Pc,
                                                 int Tc, const float* __restrict__ tz,
                                                 const uint8_t* __restrict__ tst) {
  __shared__ float sz[32][33];
  const int p0 = blockIdx.x * 32, t0 = blockIdx.y * 32, lx = threadIdx.x, ly = threadIdx.y;
  for (int j = ly; j < 32; j += 8) {
    const int t = t0 + j, p = p0 + lx;
    sz[lx][j] = (t < Tc && p < Pc) ? tz[(size_t)t * Pc + p] : 0.f;
  }
  __syncthreads();
  for (int j = ly; j < 32; j += 8) {
    const int p = p0 + j, t = t0 + lx;
    const int sid = p < Pc ? sids[p] : -1;
    if (sid < 0) continue;
    const int64_t os = a.off[sid];
    const int T = (int)(a.off[sid + 1] - os);
    float m = 0.f;
    if (t < T) {
      const float v = sz[j][lx];
      a.z[os + t] = v;
      m = fabsf(v);
    }
    if (a.zmax != nullptr) {  // max |z| over the series (non-negative floats order as integers)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lx == 0) atomicMax(reinterpret_cast<int*>(a.zmax) + sid, __float_as_int(m));
    }
    if (blockIdx.y == 0 && lx == 0 && a.status != nullptr) a.status[sid] = tst[p];
  }
}

// After the length classes' tile refinement step: z of the tile back into the packed
// series, and per series the largest |correction| over its days (against the z it
// replaces), for the step's settle test. NaN corrections order above every finite value
// (the integer max of the bit patterns keeps them).
__global__ void __launch_bounds__(256) k_scatter_refine(const RaggedArgs a, const int32_t* __restrict__ sids,
                                                        int Pc, int Tc, const float* __restrict__ tz,
                                                        float* __restrict__ tcorr) {
  __shared__ float sz[32][33];
  const int p0 = blockIdx.x * 32, t0 = blockIdx.y * 32, lx = threadIdx.x, ly = threadIdx.y;
  for (int j = ly; j < 32; j += 8) {
    const int t = t0 + j, p = p0 + lx;
    sz[lx][j] = (t < Tc && p < Pc) ? tz[(size_t)t * Pc + p] : 0.f;
  }
  __syncthreads();
  // a warp handles four series (rows j = ly + 8q) of 32 days: every load is issued before the
  // first store (the stores could alias them for the compiler)
  const int t = t0 + lx;
  int sid[4];
  int64_t os[4];
  bool in[4];
  float old[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int p = p0 + ly + 8 * q;
    sid[q] = p < Pc ? sids[p] : -1;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    os[q] = sid[q] >= 0 ? a.off[sid[q]] : 0;
    in[q] = sid[q] >= 0 && t < (int)(a.off[sid[q] + 1] - os[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) old[q] = in[q] ? a.z[os[q] + t] : 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (sid[q] < 0) continue;  // uniform over the warp (one series per row)
    int m = 0;
    if (in[q]) {
      const float v = sz[ly + 8 * q][lx];
      m = __float_as_int(fabsf(v - old[q]));
      a.z[os[q] + t] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lx == 0) atomicMax(reinterpret_cast<int*>(tcorr) + sid[q], m);
  }
}

// Settle test of the tile refinement step, per series of the length classes: the first step's
// test of the per-lane correction kernel (no previous correction): listed for the
// double-float re-solve above tau_cond * max|z|, settled and done below tau_drop * max|z|,
// otherwise left to the next FP32 step.
__global__ void __launch_bounds__(256) k_tile_settle(const RaggedArgs a, const int32_t* __restrict__ sids, int n,
                                                     const float* __restrict__ tcorr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int sid = sids[i];
  if (sid < 0) return;
  const float zm = a.zmax[sid], amax = tcorr[sid];
  const bool small = amax <= a.tau_drop * zm;
  const bool suspect = amax > a.tau_cond * zm;
  const bool done = small || suspect;
  const bool settled = !suspect && small;
  a.prevc[sid] = amax;
  a.conv[sid] = (settled ? 1 : 0) | (done ? 2 : 0) | (suspect ? 4 : 0);
  if (suspect) a.list64[atomicAdd(a.count64, 1)] = sid;
}

}  // namespace ws

using namespace ws;

struct LenClass {
  int d, Tc, Pc;
  size_t base;     // element offset of the class tile in the tile arrays
  int sid_base;    // offset of the class's series ids in d_class_sid
};

struct ws_plan {
  ws_ragged rg;
  int n_items = 0, max_t = 0, max_d = 1;
  int RC = 16, warps = 8, grid = 0;
  int64_t N = 0;
  int32_t* d_order = nullptr;
  int8_t* d_item_d = nullptr;
  int32_t* d_item_t = nullptr;
  int* d_counter = nullptr;
  unsigned* d_err = nullptr;
  // per-execute scratch: views into the caller's workspace (ws_plan_workspace_size), bound
  // by each ws_plan_execute; the plan owns only its tables
  float* d_ckpt = nullptr;
  void* ws_base = nullptr;     // workspace of the last execute
  uint32_t ws_flags = 0;       // flags it was laid out for
  // refinement state (WS_PLAN_REFINE)
  float* d_resid = nullptr;    // N floats (one band at a time)
  uint8_t* d_active = nullptr; // n_items
  uint8_t* d_conv = nullptr;   // n_series
  float* d_zmax = nullptr;     // n_series
  float* d_tcorr = nullptr;    // n_series: max |correction| of the length classes' tile refinement step
  float* d_prevc = nullptr;    // n_series
  int32_t* d_list64 = nullptr; // n_series
  int* d_count64 = nullptr;    // n_bands
  double* d_ck64 = nullptr;
  int8_t* d_dof = nullptr;     // n_series
  int max_t64 = 0, sf64 = 1, grid64 = 0;  // longest series, words per day (1 + largest d)
  // regrouped items of refinement steps 2.. (two sets, written alternately)
  int creg[5] = {0, 0, 0, 0, 0};  // first slot of each order's region; creg[4] = all slots
  int32_t* d_corder = nullptr;     // 2 x creg[4]
  int8_t* d_citem_d = nullptr;     // 2 x creg[4] / 32
  int32_t* d_citem_t = nullptr;
  uint8_t* d_cactive = nullptr;
  int* d_ccount = nullptr;         // 2 x 4
  bool tuned = false;
  bool tiles_win = true;  // the autotuner found the length-class tiles faster (or has not run)
  float tuned_ms = 0.f;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> knodes;
  // length-class tiles (WS_PLAN_TILES)
  std::vector<LenClass> classes;
  int32_t* d_class_sid = nullptr;
  int n_class_sid = 0;         // entries of d_class_sid (-1: padding columns)
  uint8_t* d_item_tiled = nullptr;
  size_t tile_elems = 0, tile_ws_bytes = 0, tile_st_bytes = 0;
  float* d_tiles = nullptr;        // 4 * tile_elems floats: x, w, lambda, z
  uint8_t* d_tile_st = nullptr;    // status of every class column
  void* d_tile_ws = nullptr;       // kTileStreams tile-kernel workspaces (the largest class's size each)
  cudaStream_t tstream[kTileStreams] = {};  // classes run concurrently, class i on stream i % kTileStreams
  cudaEvent_t tev[kTileStreams + 1] = {};  // fork + one join event per stream
  int graph_rc = 0, graph_warps = 0;
  bool graph_refine = false, graph_tiles = false;
  void* graph_ws = nullptr;    // workspace the graph was captured with
};

static size_t ragged_smem(int RC, int warps, int max_d) {
  return (size_t)warps * ragged_warp_rows(RC, max_d) * kPitch * sizeof(float);
}

static const void* ragged_kernel(int RC, int mode) {
  if (RC == 8) return mode == MODE_RAW ? (const void*)k_ragged<8, MODE_RAW> : (const void*)k_ragged<8, MODE_SMOOTH>;
  if (RC == 16) return mode == MODE_RAW ? (const void*)k_ragged<16, MODE_RAW> : (const void*)k_ragged<16, MODE_SMOOTH>;
  return mode == MODE_RAW ? (const void*)k_ragged<32, MODE_RAW> : (const void*)k_ragged<32, MODE_SMOOTH>;
}

static int ragged_grid(int RC, int warps, int items, int max_d, int* grid) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  const void* kern = ragged_kernel(RC, MODE_SMOOTH);
  const size_t smem = ragged_smem(RC, warps, max_d);
  if (smem > (size_t)di.smem_optin) return WS_EUNSUPPORTED;  // the candidate does not fit
  for (int m : {MODE_SMOOTH, MODE_RAW})
    if (cudaFuncSetAttribute(ragged_kernel(RC, m), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return set_error(WS_ECUDA, "ragged: cudaFuncSetAttribute");
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem) != cudaSuccess || occ < 1)
    return set_error(WS_ECUDA, "ragged: occupancy query");
  const int max_warps = di.sm_count * occ * warps;
  const int need = (items + warps - 1) / warps;
  *grid = std::min(di.sm_count * occ, std::max(1, need));
  (void)max_warps;
  return WS_OK;
}

constexpr int kRefineSteps = 3;     // FP32 refinement steps before the double-float re-solve
constexpr float kRefineTau = 3e-5f;  // settled: correction <= tau * max|z|
constexpr float kRefineTauDrop = 3e-6f;  // done (left out of later steps): correction <= tau_drop * max|z|
constexpr float kRefineTauCond = 1e-4f;  // first correction above tau_cond * max|z|: double-float at once

static void fill_refine_args(const ws_plan* pl, RaggedArgs& a) {
  a.resid = pl->d_resid;
  a.active = pl->d_active;
  a.conv = pl->d_conv;
  a.zmax = pl->d_zmax;
  a.prevc = pl->d_prevc;
  a.list64 = pl->d_list64;
  a.count64 = pl->d_count64 + a.band;
  a.ck64 = pl->d_ck64;
  a.d_of = pl->d_dof;
  a.tau = kRefineTau;
  a.tau_drop = kRefineTauDrop;
  a.tau_cond = kRefineTauCond;
}

// The items a launch runs: the plan's own, or a regrouped set of a refinement step.
struct ItemSet {
  const int32_t* order;
  const int8_t* item_d;
  const int32_t* item_t;
  uint8_t* active;
  int n_items;
};

static int ragged_launch(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                         int band, cudaStream_t st, int mode = MODE_SMOOTH, bool refine = false,
                         bool tiles = false, const ItemSet* items = nullptr) {
  RaggedArgs a;
  memset(&a, 0, sizeof(a));
  a.item_tiled = tiles ? pl->d_item_tiled : nullptr;
  a.off = pl->rg.offsets;
  a.order = pl->d_order;
  a.item_d = pl->d_item_d;
  a.item_t = pl->d_item_t;
  a.n_items = pl->n_items;
  a.N = pl->N;
  a.B = pl->rg.n_bands;
  a.band = band;
  a.lam_scalar = pl->rg.lam_mode == WS_LAM_SCALAR;
  a.x = (const float*)x;
  a.w = (const float*)w;
  a.lam = (const float*)lam;
  a.z = (float*)z;
  a.status = status;
  a.ckpt = pl->d_ckpt;
  a.max_nch = (pl->max_t + pl->RC - 1) / pl->RC;
  a.counter = pl->d_counter + band;
  a.err = pl->d_err;
  if (refine) fill_refine_args(pl, a);
  if (items != nullptr) {
    a.order = items->order;
    a.item_d = items->item_d;
    a.item_t = items->item_t;
    a.active = items->active;
    a.n_items = items->n_items;
  }
  a.warp_rows = ragged_warp_rows(pl->RC, pl->max_d);
  const size_t smem = ragged_smem(pl->RC, pl->warps, pl->max_d);
  if (cudaMemsetAsync(a.counter, 0, sizeof(int), st) != cudaSuccess) return set_error(WS_ECUDA, "ragged: memset");
  const dim3 g(pl->grid), blk(pl->warps * 32);
  if (pl->RC == 8) {
    if (mode == MODE_RAW) k_ragged<8, MODE_RAW><<<g, blk, smem, st>>>(a); else k_ragged<8, MODE_SMOOTH><<<g, blk, smem, st>>>(a);
  } else if (pl->RC == 16) {
    if (mode == MODE_RAW) k_ragged<16, MODE_RAW><<<g, blk, smem, st>>>(a); else k_ragged<16, MODE_SMOOTH><<<g, blk, smem, st>>>(a);
  } else {
    if (mode == MODE_RAW) k_ragged<32, MODE_RAW><<<g, blk, smem, st>>>(a); else k_ragged<32, MODE_SMOOTH><<<g, blk, smem, st>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

// Refinement of a ragged solution z in place. Up to kRefineSteps FP32 steps
// (r = W x - Omega z with a double-word combination, z += Omega^{-1} r); an item drops out
// once all its series have settled. Series still unsettled after the last step are listed
// and solved again from scratch in double-float arithmetic. tile_step: the length classes'
// series had their first step on the class tiles (ragged_tiles); their settle test runs
// here and the first per-lane step leaves their items out.
static int ragged_refine(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, int band,
                         cudaStream_t st, bool tile_step = false) {
  RaggedArgs a;
  memset(&a, 0, sizeof(a));
  a.off = pl->rg.offsets;
  a.order = pl->d_order;
  a.item_d = pl->d_item_d;
  a.n_items = pl->n_items;
  a.N = pl->N;
  a.B = pl->rg.n_bands;
  a.band = band;
  a.lam_scalar = pl->rg.lam_mode == WS_LAM_SCALAR;
  a.x = (const float*)x;
  a.w = (const float*)w;
  a.lam = (const float*)lam;
  a.z = (float*)z;
  fill_refine_args(pl, a);
  if (cudaMemsetAsync(pl->d_active, 1, pl->n_items, st) != cudaSuccess ||
      cudaMemsetAsync(pl->d_prevc, 0, sizeof(float) * pl->rg.n_series, st) != cudaSuccess ||
      cudaMemsetAsync(a.count64, 0, sizeof(int), st) != cudaSuccess)
    return set_error(WS_ECUDA, "ragged: memset");
  if (tile_step && pl->n_class_sid > 0) {
    k_tile_settle<<<(pl->n_class_sid + 255) / 256, 256, 0, st>>>(a, pl->d_class_sid, pl->n_class_sid, pl->d_tcorr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged tile settle launch: %s", cudaGetErrorString(e));
  }
  ItemSet cur{pl->d_order, pl->d_item_d, pl->d_item_t, pl->d_active, pl->n_items};
  const int4 reg = make_int4(pl->creg[0], pl->creg[1], pl->creg[2], pl->creg[3]);
  const int nci = pl->creg[4] / 32;
  for (int k = 0; k < kRefineSteps; ++k) {
    a.order = cur.order;
    a.item_d = cur.item_d;
    a.item_t = cur.item_t;
    a.active = cur.active;
    a.n_items = cur.n_items;
    const bool skip_tiled = tile_step && k == 0;  // the plan's own items: d_item_tiled applies
    a.item_tiled = skip_tiled ? pl->d_item_tiled : nullptr;
    const int gi = (cur.n_items + 7) / 8;
    k_ragged_resid<<<gi, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged residual launch: %s", cudaGetErrorString(e));
    int rc = ragged_launch(pl, x, w, lam, z, nullptr, band, st, MODE_RAW, true, skip_tiled, &cur);
    if (rc != WS_OK) return rc;
    if (k + 1 == kRefineSteps || nci == 0) continue;
    // the next step runs the still unsettled series only, regrouped
    const int q = k & 1;
    ItemSet nxt{pl->d_corder + (size_t)q * pl->creg[4], pl->d_citem_d + (size_t)q * nci,
                pl->d_citem_t + (size_t)q * nci, pl->d_cactive + (size_t)q * nci, nci};
    int* cnt = pl->d_ccount + 4 * q;
    if (cudaMemsetAsync(cnt, 0, 4 * sizeof(int), st) != cudaSuccess) return set_error(WS_ECUDA, "ragged: memset");
    k_ragged_compact<<<gi, 256, 0, st>>>(a, const_cast<int32_t*>(nxt.order), cnt, reg);
    k_ragged_regroup<<<(nci + 7) / 8, 256, 0, st>>>(pl->rg.offsets, const_cast<int32_t*>(nxt.order), cnt, reg, nci,
                                                     const_cast<int8_t*>(nxt.item_d), const_cast<int32_t*>(nxt.item_t),
                                                     nxt.active);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged regroup launch: %s", cudaGetErrorString(e));
    cur = nxt;
  }
  a.order = cur.order;
  a.item_d = cur.item_d;
  a.item_t = cur.item_t;
  a.active = cur.active;
  a.n_items = cur.n_items;
  a.item_tiled = nullptr;
  const int gi = (cur.n_items + 7) / 8;
  k_ragged_collect<<<gi, 256, 0, st>>>(a);
  k_ragged64<<<pl->grid64, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged double-float re-solve launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

// The length classes: gather -> tile smoothing -> scatter, one class after another.
static int ragged_tiles(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                        bool refine, cudaStream_t st) {
  RaggedArgs a;
  memset(&a, 0, sizeof(a));
  a.off = pl->rg.offsets;
  a.N = pl->N;
  a.B = 1;
  a.lam_scalar = pl->rg.lam_mode == WS_LAM_SCALAR;
  a.x = (const float*)x;
  a.w = (const float*)w;
  a.lam = (const float*)lam;
  a.z = (float*)z;
  a.status = status;
  a.zmax = refine ? pl->d_zmax : nullptr;
  float* tx = pl->d_tiles;
  float* tw = tx + pl->tile_elems;
  float* tl = tw + pl->tile_elems;
  float* tz = tl + pl->tile_elems;
  float* tr = refine ? tz + pl->tile_elems : nullptr;  // residual of the refinement step
  size_t stoff = 0;
  // fork: the class streams wait for the work queued before on st (also under capture)
  if (cudaEventRecord(pl->tev[0], st) != cudaSuccess) return set_error(WS_ECUDA, "ragged tiles: fork");
  for (int k = 0; k < kTileStreams; ++k)
    if (cudaStreamWaitEvent(pl->tstream[k], pl->tev[0], 0) != cudaSuccess) return set_error(WS_ECUDA, "ragged tiles: fork");
  int ci = 0;
  for (const LenClass& c : pl->classes) {
    const int k = ci++ % kTileStreams;
    cudaStream_t cs = pl->tstream[k];
    void* wsk = static_cast<char*>(pl->d_tile_ws) + (size_t)k * pl->tile_ws_bytes;
    const dim3 blk(32, 8), grd((unsigned)((c.Pc + 31) / 32), (unsigned)((c.Tc + 31) / 32));
    const int32_t* sids = pl->d_class_sid + c.sid_base;
    k_gather<<<grd, blk, 0, cs>>>(a, sids, c.Pc, c.Tc, tx + c.base, tw + c.base, tl + c.base);
    ws_problem P;
    memset(&P, 0, sizeof(P));
    P.n_series = c.Pc;
    P.T = c.Tc;
    P.d = c.d;
    P.n_bands = 1;
    P.layout = WS_LAYOUT_TILE;
    P.dtype = WS_F32;
    P.lam_mode = WS_LAM_PER_DAY;
    int rc = tile_smooth(P, tx + c.base, tw + c.base, tl + c.base, tz + c.base, pl->d_tile_st + stoff, wsk, cs);
    if (rc != WS_OK) return rc;
    k_scatter<<<grd, blk, 0, cs>>>(a, sids, c.Pc, c.Tc, tz + c.base, pl->d_tile_st + stoff);
    if (refine) {  // the first refinement step on the tile, then z and the correction sizes back
      rc = tile_refine(P, tx + c.base, tw + c.base, tl + c.base, tz + c.base, tr + c.base, wsk, cs);
      if (rc != WS_OK) return rc;
      k_scatter_refine<<<grd, blk, 0, cs>>>(a, sids, c.Pc, c.Tc, tz + c.base, pl->d_tcorr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(WS_ECUDA, "ragged tiles launch: %s", cudaGetErrorString(e));
    stoff += (size_t)c.Pc;
  }
  // join: st waits for every class stream
  for (int k = 0; k < kTileStreams; ++k) {
    if (cudaEventRecord(pl->tev[1 + k], pl->tstream[k]) != cudaSuccess ||
        cudaStreamWaitEvent(st, pl->tev[1 + k], 0) != cudaSuccess)
      return set_error(WS_ECUDA, "ragged tiles: join");
  }
  return WS_OK;
}

// Size of one length class's tile-kernel workspace (the largest class's, 256-byte multiple).
static int tile_ws_size(const ws_plan* pl, size_t* out) {
  size_t wsb = 0;
  for (const LenClass& c : pl->classes) {
    ws_problem P;
    memset(&P, 0, sizeof(P));
    P.n_series = c.Pc;
    P.T = c.Tc;
    P.d = c.d;
    P.n_bands = 1;
    P.layout = WS_LAYOUT_TILE;
    P.dtype = WS_F32;
    P.lam_mode = WS_LAM_PER_DAY;
    const size_t b = tile_workspace_bytes(P);
    if (b == 0) return WS_ECUDA;
    wsb = std::max(wsb, b);
  }
  *out = (wsb + 255) & ~(size_t)255;
  return WS_OK;
}

static size_t r256(size_t v) { return (v + 255) & ~(size_t)255; }

// Checkpoint bytes of the per-lane kernel in configuration (RC, warps).
static int ckpt_need(const ws_plan* pl, int RC, int warps, size_t* out) {
  int grid = 0;
  int rc = ragged_grid(RC, warps, pl->n_items, pl->max_d, &grid);
  if (rc != WS_OK) return rc;
  *out = (size_t)grid * warps * ((pl->max_t + RC - 1) / RC) * kFieldsMax * 32 * 4;
  return WS_OK;
}

static const int kCands[][2] = {{8, 8}, {8, 16}, {16, 4}, {16, 6}, {16, 8}, {16, 12}, {16, 16}, {32, 4}, {32, 8}};
constexpr int kNCands = sizeof(kCands) / sizeof(kCands[0]);

// Workspace layout of one execute: checkpoints (the largest candidate's when the autotuner
// is still to run), then the length-class tiles, then the refinement state.
struct PlanWs {
  size_t ckpt = 0, tiles = 0, tile_st = 0, tile_ws = 0, refine = 0, total = 0;
  size_t resid = 0, active = 0, conv = 0, zmax = 0, tcorr = 0, prevc = 0, list64 = 0, count64 = 0, ck64 = 0;
  size_t corder = 0, citem_d = 0, citem_t = 0, cactive = 0, ccount = 0;
};

static int plan_ws(const ws_plan* pl, uint32_t flags, PlanWs* L) {
  *L = PlanWs();
  size_t off = 0;
  size_t ck = 0;
  int rc = ckpt_need(pl, pl->RC, pl->warps, &ck);
  if (rc != WS_OK) return rc;
  if ((flags & WS_PLAN_AUTOTUNE) && !pl->tuned)
    for (int c = 0; c < kNCands; ++c) {
      size_t q = 0;
      rc = ckpt_need(pl, kCands[c][0], kCands[c][1], &q);
      if (rc == WS_EUNSUPPORTED) continue;
      if (rc != WS_OK) return rc;
      ck = std::max(ck, q);
    }
  L->ckpt = off;
  off += r256(ck);
  const bool tiles = (flags & WS_PLAN_TILES) && pl->rg.n_bands == 1 && !pl->classes.empty();
  if (tiles) {
    L->tiles = off;  // x, w, lambda, z (+ r of the refinement step) of every class
    off += r256(((flags & WS_PLAN_REFINE) ? 5 : 4) * pl->tile_elems * sizeof(float));
    L->tile_st = off;
    off += r256(std::max<size_t>(1, pl->tile_st_bytes));
    L->tile_ws = off;
    off += pl->tile_ws_bytes * kTileStreams;
  }
  if (flags & WS_PLAN_REFINE) {
    const size_t n = (size_t)std::max<int64_t>(1, pl->rg.n_series), ni = (size_t)std::max(1, pl->n_items);
    const size_t cs = (size_t)std::max(32, pl->creg[4]), cni = cs / 32;
    L->refine = off;
    L->resid = off;   off += r256(sizeof(float) * (size_t)std::max<int64_t>(1, pl->N));
    L->active = off;  off += r256(ni);
    L->conv = off;    off += r256(n);
    L->zmax = off;    off += r256(4 * n);
    L->tcorr = off;   off += r256(4 * n);
    L->prevc = off;   off += r256(4 * n);
    L->list64 = off;  off += r256(4 * n);
    L->count64 = off; off += r256(sizeof(int) * pl->rg.n_bands);
    L->ck64 = off;    off += r256((size_t)pl->grid64 * 128 * std::max(1, pl->max_t64) * pl->sf64 * sizeof(double));
    L->corder = off;  off += r256(2 * cs * 4);
    L->citem_d = off; off += r256(2 * cni);
    L->citem_t = off; off += r256(2 * cni * 4);
    L->cactive = off; off += r256(2 * cni);
    L->ccount = off;  off += r256(2 * 4 * sizeof(int));
  }
  L->total = std::max<size_t>(off, 256);
  return WS_OK;
}

// Point the plan's scratch views into `ws` laid out for `flags`.
static void bind_ws(ws_plan* pl, uint32_t flags, const PlanWs& L, void* ws) {
  char* b = static_cast<char*>(ws);
  pl->d_ckpt = reinterpret_cast<float*>(b + L.ckpt);
  const bool tiles = (flags & WS_PLAN_TILES) && pl->rg.n_bands == 1 && !pl->classes.empty();
  pl->d_tiles = tiles ? reinterpret_cast<float*>(b + L.tiles) : nullptr;
  pl->d_tile_st = tiles ? reinterpret_cast<uint8_t*>(b + L.tile_st) : nullptr;
  pl->d_tile_ws = tiles ? static_cast<void*>(b + L.tile_ws) : nullptr;
  const bool refine = (flags & WS_PLAN_REFINE) != 0;
  pl->d_resid = refine ? reinterpret_cast<float*>(b + L.resid) : nullptr;
  pl->d_active = refine ? reinterpret_cast<uint8_t*>(b + L.active) : nullptr;
  pl->d_conv = refine ? reinterpret_cast<uint8_t*>(b + L.conv) : nullptr;
  pl->d_zmax = refine ? reinterpret_cast<float*>(b + L.zmax) : nullptr;
  pl->d_tcorr = refine ? reinterpret_cast<float*>(b + L.tcorr) : nullptr;
  pl->d_prevc = refine ? reinterpret_cast<float*>(b + L.prevc) : nullptr;
  pl->d_list64 = refine ? reinterpret_cast<int32_t*>(b + L.list64) : nullptr;
  pl->d_count64 = refine ? reinterpret_cast<int*>(b + L.count64) : nullptr;
  pl->d_ck64 = refine ? reinterpret_cast<double*>(b + L.ck64) : nullptr;
  pl->d_corder = refine ? reinterpret_cast<int32_t*>(b + L.corder) : nullptr;
  pl->d_citem_d = refine ? reinterpret_cast<int8_t*>(b + L.citem_d) : nullptr;
  pl->d_citem_t = refine ? reinterpret_cast<int32_t*>(b + L.citem_t) : nullptr;
  pl->d_cactive = refine ? reinterpret_cast<uint8_t*>(b + L.cactive) : nullptr;
  pl->d_ccount = refine ? reinterpret_cast<int*>(b + L.ccount) : nullptr;
  pl->ws_base = ws;
  pl->ws_flags = flags;
}

static int ragged_config(ws_plan* pl, int RC, int warps) {
  pl->RC = RC;
  pl->warps = warps;
  return ragged_grid(RC, warps, pl->n_items, pl->max_d, &pl->grid);
}

extern "C" int ws_plan_create(const ws_ragged* rg, ws_plan** out, void* stream) {
  if (out == nullptr || rg == nullptr) return set_error(WS_EINVAL, "plan: NULL argument");
  *out = nullptr;
  if (rg->n_series < 0 || rg->n_series > 0x7fffffffLL) return set_error(WS_EINVAL, "plan: n_series out of range");
  if (rg->dtype != WS_F32) return set_error(WS_EUNSUPPORTED, "ragged path: FP32 only");
  if (rg->n_bands < 1) return set_error(WS_EINVAL, "plan: n_bands must be >= 1");
  if (rg->lam_mode != WS_LAM_PER_DAY && rg->lam_mode != WS_LAM_SCALAR) return set_error(WS_EINVAL, "plan: lam_mode");
  if (rg->offsets == nullptr) return set_error(WS_EINVAL, "plan: offsets is NULL");
  if (rg->d_per_series == nullptr && (rg->d_uniform < 1 || rg->d_uniform > 4))
    return set_error(WS_EINVAL, "plan: d_uniform must be 1..4 when d_per_series is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = (int)rg->n_series;
  std::vector<int64_t> off(n + 1);
  std::vector<int8_t> dd(n, (int8_t)rg->d_uniform);
  if (cudaMemcpyAsync(off.data(), rg->offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return set_error(WS_ECUDA, "plan: reading offsets");
  if (rg->d_per_series && n > 0 &&
      cudaMemcpyAsync(dd.data(), rg->d_per_series, n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return set_error(WS_ECUDA, "plan: reading orders");
  if (cudaStreamSynchronize(st) != cudaSuccess) return set_error(WS_ECUDA, "plan: synchronise");
  if (off[0] != 0) return set_error(WS_EINVAL, "plan: offsets[0] must be 0");
  for (int i = 0; i < n; ++i) {
    if (off[i + 1] < off[i]) return set_error(WS_EINVAL, "plan: offsets not non-decreasing at %d", i);
    if (off[i + 1] - off[i] > 0x7fffffff) return set_error(WS_EINVAL, "plan: series %d too long", i);
    if (dd[i] < 1 || dd[i] > 4) return set_error(WS_EINVAL, "plan: order of series %d is %d (1..4)", i, (int)dd[i]);
  }
  // sort by (order, length descending); cut into items of 32
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (dd[a] != dd[b]) return dd[a] < dd[b];
    return off[a + 1] - off[a] > off[b + 1] - off[b];
  });
  struct Item {
    int first, count, d;
    int64_t tmax;
  };
  std::vector<Item> items;
  for (int i = 0; i < n;) {
    int j = i;
    while (j < n && j - i < 32 && dd[idx[j]] == dd[idx[i]]) ++j;
    items.push_back({i, j - i, dd[idx[i]], off[idx[i] + 1] - off[idx[i]]});
    i = j;
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.tmax > b.tmax; });
  ws_plan* pl = new ws_plan();
  pl->rg = *rg;
  pl->n_items = (int)items.size();
  pl->N = off[n];
  std::vector<int32_t> order((size_t)pl->n_items * 32, -1), itt(pl->n_items);
  std::vector<int8_t> idd(pl->n_items);
  for (int k = 0; k < pl->n_items; ++k) {
    for (int l = 0; l < items[k].count; ++l) order[(size_t)k * 32 + l] = idx[items[k].first + l];
    idd[k] = (int8_t)items[k].d;
    itt[k] = (int32_t)items[k].tmax;
    pl->max_t = std::max(pl->max_t, itt[k]);
    pl->max_d = std::max(pl->max_d, (int)idd[k]);
  }
  const size_t ni = std::max(1, pl->n_items);
  bool okm = cudaMalloc(&pl->d_order, ni * 32 * 4) == cudaSuccess && cudaMalloc(&pl->d_item_d, ni) == cudaSuccess &&
             cudaMalloc(&pl->d_item_t, ni * 4) == cudaSuccess &&
             cudaMalloc(&pl->d_counter, sizeof(int) * rg->n_bands) == cudaSuccess &&
             cudaMalloc(&pl->d_err, 4) == cudaSuccess && cudaMalloc(&pl->d_dof, std::max(1, n)) == cudaSuccess;
  if (!okm) {
    ws_plan_destroy(pl);
    return set_error(WS_ECUDA, "plan: device allocation");
  }
  if (pl->n_items > 0) {
    cudaMemcpy(pl->d_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(pl->d_item_d, idd.data(), idd.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(pl->d_item_t, itt.data(), itt.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(pl->d_dof, dd.data(), n, cudaMemcpyHostToDevice);
  }
  for (const Item& it : items) {
    pl->max_t64 = std::max(pl->max_t64, (int)it.tmax);
    pl->sf64 = std::max(pl->sf64, 1 + it.d);
  }
  {
    int nd[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) ++nd[dd[i] - 1];
    for (int q = 0; q < 4; ++q) pl->creg[q + 1] = pl->creg[q] + (nd[q] + 31) / 32 * 32;
  }
  // Length classes for WS_PLAN_TILES (one band, FP32): the series of items whose shortest
  // series has at least kTileMinT days, grouped by (order, length rounded up to kClassRound)
  if (rg->n_bands == 1 && pl->n_items > 0) {
    std::vector<uint8_t> tiled(pl->n_items, 0);
    std::vector<std::vector<int>> byk;  // per (d, Tc) key
    std::vector<std::pair<int, int>> keys;
    std::map<int64_t, int> keymap;
    for (int k = 0; k < pl->n_items; ++k) {
      const Item& it = items[k];
      const int sid_last = idx[it.first + it.count - 1];
      if (off[sid_last + 1] - off[sid_last] < kTileMinT) continue;
      tiled[k] = 1;
      for (int l = 0; l < it.count; ++l) {
        const int sid = idx[it.first + l];
        const int T = (int)(off[sid + 1] - off[sid]);
        const int Tc = (T + kClassRound - 1) / kClassRound * kClassRound;
        const int64_t kk = (int64_t)it.d * (1LL << 40) + Tc;
        auto fk = keymap.find(kk);
        int key = fk == keymap.end() ? -1 : fk->second;
        if (key < 0) {
          keymap[kk] = (int)keys.size();
          key = (int)keys.size();
          keys.push_back({it.d, Tc});
          byk.emplace_back();
        }
        byk[key].push_back(sid);
      }
    }
    std::vector<int32_t> csid;
    size_t base = 0, st = 0;
    for (size_t q = 0; q < keys.size(); ++q) {
      LenClass c;
      c.d = keys[q].first;
      c.Tc = keys[q].second;
      c.Pc = ((int)byk[q].size() + 3) / 4 * 4;  // a multiple of 4 columns: 16-byte rows for TMA
      c.base = base;
      c.sid_base = (int)csid.size();
      for (int sid : byk[q]) csid.push_back(sid);
      for (int e = (int)byk[q].size(); e < c.Pc; ++e) csid.push_back(-1);
      base += (size_t)c.Tc * c.Pc;
      st += (size_t)c.Pc;
      pl->classes.push_back(c);
    }
    pl->tile_elems = base;
    pl->tile_st_bytes = st;
    pl->n_class_sid = (int)csid.size();
    if (!csid.empty()) {
      bool ok = cudaMalloc(&pl->d_class_sid, csid.size() * 4) == cudaSuccess &&
                cudaMalloc(&pl->d_item_tiled, pl->n_items) == cudaSuccess;
      if (!ok) {
        ws_plan_destroy(pl);
        return set_error(WS_ECUDA, "plan: class tables");
      }
      cudaMemcpy(pl->d_class_sid, csid.data(), csid.size() * 4, cudaMemcpyHostToDevice);
      cudaMemcpy(pl->d_item_tiled, tiled.data(), pl->n_items, cudaMemcpyHostToDevice);
    }
  }
  cudaMemset(pl->d_err, 0, 4);
  int rc = ragged_config(pl, 16, 8);
  DeviceInfo di;
  if (rc == WS_OK) rc = device_info(di);
  if (rc == WS_OK) {
    pl->grid64 = di.sm_count * kHPBlocksPerSM;
    if (!pl->classes.empty()) {  // the length classes' streams and fork/join events
      rc = tile_ws_size(pl, &pl->tile_ws_bytes);
      bool ok = rc == WS_OK;
      for (int k = 0; ok && k < kTileStreams; ++k)
        ok = cudaStreamCreateWithFlags(&pl->tstream[k], cudaStreamNonBlocking) == cudaSuccess;
      for (int k = 0; ok && k <= kTileStreams; ++k)
        ok = cudaEventCreateWithFlags(&pl->tev[k], cudaEventDisableTiming) == cudaSuccess;
      if (!ok && rc == WS_OK) rc = set_error(WS_ECUDA, "plan: length-class streams");
    }
  }
  if (rc != WS_OK) {
    ws_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return WS_OK;
}

static int ragged_tiles(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                        bool refine, cudaStream_t st);

// Autotuner: time every (chunk, warps per CTA) candidate on the plan's own data, keep the
// fastest; with try_tiles, time the length-class tiles (short series per lane) against it.
static int ragged_autotune(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, bool try_tiles,
                           cudaStream_t st) {
  const auto& cands = kCands;
  constexpr int nc = kNCands;
  float best = 1e30f;
  int bi = -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int c = 0; c < nc; ++c) {
    int rc = ragged_config(pl, cands[c][0], cands[c][1]);
    if (rc == WS_EUNSUPPORTED) continue;  // more shared memory than a CTA may have
    if (rc != WS_OK) return rc;
    if ((rc = ragged_launch(pl, x, w, lam, z, nullptr, 0, st)) != WS_OK) return rc;  // warm-up
    cudaEventRecord(e0, st);
    if ((rc = ragged_launch(pl, x, w, lam, z, nullptr, 0, st)) != WS_OK) return rc;
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bi = c;
    }
  }
  if (bi < 0) return set_error(WS_EUNSUPPORTED, "ragged autotune: no configuration fits");
  int rc = ragged_config(pl, cands[bi][0], cands[bi][1]);
  if (rc != WS_OK) return rc;
  pl->tuned = true;
  pl->tuned_ms = best;
  if (try_tiles) {
    float ms = 0.f;
    for (int it = 0; it < 2; ++it) {  // warm-up, then timed
      cudaEventRecord(e0, st);
      if ((rc = ragged_launch(pl, x, w, lam, z, nullptr, 0, st, MODE_SMOOTH, false, true)) != WS_OK) return rc;
      if ((rc = ragged_tiles(pl, x, w, lam, z, nullptr, false, st)) != WS_OK) return rc;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    pl->tiles_win = ms < best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return WS_OK;
}

extern "C" size_t ws_plan_workspace_size(const ws_plan* pl, uint32_t flags) {
  if (pl == nullptr) {
    set_error(WS_EINVAL, "plan is NULL");
    return 0;
  }
  PlanWs L;
  if (plan_ws(pl, flags, &L) != WS_OK) return 0;
  return L.total;
}

extern "C" int ws_plan_execute(ws_plan* pl, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                               uint32_t flags, void* workspace, size_t ws_bytes, void* stream) {
  if (pl == nullptr) return set_error(WS_EINVAL, "plan is NULL");
  if (flags & ~(WS_PLAN_AUTOTUNE | WS_PLAN_GRAPH | WS_PLAN_REFINE | WS_PLAN_TILES))
    return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  const bool refine = (flags & WS_PLAN_REFINE) != 0;
  const bool tiles_req = (flags & WS_PLAN_TILES) != 0 && pl->rg.n_bands == 1 && !pl->classes.empty();
  if (pl->n_items == 0) return WS_OK;
  int rc;
  PlanWs L;
  if ((rc = plan_ws(pl, flags, &L)) != WS_OK) return rc;
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < L.total) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, L.total);
  bind_ws(pl, flags, L, workspace);
  // with no days at all (every series empty) only the status codes are written
  if (pl->N > 0 && (!x || !w || !z)) return set_error(WS_EINVAL, "x, w and z must be non-NULL");
  if (!lam && (pl->N > 0 || pl->rg.lam_mode == WS_LAM_SCALAR)) return set_error(WS_EINVAL, "lam must be non-NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((flags & WS_PLAN_AUTOTUNE) && !pl->tuned && (rc = ragged_autotune(pl, x, w, lam, z, tiles_req, st)) != WS_OK)
    return rc;
  const bool tiles = tiles_req && pl->tiles_win;
  if (tiles)
    for (int k = 0; k < kTileStreams; ++k)
      if (cudaMemsetAsync(static_cast<char*>(pl->d_tile_ws) + (size_t)k * pl->tile_ws_bytes, 0, kHeaderBytes, st) !=
          cudaSuccess)
        return set_error(WS_ECUDA, "ragged: memset");
  if (!(flags & WS_PLAN_GRAPH) || pl->rg.n_bands > 1) {
    for (int b = 0; b < pl->rg.n_bands; ++b) {
      if (tiles && refine && (cudaMemsetAsync(pl->d_zmax, 0, sizeof(float) * pl->rg.n_series, st) != cudaSuccess ||
                              cudaMemsetAsync(pl->d_tcorr, 0, sizeof(float) * pl->rg.n_series, st) != cudaSuccess))
        return set_error(WS_ECUDA, "ragged: memset");
      if ((rc = ragged_launch(pl, x, w, lam, z, status, b, st, MODE_SMOOTH, refine, tiles)) != WS_OK) return rc;
      if (tiles && (rc = ragged_tiles(pl, x, w, lam, z, status, refine, st)) != WS_OK) return rc;
      if (refine && (rc = ragged_refine(pl, x, w, lam, z, b, st, tiles)) != WS_OK) return rc;
    }
    return WS_OK;
  }
  // CUDA graph: captured once per configuration, kernel arguments updated on each replay
  // (re-captured when the configuration or the workspace changes: the length classes' tile
  // kernels take tensor maps of workspace arrays)
  if (pl->exec == nullptr || pl->graph_rc != pl->RC || pl->graph_warps != pl->warps || pl->graph_refine != refine ||
      pl->graph_tiles != tiles || pl->graph_ws != workspace) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    pl->exec = nullptr;
    pl->graph = nullptr;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return set_error(WS_ECUDA, "graph stream");
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cs);
      return set_error(WS_ECUDA, "graph capture");
    }
    if (tiles && refine && (cudaMemsetAsync(pl->d_zmax, 0, sizeof(float) * pl->rg.n_series, cs) != cudaSuccess ||
                            cudaMemsetAsync(pl->d_tcorr, 0, sizeof(float) * pl->rg.n_series, cs) != cudaSuccess))
      rc = set_error(WS_ECUDA, "ragged: memset");
    else
      rc = ragged_launch(pl, x, w, lam, z, status, 0, cs, MODE_SMOOTH, refine, tiles);
    if (rc == WS_OK && tiles) rc = ragged_tiles(pl, x, w, lam, z, status, refine, cs);
    if (rc == WS_OK && refine) rc = ragged_refine(pl, x, w, lam, z, 0, cs, tiles);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != WS_OK || e != cudaSuccess) return set_error(WS_ECUDA, "graph capture failed");
    if (cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      return set_error(WS_ECUDA, "graph instantiate");
    }
    pl->graph = g;
    pl->graph_rc = pl->RC;
    pl->graph_warps = pl->warps;
    pl->graph_refine = refine;
    pl->graph_tiles = tiles;
    pl->graph_ws = workspace;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    pl->knodes.clear();
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      cudaGraphNodeGetType(nd, &t);
      if (t == cudaGraphNodeTypeKernel) pl->knodes.push_back(nd);
    }
  } else {
    // new buffers: the ragged kernels take RaggedArgs first (only its user buffers change; the
    // other parameters are kept); the tile kernels of the length classes read workspace
    // arrays only (the same workspace) and are left as captured
    for (auto nd : pl->knodes) {
      cudaKernelNodeParams kp;
      if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) return set_error(WS_ECUDA, "graph params");
      int nparams = 0;
      if (kp.func == (void*)k_gather) nparams = 7;
      else if (kp.func == (void*)k_scatter) nparams = 6;
      else if (kp.func == (void*)k_ragged_resid || kp.func == (void*)k_ragged_collect || kp.func == (void*)k_ragged64)
        nparams = 1;
      else
        for (int rcv : {8, 16, 32})
          for (int m : {MODE_SMOOTH, MODE_RAW})
            if (kp.func == ragged_kernel(rcv, m)) nparams = 1;
      if (nparams == 0) continue;
      RaggedArgs na = *static_cast<RaggedArgs*>(kp.kernelParams[0]);
      na.x = (const float*)x;
      na.w = (const float*)w;
      na.lam = (const float*)lam;
      na.z = (float*)z;
      na.status = status;  // read by the smoothing and scatter launches only
      void* args[8] = {&na};
      for (int i = 1; i < nparams; ++i) args[i] = kp.kernelParams[i];
      kp.kernelParams = args;
      if (cudaGraphExecKernelNodeSetParams(pl->exec, nd, &kp) != cudaSuccess)
        return set_error(WS_ECUDA, "graph update");
    }
  }
  if (cudaGraphLaunch(pl->exec, st) != cudaSuccess) return set_error(WS_ECUDA, "graph launch");
  return WS_OK;
}

extern "C" int ws_plan_info(const ws_plan* pl, ws_plan_stats* out) {
  if (pl == nullptr || out == nullptr) return set_error(WS_EINVAL, "NULL argument");
  out->n_items = pl->n_items;
  out->chunk_days = pl->RC;
  out->warps_per_cta = pl->warps;
  out->grid = pl->grid;
  out->tuned = pl->tuned ? 1 : 0;
  out->tuned_ms = pl->tuned_ms;
  out->graph = pl->exec != nullptr ? 1 : 0;
  out->hp_series = 0;
  out->tiles = pl->tiles_win ? 1 : 0;
  if (pl->d_count64 != nullptr && cudaMemcpy(&out->hp_series, pl->d_count64, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(WS_ECUDA, "plan info: reading the re-solve count");
  return WS_OK;
}

extern "C" void ws_plan_destroy(ws_plan* pl) {
  if (pl == nullptr) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  cudaFree(pl->d_order);
  cudaFree(pl->d_item_d);
  cudaFree(pl->d_item_t);
  cudaFree(pl->d_class_sid);
  cudaFree(pl->d_item_tiled);
  for (int k = 0; k < kTileStreams; ++k)
    if (pl->tstream[k]) cudaStreamDestroy(pl->tstream[k]);
  for (int k = 0; k <= kTileStreams; ++k)
    if (pl->tev[k]) cudaEventDestroy(pl->tev[k]);
  cudaFree(pl->d_counter);
  cudaFree(pl->d_err);
  cudaFree(pl->d_dof);
  delete pl;
}
