// Double-float re-solve of the adjoint (Section 2.3, Eqs. 4-5) for the series whose refined
// FP32 adjoint did not settle.
//
// On sparse series (a handful of valid days, lambda ~ 1e5) Omega is nearly singular along
// the polynomials of degree < d that D annihilates: g = Omega^{-1} gz carries a large
// component in that direction, and D g, which dL/dlambda_k = -sum_b (D g_b)_k (D z_b)_k
// needs, is many orders of magnitude smaller than g. FP32 then cannot resolve D g: even the
// exact g rounded to FP32 leaves rounding noise that D^d turns into an error larger than D g,
// and with eps32 * cond(Omega) near or above 1 the refinement step does not converge.
//
// The correction pass of the refined adjoint (tile kernel, MODE_ADJ with accumulation)
// tracks per series the largest correction |delta|, |g| and |D^d g| and lists the series
// for which the error left after the step, estimated as |delta|^2 / |g| (one step of a
// contracting refinement squares the relative error) plus g's own FP32 rounding, could reach
// 1e-4 of |D^d g| once differenced (a factor 2^d). This kernel re-solves each listed
// series in double-float arithmetic (dwf: about 48 significant bits, FP32 operations only;
// B300's FP64 rate is a small fraction of its FP32 rate): one thread per series, the same
// rotation factor and two-pass recurrence (checkpoints every kDfChunk days in the thread's
// slot, the chunk's recomputed (yhat, rho) in local arrays), then gx = W g (or g) and
// dL/dlambda from nested first differences of g and z in double-float, summed over the bands
// in a per-day double-float accumulator. It overwrites gx and glam of the listed series.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_sweep.cuh"

namespace ws {

constexpr int kDfChunk = 64;      // days per checkpoint
constexpr int kDfThreads = 64;    // threads per CTA
constexpr int kDfSlotsMax = 2048; // series re-solved at the same time (one slot each)
constexpr int kDfFieldsMax = 4 * 5 + 4;  // checkpoint words of Sweep<dwf, 4, 1>

struct AdjDfArgs {
  int T, P, B, nch;
  int lam_scalar, grad_loglam, raw_g;
  const float* gz;
  const float* w;
  const float* lam;
  const float* z;
  float* gx;
  float* glam;
  const int* list;
  const unsigned* count;
  char* slots;
  size_t slot_bytes;
  int n_slots;
};

template <int D>
__device__ void adj_df_series(const AdjDfArgs& a, int p, dwf* ck, dwf* acc) {
  using HP = dwf;
  using SW = Sweep<HP, D, 1>;
  constexpr int kFF = SW::kFactorFields;
  constexpr int kF = kFF + D;
  constexpr int DT = D > 1 ? D - 1 : 1;
  const int T = a.T, P = a.P;
  const size_t tstride = (size_t)a.B * P;
  const HP zero(0.f);
  auto w_at = [&](int i) -> HP { return HP(i < T ? a.w[(size_t)i * P + p] : 0.f); };
  auto lam_at = [&](int i) -> HP { return HP(a.lam_scalar ? a.lam[p] : a.lam[(size_t)i * P + p]); };
  const bool want_glam = a.glam != nullptr;
  if (want_glam)
    for (int i = 0; i < T; ++i) acc[i] = zero;
  HP yk[kDfChunk], rk[kDfChunk][D];
  for (int b = 0; b < a.B; ++b) {
    const float* gin = a.gz + (size_t)b * P + p;   // element (t, b, p) at gin[t * tstride]
    const float* zin = a.z + (size_t)b * P + p;
    float* gout = a.gx != nullptr ? a.gx + (size_t)b * P + p : nullptr;
    SW s;
    s.reset();
    for (int m = 0; m < D && m < T; ++m) s.init_weight(m, w_at(m));
    for (int c = 0; c < a.nch; ++c) {
      s.save_factor(ck + (size_t)c * kF, 1);
      s.save_y(ck + (size_t)c * kF + kFF, 1);
      const int i1 = min(T, (c + 1) * kDfChunk);
      for (int i = c * kDfChunk; i < i1; ++i) {
        HP bv[1] = {HP(gin[(size_t)i * tstride])};
        HP rho[D], yh[1], invD;
        const bool hr = i < T - D;
        s.factor_step(hr, hr ? lam_at(i) : zero, w_at(i + D), rho, invD);
        s.subst_step(rho, invD, bv, yh);
      }
    }
    // back substitution; zc[j] = g_{t+1+j}. Difference triangles at day t+1 for the nested
    // first differences (Delta^q v_t = Delta^{q-1} v_{t+1} - Delta^{q-1} v_t):
    // gt[q-1] = Delta^q g_{t+1}, zt[q-1] = Delta^q z_{t+1} (q = 1..D-1), gn/zn = g/z at t+1.
    HP zc[D], gt[DT], zt[DT], gn = zero, zn = zero;
#pragma unroll
    for (int j = 0; j < D; ++j) zc[j] = zero;
#pragma unroll
    for (int q = 0; q < DT; ++q) gt[q] = zt[q] = zero;
    for (int c = a.nch - 1; c >= 0; --c) {
      s.load_factor(ck + (size_t)c * kF, 1);
      s.load_y(ck + (size_t)c * kF + kFF, 1);
      const int i0 = c * kDfChunk, nd = min(kDfChunk, T - i0);
      for (int k = 0; k < nd; ++k) {
        const int i = i0 + k;
        HP bv[1] = {HP(gin[(size_t)i * tstride])};
        HP rho[D], yh[1], invD;
        const bool hr = i < T - D;
        s.factor_step(hr, hr ? lam_at(i) : zero, w_at(i + D), rho, invD);
        s.subst_step(rho, invD, bv, yh);
        yk[k] = yh[0];
#pragma unroll
        for (int j = 0; j < D; ++j) rk[k][j] = rho[j];
      }
      for (int k = nd - 1; k >= 0; --k) {
        const int i = i0 + k;
        HP g = yk[k];
#pragma unroll
        for (int j = 1; j <= D; ++j) g = fma(-rk[k][j - 1], zc[j - 1], g);
#pragma unroll
        for (int j = D - 1; j > 0; --j) zc[j] = zc[j - 1];
        zc[0] = g;
        if (gout != nullptr) {
          const float wi = a.w[(size_t)i * P + p];
          gout[(size_t)i * tstride] = a.raw_g ? g.to_float() : (HP(wi) * g).to_float();
        }
        if (want_glam) {
          const HP zv(zin[(size_t)i * tstride]);
          HP cg = g, cz = zv, pg = gn, pz = zn;
          gn = g;
          zn = zv;
#pragma unroll
          for (int q = 1; q <= D; ++q) {
            const HP ng = pg - cg, nz = pz - cz;
            if (q < D) {
              pg = gt[q - 1];
              pz = zt[q - 1];
              gt[q - 1] = ng;
              zt[q - 1] = nz;
            }
            cg = ng;
            cz = nz;
          }
          if (i < T - D) acc[i] = acc[i] + cg * cz;
        }
      }
    }
  }
  if (!want_glam) return;
  if (a.lam_scalar) {
    HP sum = zero;
    for (int i = 0; i < T - D; ++i) sum = sum + acc[i];
    HP v = -sum;
    if (a.grad_loglam) v = v * HP(a.lam[p]);
    a.glam[p] = v.to_float();
  } else {
    for (int i = 0; i < T; ++i) {
      float v = 0.f;
      if (i < T - D) {
        HP q = -acc[i];
        if (a.grad_loglam) q = q * HP(a.lam[(size_t)i * P + p]);
        v = q.to_float();
      }
      a.glam[(size_t)i * P + p] = v;
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kDfThreads) k_adj_df(const AdjDfArgs a) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= a.n_slots) return;
  char* slot = a.slots + (size_t)gt * a.slot_bytes;
  dwf* ck = reinterpret_cast<dwf*>(slot);
  dwf* acc = ck + (size_t)a.nch * kDfFieldsMax;
  const int n = (int)*a.count;
  for (int j = gt; j < n; j += a.n_slots) adj_df_series<D>(a, a.list[j], ck, acc);
}

static size_t r256(size_t v) { return (v + 255) & ~(size_t)255; }

static int df_slots(const ws_problem& pb) {
  return (int)(pb.n_series < kDfSlotsMax ? pb.n_series : kDfSlotsMax);
}

static size_t df_slot_bytes(const ws_problem& pb) {
  const size_t nch = ((size_t)pb.T + kDfChunk - 1) / kDfChunk;
  return r256((nch * kDfFieldsMax + (size_t)pb.T) * sizeof(dwf));
}

// Scratch of the re-solve: per-series marks, the list count, the list, the slots.
size_t adj_df_bytes(const ws_problem& pb) {
  if (pb.dtype != WS_F32 || pb.n_series == 0 || pb.T == 0) return 0;
  return r256((size_t)pb.n_series * 4) + 256 + r256((size_t)pb.n_series * 4) + (size_t)df_slots(pb) * df_slot_bytes(pb);
}

void adj_df_layout(const ws_problem& pb, void* base, unsigned** mark, unsigned** count, int** list, char** slots) {
  char* p = static_cast<char*>(base);
  *mark = reinterpret_cast<unsigned*>(p);
  p += r256((size_t)pb.n_series * 4);
  *count = reinterpret_cast<unsigned*>(p);
  p += 256;
  *list = reinterpret_cast<int*>(p);
  p += r256((size_t)pb.n_series * 4);
  *slots = p;
}

int launch_adj_df(const ws_problem& pb, const void* gz, const void* w, const void* lam, const void* z, void* gx,
                  void* glam, int adj_flags, void* base, cudaStream_t st) {
  AdjDfArgs a;
  a.T = pb.T;
  a.P = (int)pb.n_series;
  a.B = pb.n_bands;
  a.nch = (pb.T + kDfChunk - 1) / kDfChunk;
  a.lam_scalar = pb.lam_mode == WS_LAM_SCALAR;
  a.grad_loglam = adj_flags & 1;
  a.raw_g = (adj_flags >> 1) & 1;
  a.gz = static_cast<const float*>(gz);
  a.w = static_cast<const float*>(w);
  a.lam = static_cast<const float*>(lam);
  a.z = static_cast<const float*>(z);
  a.gx = static_cast<float*>(gx);
  a.glam = static_cast<float*>(glam);
  unsigned* mark = nullptr;
  unsigned* count = nullptr;
  int* list = nullptr;
  char* slots = nullptr;
  adj_df_layout(pb, base, &mark, &count, &list, &slots);
  a.list = list;
  a.count = count;
  a.slots = slots;
  a.slot_bytes = df_slot_bytes(pb);
  a.n_slots = df_slots(pb);
  const int grid = (a.n_slots + kDfThreads - 1) / kDfThreads;
  switch (pb.d) {
    case 1: k_adj_df<1><<<grid, kDfThreads, 0, st>>>(a); break;
    case 2: k_adj_df<2><<<grid, kDfThreads, 0, st>>>(a); break;
    case 3: k_adj_df<3><<<grid, kDfThreads, 0, st>>>(a); break;
    default: k_adj_df<4><<<grid, kDfThreads, 0, st>>>(a); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "adjoint re-solve launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

}  // namespace ws
