// Partitioned parallel-in-time solve for few long series (Section 2.3's cost argument: the
// one-series-per-thread recurrence leaves most of the GPU idle when only a few series are
// smoothed; here each series is cut into blocks solved at the same time).
//
// z = Omega^{-1} W x (Eq. 3) with Omega = W + D^T Lambda D banded (bandwidth d) and SPD. Days
// are cut into K domains of m days; the last d days of every domain but the last are a
// separator S_j, the rest of domain j its interior I_j. A row of Omega couples days at most
// d apart, and interiors are at least d + 1 days apart, so interiors couple only through
// the separators on either side (m >= 2d keeps separators from touching each other):
//   Omega = [Omega_II  Omega_IS; Omega_SI  Omega_SS],  Omega_II block diagonal.
// Eliminating the interiors leaves the Schur complement on the separators,
//   S = Omega_SS - Omega_SI Omega_II^{-1} Omega_IS,   S z_S = b_S - Omega_SI Omega_II^{-1} b_I,
// block tridiagonal with d x d blocks; then z_I = Omega_II^{-1} (b_I - Omega_IS z_S).
// (The SPIKE / substructuring decomposition of a banded SPD system.)
//
// Kernels (all arithmetic in H: double-float hi + lo FP32 pairs for FP32 data, about 48
// bits, since B300's FP64 rate is a small fraction of its FP32 rate; FP64 for FP64 data):
//   k_part_block   one thread per (series, domain): LDL^T of the interior band (assembled
//                  from w and lambda, Eq. 3), solves with the 2d coupling columns E_L =
//                  Omega_{I_j, S_(j-1)} and E_R = Omega_{I_j, S_j}, and writes the Schur pieces
//                  E^T Omega_II^{-1} E (only the first and last d rows of E are nonzero) and
//                  the interior factor;
//   k_part_rhs     one thread per (series, domain, band): E^T Omega_II^{-1} b with the stored
//                  factor;
//   k_part_reduce  one thread per series: status codes, then block LDL^T of S;
//   k_part_rsolve  one thread per (series, band): block forward / back substitution on S,
//                  z on the separator days;
//   k_part_finish  one thread per (series, domain, band): z_I = Omega_II^{-1} (b_I -
//                  E_L z_S(j-1) - E_R z_S(j)) with the stored factor; non-finite outputs flagged.
// Scratch lives in the caller's workspace; slot-major layouts ([field][slot], slot =
// domain * P + series) keep a warp's accesses contiguous.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_df.cuh"
#include "ws_internal.h"
#include "ws_sweep.cuh"

namespace ws {

constexpr int kPartMaxM = 64;    // domain length bound (interior <= kPartMaxM days)
constexpr int kPartThreads = 64;

// H arithmetic: conversions and the reciprocal.
template <typename H>
__device__ __forceinline__ H h_of(float v);
template <>
__device__ __forceinline__ dwf h_of<dwf>(float v) { return dwf(v); }
template <>
__device__ __forceinline__ double h_of<double>(float v) { return (double)v; }
template <typename H>
__device__ __forceinline__ H h_ofd(double v);
template <>
__device__ __forceinline__ dwf h_ofd<dwf>(double v) {
  const float hi = (float)v;
  return dwf(hi, (float)(v - (double)hi));
}
template <>
__device__ __forceinline__ double h_ofd<double>(double v) { return v; }
// 1/x for x > 0: FP32 reciprocal, then one Newton step r + r (1 - x r) in double-float.
__device__ __forceinline__ dwf h_inv(dwf x) {
  const float r0 = 1.0f / x.hi;
  const dwf e = dwf(1.0f) - x * dwf(r0);
  return dwf(r0) + dwf(r0) * e;
}
__device__ __forceinline__ double h_inv(double x) { return 1.0 / x; }
__device__ __forceinline__ float h_f(dwf v) { return v.to_float(); }
__device__ __forceinline__ float h_f(double v) { return (float)v; }
__device__ __forceinline__ double h_d(dwf v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ double h_d(double v) { return v; }
__device__ __forceinline__ bool h_pos(dwf v) { return v.hi > 0.f; }
__device__ __forceinline__ bool h_pos(double v) { return v > 0.0; }

struct PartArgs {
  int T, P, B, K, m, lam_scalar;
  const void* x;
  const void* w;
  const void* lam;
  void* z;
  uint8_t* status;
  // scratch
  void* fac;      // [i * (d + 1) + q][slot]: interior LDL^T (q = 0: D, q >= 1: L[i][i - q])
  void* gl;       // [a * d + b][slot] (FP64): -(E_L^T Omega_II^{-1} E_L)
  void* gr;       // Omega_(S_j S_j) - E_R^T Omega_II^{-1} E_R
  void* gc;       // -(E_L^T Omega_II^{-1} E_R): coupling S_(j-1) -> S_j
  void* hl;       // [a * B + b][slot]: E_L^T Omega_II^{-1} b
  void* hr;       // b_(S_j) - E_R^T Omega_II^{-1} b
  void* rl;       // [(j * d + a) * d + b][p]: unit lower factor of S's diagonal block j
  void* rd;       // [j * d + a][p]: pivots of S's diagonal block j
  void* rc;       // [(j * d + a) * d + b][p]: L_(j+1, j) (block j+1, rows of S_(j+1))
  void* zs;       // [((j * d + a) * B + b)][p]: z on the separator days
  uint32_t* flags;  // per series: bit 0 a non-positive pivot, bit 1 a non-finite output,
                    // bit 2 an invalid weight or lambda
  int32_t* npos;    // per series: positive weights
  uint8_t* code;    // per series: status before the non-finite check
};

template <typename F>
__device__ __forceinline__ double ldf(const void* p, size_t i) {
  return (double)static_cast<const F*>(p)[i];
}

// Omega[t][t + r] (0 <= r <= d) from its definition (Eq. 3): w_t [r = 0] + sum over the
// difference rows k covering both days of lambda_k c_(t-k) c_(t+r-k).
template <typename F, typename H, int D>
__device__ H omega_entry(const PartArgs& a, int p, int t, int r) {
  H v = h_of<H>(0.f);
  if (r == 0) {
    if constexpr (sizeof(F) == 8)
      v = h_ofd<H>(static_cast<const double*>(a.w)[(size_t)t * a.P + p]);
    else
      v = h_of<H>(static_cast<const float*>(a.w)[(size_t)t * a.P + p]);
  }
  const int k0 = max(0, t + r - D), k1 = min(t, a.T - D - 1);
  for (int k = k0; k <= k1; ++k) {
    H lk;
    if constexpr (sizeof(F) == 8)
      lk = h_ofd<H>(a.lam_scalar ? static_cast<const double*>(a.lam)[p] : static_cast<const double*>(a.lam)[(size_t)k * a.P + p]);
    else
      lk = h_of<H>(a.lam_scalar ? static_cast<const float*>(a.lam)[p] : static_cast<const float*>(a.lam)[(size_t)k * a.P + p]);
    const int cc = dcoef<D>(t - k) * dcoef<D>(t + r - k);
    v = v + lk * h_of<H>((float)cc);
  }
  return v;
}

template <typename F, typename H>
__device__ __forceinline__ H rhs_b(const PartArgs& a, int p, int t, int b) {
  const size_t it = (size_t)t * a.P + p;
  if constexpr (sizeof(F) == 8) {
    const double wt = static_cast<const double*>(a.w)[it];
    const double xt = static_cast<const double*>(a.x)[((size_t)t * a.B + b) * a.P + p];
    return wt > 0.0 ? h_ofd<H>(wt) * h_ofd<H>(xt) : h_ofd<H>(0.0);
  } else {
    const float wt = static_cast<const float*>(a.w)[it];
    const float xt = static_cast<const float*>(a.x)[((size_t)t * a.B + b) * a.P + p];
    return wt > 0.f ? h_of<H>(wt) * h_of<H>(xt) : h_of<H>(0.f);
  }
}

// Interior [s, e) of domain j and its separators.
__device__ __forceinline__ void domain(const PartArgs& a, int j, int D, int& s, int& e, bool& has_l, bool& has_r) {
  s = j * a.m;
  e = j + 1 < a.K ? (j + 1) * a.m - D : a.T;
  has_l = j > 0;
  has_r = j + 1 < a.K;
}

// Solve Omega_II u = rhs with the factor in registers-or-scratch: forward then back
// substitution over the n interior days; rhs(i) gives the right-hand side of local day i.
// The solution overwrites y[] (a thread-local array).
template <typename H, int D>
__device__ __forceinline__ void band_solve(const H* Lf, int n, H* y) {
  for (int i = 0; i < n; ++i) {
    H acc = y[i];
#pragma unroll
    for (int q = 1; q <= D; ++q)
      if (i - q >= 0) acc = acc - Lf[i * (D + 1) + q] * y[i - q];
    y[i] = acc;
  }
  for (int i = n - 1; i >= 0; --i) {
    H acc = y[i] * h_inv(Lf[i * (D + 1)]);
#pragma unroll
    for (int q = 1; q <= D; ++q)
      if (i + q < n) acc = acc - Lf[(i + q) * (D + 1) + q] * y[i + q];
    y[i] = acc;
  }
}

// The coupling columns of a domain's interior: E_L[i][c] = Omega[s-D+c][s+i] for the
// first D rows, E_R[i][c] = Omega[s+n-D+i][e+c] for the last D rows.
template <typename F, typename H, int D>
__device__ __forceinline__ void coupling(const PartArgs& a, int p, int s, int e, int n, bool has_l, bool has_r,
                                         H (&EL)[D][D], H (&ER)[D][D]) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      EL[i][c] = h_of<H>(0.f);
      ER[i][c] = h_of<H>(0.f);
      if (has_l && i < n) {
        const int u = s - D + c, t = s + i;
        if (t - u <= D) EL[i][c] = omega_entry<F, H, D>(a, p, u, t - u);
      }
      const int ii = n - D + i;
      if (has_r && ii >= 0) {
        const int t = s + ii, u = e + c;
        if (u - t <= D) ER[i][c] = omega_entry<F, H, D>(a, p, t, u - t);
      }
    }
}

template <typename F, typename H, int D>
__global__ void __launch_bounds__(kPartThreads) k_part_block(const PartArgs a) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  const int NS = a.K * a.P;
  if (slot >= NS) return;
  const int p = slot % a.P, j = slot / a.P;
  int s, e;
  bool has_l, has_r;
  domain(a, j, D, s, e, has_l, has_r);
  const int n = e - s;
  // input checks of the domain's days (w and the lambda rows it owns), for the status code
  {
    const int t1 = j + 1 < a.K ? (j + 1) * a.m : a.T;
    bool bad = false;
    int npos = 0;
    for (int t = s; t < t1; ++t) {
      const double wt = ldf<F>(a.w, (size_t)t * a.P + p);
      bad |= !(wt >= 0.0) || !isfinite(wt);
      npos += wt > 0.0;
      if (t < a.T - D && !a.lam_scalar) {
        const double lt = ldf<F>(a.lam, (size_t)t * a.P + p);
        bad |= !(lt > 0.0) || !isfinite(lt);
      }
    }
    if (j == 0 && a.lam_scalar && a.T > D) {
      const double lt = ldf<F>(a.lam, p);
      bad |= !(lt > 0.0) || !isfinite(lt);
    }
    if (bad) atomicOr(a.flags + p, 4u);
    if (npos > 0) atomicAdd(a.npos + p, npos);
  }
  H Lf[kPartMaxM * (D + 1)];
  bool badpiv = false;
  // banded LDL^T of Omega_II: L[i][i-q] D[i-q] = Omega[t][t-q] - sum_(r>q) L[i][i-r] D[i-r] L[i-q][i-r]
  for (int i = 0; i < n; ++i) {
    const int t = s + i;
#pragma unroll
    for (int q = D; q >= 1; --q) {
      if (i - q < 0) {
        Lf[i * (D + 1) + q] = h_of<H>(0.f);
        continue;
      }
      H v = omega_entry<F, H, D>(a, p, t - q, q);
#pragma unroll
      for (int r = q + 1; r <= D; ++r)
        if (i - r >= 0) v = v - Lf[i * (D + 1) + r] * Lf[(i - r) * (D + 1)] * Lf[(i - q) * (D + 1) + (r - q)];
      Lf[i * (D + 1) + q] = v * h_inv(Lf[(i - q) * (D + 1)]);
    }
    H dv = omega_entry<F, H, D>(a, p, t, 0);
#pragma unroll
    for (int q = 1; q <= D; ++q)
      if (i - q >= 0) dv = dv - Lf[i * (D + 1) + q] * Lf[i * (D + 1) + q] * Lf[(i - q) * (D + 1)];
    if (!h_pos(dv)) {
      badpiv = true;
      dv = h_of<H>(1.f);
    }
    Lf[i * (D + 1)] = dv;
  }
  if (badpiv) atomicOr(a.flags + p, 1u);
  H* fac = static_cast<H*>(a.fac);
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int q = 0; q <= D; ++q) fac[(size_t)(i * (D + 1) + q) * NS + slot] = Lf[i * (D + 1) + q];
  // coupling columns: E_L[i][c] = Omega[s-D+c][s+i] (nonzero for i <= c), E_R[i][c] =
  // Omega[s+i][e+c] (nonzero for n-1-i <= D-1-c); spikes V = Omega_II^{-1} E
  H y[kPartMaxM];
  H EL[D][D], ER[D][D];  // EL[i][c] for the first D rows, ER[i][c] for local row n-D+i
  coupling<F, H, D>(a, p, s, e, n, has_l, has_r, EL, ER);
  double* gl = static_cast<double*>(a.gl);
  double* gr = static_cast<double*>(a.gr);
  double* gc = static_cast<double*>(a.gc);
  // gl = -E_L^T V_L; gr = Omega_(S_j S_j) - E_R^T V_R (the separator's own block folded in);
  // gc = -E_L^T V_R (row of S_(j-1), column of S_j)
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (has_l) {
      for (int i = 0; i < n; ++i) y[i] = i < D ? EL[i][c] : h_of<H>(0.f);
      band_solve<H, D>(Lf, n, y);
#pragma unroll
      for (int c2 = 0; c2 < D; ++c2) {
        H acc = h_of<H>(0.f);
#pragma unroll
        for (int i = 0; i < D; ++i)
          if (i < n) acc = acc + EL[i][c2] * y[i];
        gl[(size_t)(c2 * D + c) * NS + slot] = -h_d(acc);
      }
    }
    if (has_r) {
      for (int i = 0; i < n; ++i) y[i] = h_of<H>(0.f);
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (n - D + i >= 0) y[n - D + i] = ER[i][c];
      band_solve<H, D>(Lf, n, y);
#pragma unroll
      for (int c2 = 0; c2 < D; ++c2) {
        H acc = h_of<H>(0.f);
#pragma unroll
        for (int i = 0; i < D; ++i)
          if (n - D + i >= 0) acc = acc + ER[i][c2] * y[n - D + i];
        const int lo = c2 < c ? c2 : c, hi = c2 < c ? c : c2;
        const H oss = omega_entry<F, H, D>(a, p, e + lo, hi - lo);
        gr[(size_t)(c2 * D + c) * NS + slot] = h_d(oss - acc);
        if (has_l) {
          H acc2 = h_of<H>(0.f);
#pragma unroll
          for (int i = 0; i < D; ++i)
            if (i < n) acc2 = acc2 + EL[i][c2] * y[i];
          gc[(size_t)(c2 * D + c) * NS + slot] = -h_d(acc2);
        }
      }
    }
  }
}

// One thread per (series, domain, band): y = Omega_II^{-1} b with the stored interior factor,
// then hl = E_L^T y and hr = b_(S_j) - E_R^T y.
template <typename F, typename H, int D>
__global__ void __launch_bounds__(kPartThreads) k_part_rhs(const PartArgs a) {
  const int NS = a.K * a.P;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= NS * a.B) return;
  const int slot = id % NS, b = id / NS;
  const int p = slot % a.P, j = slot / a.P;
  int s, e;
  bool has_l, has_r;
  domain(a, j, D, s, e, has_l, has_r);
  const int n = e - s;
  const H* fac = static_cast<const H*>(a.fac);
  H Lf[kPartMaxM * (D + 1)];
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int q = 0; q <= D; ++q) Lf[i * (D + 1) + q] = fac[(size_t)(i * (D + 1) + q) * NS + slot];
  H EL[D][D], ER[D][D];
  coupling<F, H, D>(a, p, s, e, n, has_l, has_r, EL, ER);
  H y[kPartMaxM];
  for (int i = 0; i < n; ++i) y[i] = rhs_b<F, H>(a, p, s + i, b);
  band_solve<H, D>(Lf, n, y);
  double* hl = static_cast<double*>(a.hl);
  double* hr = static_cast<double*>(a.hr);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (has_l) {
      H acc = h_of<H>(0.f);
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (i < n) acc = acc + EL[i][c] * y[i];
      hl[(size_t)(c * a.B + b) * NS + slot] = h_d(acc);
    }
    if (has_r) {
      H acc = h_of<H>(0.f);
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (n - D + i >= 0) acc = acc + ER[i][c] * y[n - D + i];
      hr[(size_t)(c * a.B + b) * NS + slot] = h_d(rhs_b<F, H>(a, p, e + c, b) - acc);
    }
  }
}

// One thread per series: status code, then block LDL^T of the separators' Schur complement
// S (block tridiagonal, d x d blocks) in FP64: this chain over the K-1 separators is
// sequential and latency-bound, where native FP64's short dependent chains beat
// double-float's. Each step's loads are issued one step ahead.
template <int D>
__global__ void __launch_bounds__(kPartThreads) k_part_reduce(const PartArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const uint32_t fl = a.flags[p];
  uint8_t code = (fl & 4u) ? WS_SERIES_BADARG
                           : (a.npos[p] < (D < a.T ? D : a.T) ? WS_SERIES_NOT_PD : WS_SERIES_OK);
  const int NS = a.K * a.P;
  const double* gl = static_cast<const double*>(a.gl);
  const double* gr = static_cast<const double*>(a.gr);
  const double* gc = static_cast<const double*>(a.gc);
  double* rl = static_cast<double*>(a.rl);
  double* rd = static_cast<double*>(a.rd);
  double* rc = static_cast<double*>(a.rc);
  double M[D][D];  // L_(j, j-1), rows of S_j
  double Dp[D];    // pivots of block j-1
#pragma unroll
  for (int r = 0; r < D; ++r) {
    Dp[r] = 1.0;
#pragma unroll
    for (int c = 0; c < D; ++c) M[r][c] = 0.0;
  }
  bool badpiv = (fl & 1u) != 0u;
  // step inputs: G = gr(domain j) + gl(domain j+1), C = gc(domain j+1)
  double G[D][D], C[D][D];
  auto load_step = [&](int j, double (&g)[D][D], double (&cc)[D][D]) {
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        g[r][c] = gr[(size_t)(r * D + c) * NS + j * a.P + p] + gl[(size_t)(r * D + c) * NS + (j + 1) * a.P + p];
        cc[r][c] = j + 2 < a.K ? gc[(size_t)(r * D + c) * NS + (j + 1) * a.P + p] : 0.0;
      }
  };
  if (a.K > 1) load_step(0, G, C);
  for (int j = 0; j + 1 < a.K; ++j) {
    double Gn[D][D], Cn[D][D];
    if (j + 2 < a.K) load_step(j + 1, Gn, Cn);
    double A[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        double v = G[r][c];
#pragma unroll
        for (int q = 0; q < D; ++q) v -= M[r][q] * Dp[q] * M[c][q];
        A[r][c] = v;
      }
    double Lb[D][D], Db[D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) Lb[r][c] = r == c ? 1.0 : 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double dv = A[c][c];
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (q < c) dv -= Lb[c][q] * Lb[c][q] * Db[q];
      if (!(dv > 0.0)) {
        badpiv = true;
        dv = 1.0;
      }
      Db[c] = dv;
#pragma unroll
      for (int r = 0; r < D; ++r) {
        if (r <= c) continue;
        double v = A[r][c];
#pragma unroll
        for (int q = 0; q < D; ++q)
          if (q < c) v -= Lb[r][q] * Lb[c][q] * Db[q];
        Lb[r][c] = v / dv;
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      rd[(size_t)(j * D + r) * a.P + p] = Db[r];
#pragma unroll
      for (int c = 0; c < D; ++c) rl[((size_t)(j * D + r) * D + c) * a.P + p] = Lb[r][c];
    }
    if (j + 2 < a.K) {
      // L_(j+1, j) = C^T Lb^-T diag(Db)^-1 with C = gc of domain j+1 (rows S_j, cols S_(j+1)):
      // row r of S_(j+1) solves Lb diag(Db) v = C[:, r]
#pragma unroll
      for (int r = 0; r < D; ++r) {
        double v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = C[c][r];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int q = 0; q < D; ++q)
            if (q < c) v[c] -= Lb[c][q] * v[q];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          v[c] /= Db[c];
          M[r][c] = v[c];
          rc[((size_t)(j * D + r) * D + c) * a.P + p] = v[c];
        }
      }
#pragma unroll
      for (int q = 0; q < D; ++q) Dp[q] = Db[q];
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          G[r][c] = Gn[r][c];
          C[r][c] = Cn[r][c];
        }
    }
  }
  if (badpiv && code == WS_SERIES_OK) code = WS_SERIES_NOT_PD;
  a.code[p] = code;
}

// One thread per (series, band): separators' z by block forward / back substitution (FP64,
// each step's loads issued one step ahead).
template <typename F, int D>
__global__ void __launch_bounds__(kPartThreads) k_part_rsolve(const PartArgs a) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.P * a.B) return;
  const int p = id % a.P, b = id / a.P;
  if (a.K < 2) return;
  const int NS = a.K * a.P;
  const bool ok = a.code[p] == WS_SERIES_OK;
  const double* hl = static_cast<const double*>(a.hl);
  const double* hr = static_cast<const double*>(a.hr);
  const double* rl = static_cast<const double*>(a.rl);
  const double* rd = static_cast<const double*>(a.rd);
  const double* rc = static_cast<const double*>(a.rc);
  double* zs = static_cast<double*>(a.zs);
  F* z = static_cast<F*>(a.z);
  // forward: y_j = Lb_j^-1 (rhs_j - L_(j, j-1) y_(j-1)), rhs_j = hr(domain j) - hl(domain j+1)
  auto ld_fwd = [&](int j, double (&rh)[D], double (&mm)[D][D], double (&lb)[D][D]) {
#pragma unroll
    for (int r = 0; r < D; ++r) {
      rh[r] = hr[(size_t)(r * a.B + b) * NS + j * a.P + p] - hl[(size_t)(r * a.B + b) * NS + (j + 1) * a.P + p];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        mm[r][c] = j > 0 ? rc[((size_t)((j - 1) * D + r) * D + c) * a.P + p] : 0.0;
        lb[r][c] = rl[((size_t)(j * D + r) * D + c) * a.P + p];
      }
    }
  };
  double yprev[D], rh[D], mm[D][D], lb[D][D];
#pragma unroll
  for (int q = 0; q < D; ++q) yprev[q] = 0.0;
  ld_fwd(0, rh, mm, lb);
  for (int j = 0; j + 1 < a.K; ++j) {
    double rh2[D], mm2[D][D], lb2[D][D];
    if (j + 2 < a.K) ld_fwd(j + 1, rh2, mm2, lb2);
    double v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double acc = rh[r];
#pragma unroll
      for (int c = 0; c < D; ++c) acc -= mm[r][c] * yprev[c];
      v[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c < r) v[r] -= lb[r][c] * v[c];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      yprev[r] = v[r];
      zs[((size_t)(j * D + r) * a.B + b) * a.P + p] = v[r];
    }
    if (j + 2 < a.K) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        rh[r] = rh2[r];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          mm[r][c] = mm2[r][c];
          lb[r][c] = lb2[r][c];
        }
      }
    }
  }
  // back: z_j = Lb_j^-T (Db_j^-1 y_j - L_(j+1, j)^T z_(j+1))
  auto ld_bwd = [&](int j, double (&yy)[D], double (&dd)[D], double (&mm)[D][D], double (&lb)[D][D]) {
#pragma unroll
    for (int r = 0; r < D; ++r) {
      yy[r] = zs[((size_t)(j * D + r) * a.B + b) * a.P + p];
      dd[r] = rd[(size_t)(j * D + r) * a.P + p];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        mm[r][c] = j + 2 < a.K ? rc[((size_t)(j * D + r) * D + c) * a.P + p] : 0.0;
        lb[r][c] = rl[((size_t)(j * D + r) * D + c) * a.P + p];
      }
    }
  };
  double znext[D], yy[D], dd[D];
#pragma unroll
  for (int q = 0; q < D; ++q) znext[q] = 0.0;
  ld_bwd(a.K - 2, yy, dd, mm, lb);
  for (int j = a.K - 2; j >= 0; --j) {
    double yy2[D], dd2[D], mm2[D][D], lb2[D][D];
    if (j > 0) ld_bwd(j - 1, yy2, dd2, mm2, lb2);
    const int u0 = (j + 1) * a.m - D;
    double v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      double acc = yy[r] / dd[r];
#pragma unroll
      for (int c = 0; c < D; ++c) acc -= mm[c][r] * znext[c];  // (L_(j+1, j)^T z_(j+1))[r]
      v[r] = acc;
    }
#pragma unroll
    for (int r = D - 1; r >= 0; --r)
#pragma unroll
      for (int c = 0; c < D; ++c)
        if (c > r) v[r] -= lb[c][r] * v[c];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      znext[r] = v[r];
      zs[((size_t)(j * D + r) * a.B + b) * a.P + p] = v[r];
      const F out = ok ? (F)v[r] : F(0);
      z[((size_t)(u0 + r) * a.B + b) * a.P + p] = out;
      if (ok && !isfinite((double)out)) atomicOr(a.flags + p, 2u);
    }
    if (j > 0) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        yy[r] = yy2[r];
        dd[r] = dd2[r];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          mm[r][c] = mm2[r][c];
          lb[r][c] = lb2[r][c];
        }
      }
    }
  }
}

// One thread per (series, domain, band): interior z with the separators' z known.
template <typename F, typename H, int D>
__global__ void __launch_bounds__(kPartThreads) k_part_finish(const PartArgs a) {
  const int NS = a.K * a.P;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= NS * a.B) return;
  const int slot = id % NS, b = id / NS;
  const int p = slot % a.P, j = slot / a.P;
  int s, e;
  bool has_l, has_r;
  domain(a, j, D, s, e, has_l, has_r);
  const int n = e - s;
  const bool ok = a.code[p] == WS_SERIES_OK;
  F* z = static_cast<F*>(a.z);
  if (!ok) {
    for (int i = 0; i < n; ++i) z[((size_t)(s + i) * a.B + b) * a.P + p] = F(0);
    return;
  }
  const H* fac = static_cast<const H*>(a.fac);
  const double* zs = static_cast<const double*>(a.zs);
  H Lf[kPartMaxM * (D + 1)];
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int q = 0; q <= D; ++q) Lf[i * (D + 1) + q] = fac[(size_t)(i * (D + 1) + q) * NS + slot];
  H EL[D][D], ER[D][D];
  coupling<F, H, D>(a, p, s, e, n, has_l, has_r, EL, ER);
  H y[kPartMaxM];
  for (int i = 0; i < n; ++i) y[i] = rhs_b<F, H>(a, p, s + i, b);
  // b_I - E_L z_S(j-1) - E_R z_S(j): E_L touches the first D rows, E_R the last D
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const H zl = has_l ? h_ofd<H>(zs[((size_t)((j - 1) * D + c) * a.B + b) * a.P + p]) : h_of<H>(0.f);
    const H zr = has_r ? h_ofd<H>(zs[((size_t)(j * D + c) * a.B + b) * a.P + p]) : h_of<H>(0.f);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (has_l && i < n) y[i] = y[i] - EL[i][c] * zl;
      if (has_r && n - D + i >= 0) y[n - D + i] = y[n - D + i] - ER[i][c] * zr;
    }
  }
  band_solve<H, D>(Lf, n, y);
  bool nonfin = false;
  for (int i = 0; i < n; ++i) {
    const F out = (F)h_d(y[i]);
    nonfin |= !isfinite((double)out);
    z[((size_t)(s + i) * a.B + b) * a.P + p] = out;
  }
  if (nonfin) atomicOr(a.flags + p, 2u);
}

__global__ void k_part_status(const PartArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P || a.status == nullptr) return;
  const uint8_t c = a.code[p];
  a.status[p] = c == WS_SERIES_OK && (a.flags[p] & 2u) ? WS_SERIES_NONFINITE : c;
}

// ---------------------------------------------------------------------------------- host

static size_t p256(size_t v) { return (v + 255) & ~(size_t)255; }

// Domain length: the largest of 64 / 32 / 16 days (>= 2d + 2) that still gives the domain
// phases about one warp per SM (longer domains shorten the sequential separator chain);
// series of at most 64 days use one domain.
int part_domain_len(const ws_problem& pb) {
  const int d = pb.d;
  int m = kPartMaxM;
  const long want = 148L * 32;  // threads for the domain phases
  while (m > 16 && m / 2 >= 2 * d + 2 && (long)pb.n_series * ((pb.T + m - 1) / m) < want) m /= 2;
  return m;
}

struct PartLayout {
  size_t fac, gl, gr, gc, hl, hr, rl, rd, rc, zs, flags, npos, code, total;
};

static PartLayout part_layout(const ws_problem& pb, int m) {
  const int d = pb.d, B = pb.n_bands;
  const size_t P = (size_t)pb.n_series, K = ((size_t)pb.T + m - 1) / m, NS = K * P;
  const size_t hs = pb.dtype == WS_F64 ? 8 : sizeof(dwf);
  PartLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += p256(bytes);
    return o;
  };
  L.fac = take((size_t)m * (d + 1) * NS * hs);
  L.gl = take((size_t)d * d * NS * 8);
  L.gr = take((size_t)d * d * NS * 8);
  L.gc = take((size_t)d * d * NS * 8);
  L.hl = take((size_t)d * B * NS * 8);
  L.hr = take((size_t)d * B * NS * 8);
  L.rl = take((size_t)K * d * d * P * 8);
  L.rd = take((size_t)K * d * P * 8);
  L.rc = take((size_t)K * d * d * P * 8);
  L.zs = take((size_t)K * d * B * P * 8);
  L.flags = take(P * 4);
  L.npos = take(P * 4);
  L.code = take(P);
  L.total = off;
  return L;
}

size_t part_workspace_bytes(const ws_problem& pb) {
  if (pb.n_series == 0 || pb.T == 0) return 0;
  return part_layout(pb, part_domain_len(pb)).total;
}

template <typename F, typename H, int D>
static int part_launch_t(const PartArgs& a, cudaStream_t st) {
  const int NS = a.K * a.P;
  const int gb = (NS + kPartThreads - 1) / kPartThreads;
  const int gbb = (NS * a.B + kPartThreads - 1) / kPartThreads;
  k_part_block<F, H, D><<<gb, kPartThreads, 0, st>>>(a);
  k_part_rhs<F, H, D><<<gbb, kPartThreads, 0, st>>>(a);
  k_part_reduce<D><<<(a.P + kPartThreads - 1) / kPartThreads, kPartThreads, 0, st>>>(a);
  k_part_rsolve<F, D><<<(a.P * a.B + kPartThreads - 1) / kPartThreads, kPartThreads, 0, st>>>(a);
  k_part_finish<F, H, D><<<gbb, kPartThreads, 0, st>>>(a);
  k_part_status<<<(a.P + kPartThreads - 1) / kPartThreads, kPartThreads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "partitioned solve launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int launch_partitioned(const ws_problem& pb, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                       void* scratch, cudaStream_t st) {
  const int m = part_domain_len(pb);
  const PartLayout L = part_layout(pb, m);
  char* b = static_cast<char*>(scratch);
  PartArgs a;
  a.T = pb.T;
  a.P = (int)pb.n_series;
  a.B = pb.n_bands;
  a.m = m;
  a.K = (pb.T + m - 1) / m;
  a.lam_scalar = pb.lam_mode == WS_LAM_SCALAR;
  a.x = x;
  a.w = w;
  a.lam = lam;
  a.z = z;
  a.status = status;
  a.fac = b + L.fac;
  a.gl = b + L.gl;
  a.gr = b + L.gr;
  a.gc = b + L.gc;
  a.hl = b + L.hl;
  a.hr = b + L.hr;
  a.rl = b + L.rl;
  a.rd = b + L.rd;
  a.rc = b + L.rc;
  a.zs = b + L.zs;
  a.flags = reinterpret_cast<uint32_t*>(b + L.flags);
  a.npos = reinterpret_cast<int32_t*>(b + L.npos);
  a.code = reinterpret_cast<uint8_t*>(b + L.code);
  // flags and npos are adjacent: one memset clears both
  if (cudaMemsetAsync(a.flags, 0, L.code - L.flags, st) != cudaSuccess) return set_error(WS_ECUDA, "memset failed");
  if (pb.dtype == WS_F64) {
    switch (pb.d) {
      case 1: return part_launch_t<double, double, 1>(a, st);
      case 2: return part_launch_t<double, double, 2>(a, st);
      case 3: return part_launch_t<double, double, 3>(a, st);
      default: return part_launch_t<double, double, 4>(a, st);
    }
  }
  switch (pb.d) {
    case 1: return part_launch_t<float, dwf, 1>(a, st);
    case 2: return part_launch_t<float, dwf, 2>(a, st);
    case 3: return part_launch_t<float, dwf, 3>(a, st);
    default: return part_launch_t<float, dwf, 4>(a, st);
  }
}

}  // namespace ws
