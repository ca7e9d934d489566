// Gradient with respect to the observation weights: the weights of the objective (Eq. 1)
// taken as parameters (soft weights). Differentiating Omega z = W x in w_t gives
// e_t z_t + Omega dz = e_t x_t, so dz/dw_t = Omega^{-1} e_t (x_t - z_t) and, with
// g = Omega^{-1} dL/dz (Omega symmetric; the adjoint solve of Section 2.3),
//     dL/dw_t = sum_b g_tb (x_tb - z_tb),
// where a day with w_t = 0 contributes x_t = 0 (the smoother ignores the value observed
// there; it is selected away, never multiplied, so a NaN in a gap does no harm). The same
// pass turns g into dL/dx = W g (Eq. 5, transposed).
//
// One thread per (day, series): the B bands of that pixel-day are read in turn (coalesced
// across the warp's series), so x, z and g are each read once and gx, gw written once.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"

namespace ws {

constexpr int kWgNP = 128;

template <typename F>
__global__ void __launch_bounds__(kWgNP) k_wgrad(int B, int P, int n_pb, const F* __restrict__ x,
                                                 const F* __restrict__ w, const F* __restrict__ z, const F* g,
                                                 F* gx, F* __restrict__ gw) {
  const int t = blockIdx.x / n_pb;
  const int p = (blockIdx.x % n_pb) * kWgNP + threadIdx.x;
  if (p >= P) return;
  const size_t sP = (size_t)P;
  const F wt = w[(size_t)t * sP + p];
  const bool on = wt > F(0);
  F acc = F(0);
  for (int b = 0; b < B; ++b) {
    const size_t o = ((size_t)t * B + b) * sP + p;
    const F gv = g[o];  // g and gx may be the same array: read before the write
    const F xv = on ? x[o] : F(0);
    acc = fma(gv, xv - z[o], acc);
    if (gx != nullptr) gx[o] = wt * gv;
  }
  gw[(size_t)t * sP + p] = acc;
}

int launch_wgrad(const ws_problem& pb, const void* x, const void* w, const void* z, void* g, void* gx, void* gw,
                 cudaStream_t st) {
  const int P = (int)pb.n_series;
  const int n_pb = (P + kWgNP - 1) / kWgNP;
  const long long blocks = (long long)pb.T * n_pb;
  if (blocks > 0x7fffffffLL) return set_error(WS_EINVAL, "weight gradient: too many days x series");
  if (pb.dtype == WS_F64)
    k_wgrad<double><<<(unsigned)blocks, kWgNP, 0, st>>>(pb.n_bands, P, n_pb, static_cast<const double*>(x),
                                                        static_cast<const double*>(w), static_cast<const double*>(z),
                                                        static_cast<const double*>(g), static_cast<double*>(gx),
                                                        static_cast<double*>(gw));
  else
    k_wgrad<float><<<(unsigned)blocks, kWgNP, 0, st>>>(pb.n_bands, P, n_pb, static_cast<const float*>(x),
                                                       static_cast<const float*>(w), static_cast<const float*>(z),
                                                       static_cast<const float*>(g), static_cast<float*>(gx),
                                                       static_cast<float*>(gw));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "weight gradient kernel launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

}  // namespace ws
