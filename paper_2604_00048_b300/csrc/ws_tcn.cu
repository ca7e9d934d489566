// Temporal convolution network g_theta: (x, w) per day -> log lambda per day, and its
// training kernels (forward with stored activations, backward, Adam).
//
// The paper's lambda network (Section 4.2) maps the series to a per-day Lambda through a
// sigmoid range; here it is a 4-layer 1-D convolution net, kernel 9, "same" zero padding,
// channels 2 -> 64 -> 64 -> 64 -> 1, ReLU between layers, BF16 weights and activations with
// FP32 accumulation, and log lambda = Lmin + sigmoid(o) (Lmax - Lmin).
//
// Rows. A batch of n series of T days is laid out as a stream of R = n (T + G) rows, series s
// at rows s (T + G) .. s (T + G) + T - 1 followed by G = 4 gap rows. Every layer writes zeros
// on gap rows, so the 4-row reach of a kernel-9 convolution never crosses from one series to
// the next: the stream is exactly the per-series "same"-padded convolution.
//
// Kernels:
//   k_tcn_in      (x, w) in the [T][P] tile layout -> in0[R][2] (BF16), zero on gaps
//   k_tcn_fused   the forward: all four layers per tile on the tensor cores (tcgen05, BF16 x
//                 BF16 -> FP32 in TMEM, ~151 kFLOP / row), sigmoid range -> lambda in [T][P]
//   k_conv64      one 64 -> 64 layer on the tensor cores; the backward uses it for the data
//                 gradients of layers 3 and 2 (flipped, transposed weights)
//   backward      d o, layer-4 data gradient, weight gradients (CUDA cores), Adam
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "ws_internal.h"
#include "ws_ptx.cuh"
#include "ws_tc.cuh"

namespace ws {

constexpr int kCh = 64, kTaps = 9, kHalf = 4, kGap = 4;
constexpr int kTileRows = 384;                  // output rows of one conv64 tile (3 x M = 128)
constexpr int kInRows = kTileRows + 2 * kHalf;  // staged input rows
constexpr int kPlaneBytes = kInRows * 16;       // one 8-channel plane of the staged input
constexpr int kActBytes = 8 * kPlaneBytes;      // 50,176
constexpr int kWBytes = kTaps * 8 * kCh * 16;   // 73,728: [tap][ci chunk][co][8 ci]
constexpr int kConvThreads = 128;
constexpr uint32_t kTmemCols = 256;

// parameter offsets in the FP32 master vector (PyTorch conv1d layouts [out][in][k])
constexpr int kOW1 = 0, kOB1 = kOW1 + kCh * 2 * kTaps, kOW2 = kOB1 + kCh, kOB2 = kOW2 + kCh * kCh * kTaps,
              kOW3 = kOB2 + kCh, kOB3 = kOW3 + kCh * kCh * kTaps, kOW4 = kOB3 + kCh, kOB4 = kOW4 + kCh * kTaps,
              kNParams = kOB4 + 1;
static_assert(kNParams == WS_TCN_PARAMS, "parameter count");
// packed BF16 buffer (elements): W1 [co][c][k], W2 fwd, W2 bwd, W3 fwd, W3 bwd ([tap][chunk][row][8]), W4 [ci][k]
// + tensor-core copies of W1 (K = 2 x 9 -> 32: [4 chunks][64 co][8]) and W4 as taps x channels
// ([16 rows: tap 0..8, zero beyond][64 ci])
constexpr int kPW1 = 0, kPW2F = kPW1 + kCh * 2 * kTaps, kPW2B = kPW2F + kCh * kCh * kTaps,
              kPW3F = kPW2B + kCh * kCh * kTaps, kPW3B = kPW3F + kCh * kCh * kTaps,
              kPW4 = kPW3B + kCh * kCh * kTaps, kPW1T = kPW4 + kCh * kTaps, kPW4T = kPW1T + 4 * kCh * 8,
              kPackedElems = kPW4T + 16 * kCh;
static_assert(WS_TCN_PACKED_BYTES == kPackedElems * 2, "packed size");

__device__ __forceinline__ bool is_gap(int64_t r, int T) { return (int)(r % (T + kGap)) >= T; }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// ---------------------------------------------------------------------------------------
// Input rows: in0[r] = (x if w > 0 else 0, w) in BF16, zero on gap rows.
__global__ void k_tcn_in(const float* __restrict__ x, const float* __restrict__ w, uint32_t* __restrict__ in0,
                         int T, int P, int64_t R) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int s = (int)(r / (T + kGap)), t = (int)(r % (T + kGap));
  float xv = 0.f, wv = 0.f;
  if (t < T) {
    wv = w[(size_t)t * P + s];
    xv = wv > 0.f ? x[(size_t)t * P + s] : 0.f;
  }
  in0[r] = pack_bf16x2(xv, wv);
}

// ---------------------------------------------------------------------------------------
// 64 -> 64 convolution over stream rows on the tensor cores.
//   out[r][co] = epi( sum_{tap, ci} Wp[tap][ci chunk][co][ci % 8] * in[r + tap - 4][ci] )
// MODE_FWD: epi = ReLU(. + bias), zero on gap rows. MODE_BWD: epi = . * (mask[r][co] > 0)
// (the data gradient through a ReLU layer; the caller passes the flipped, transposed weights).
// Per tile: 392 input rows staged as 8 planes; for each of 3 M-blocks of 128 rows, 9 taps x
// 4 K-steps of M128 x N64 x K16 MMAs accumulate in TMEM columns [64 b, 64 b + 64).
enum { CONV_FWD = 0, CONV_BWD = 1 };

struct ConvArgs {
  const uint4* in;     // [R][8] 16-byte chunks (64 BF16)
  const uint4* wp;     // kWBytes, plane layout
  const float* bias;   // FWD
  const uint4* mask;   // BWD: [R][8]
  uint4* out;          // [R][8]
  int64_t R;
  int T;
  int n_tiles;
  unsigned* err;
};

template <int MODE>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv64(const ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* act = smem;                 // kActBytes
  unsigned char* wts = smem + kActBytes;     // kWBytes
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kActBytes + kWBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kActBytes + kWBytes + 8);
  int* sflag = reinterpret_cast<int*>(smem + kActBytes + kWBytes + 12);
  __shared__ float sbias[kCh];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *sflag = 0;
  }
  if (MODE == CONV_FWD && tid < kCh) sbias[tid] = a.bias[tid];
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  // weights once per CTA: plane layout in global ([tap][chunk][row][8]) -> 128-byte swizzled
  // rows in shared memory ([tap][row][chunk ^ (row % 8)])
  for (int i = tid; i < kWBytes / 16; i += kConvThreads) {
    const int row = i & 63, chunk = (i >> 6) & 7, tap = i >> 9;
    cp_async16(wts + tap * 8192 + row * 128 + ((chunk ^ (row & 7)) << 4), a.wp + i, true);
  }
  cp_async_commit();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = umma_idesc_bf16(128, 64);
  const uint32_t act_s = smem_u32(act), wts_s = smem_u32(wts);
  uint32_t phase = 0;

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * kTileRows;
    // stage input rows r0 - 4 .. r0 + 387, 128-byte swizzled: chunk j of row i at
    // act + 128 i + 16 (j ^ (i % 8))
    for (int e = tid; e < kInRows * 8; e += kConvThreads) {
      const int i = e >> 3, j = e & 7;
      const int64_t r = r0 - kHalf + i;
      const bool v = r >= 0 && r < a.R;
      cp_async16(act + 128 * i + ((j ^ (i & 7)) << 4), a.in + (v ? r * 8 + j : 0), v);
    }
    cp_async_commit();
    cp_async_wait<0>();
    fence_proxy_async_smem();  // generic/LDGSTS writes -> visible to the tensor core (async proxy)
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int b = 0; b < 3; ++b) {
        const uint32_t d = tmem + (uint32_t)(b * 64);
        for (int tap = 0; tap < kTaps; ++tap) {
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const uint64_t ad = umma_desc_sw128(act_s + (uint32_t)((b * 128 + tap) * 128 + 32 * s));
            const uint64_t bd = umma_desc_sw128(wts_s + (uint32_t)(tap * 8192 + 32 * s));
            umma_bf16(d, ad, bd, idesc, (tap | s) != 0);
          }
        }
      }
      umma_commit(bar);
    }
    // wait for the MMAs (bounded; thread 0 polls, the rest sleep at the barrier)
    if (tid == 0 && !mbar_wait_bounded(bar, phase)) {
      atomicOr(a.err, kDevErrTimeout);
      *sflag = 1;
    }
    __syncthreads();
    if (*sflag) break;
    phase ^= 1u;
    tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (rows), 64 columns per M-block
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
      const int row = b * 128 + warp * 32 + lane;
      const int64_t r = r0 + row;
      const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * 64);
      uint32_t v[4][16];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(tbase + 16 * q, v[q]);
      tmem_ld_wait();
      if (r >= a.R) continue;
      const bool gap = MODE == CONV_FWD && is_gap(r, a.T);
      uint4 m8[8];
      if (MODE == CONV_BWD) {
#pragma unroll
        for (int j = 0; j < 8; ++j) m8[j] = a.mask[r * 8 + j];
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int co = 8 * j + e;
          float acc = __uint_as_float(v[co >> 4][co & 15]);
          if (MODE == CONV_FWD) {
            acc = gap ? 0.f : fmaxf(acc + sbias[co], 0.f);
          } else {
            const uint32_t mw = (e < 2) ? m8[j].x : (e < 4) ? m8[j].y : (e < 6) ? m8[j].z : m8[j].w;
            const float mv = (e & 1) ? bf16_hi(mw) : bf16_lo(mw);
            acc = mv > 0.f ? acc : 0.f;
          }
          f[e] = acc;
        }
        a.out[r * 8 + j] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                                      pack_bf16x2(f[6], f[7]));
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  __syncthreads();
  if (*sflag && tid == 0) {
    // a wait gave up: give the MMAs in flight a second bounded wait before freeing TMEM
    mbar_wait_bounded(bar, phase);
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------------------
// Fused forward: the four layers of one tile of 384 computed rows, activations kept in
// shared memory, all weights resident (one CTA per SM).
//   layer 1: tensor cores, im2col of the 2 input channels x 9 taps (K = 18 padded to 32)
//   layers 2, 3: tensor cores, 9 taps x 4 K-steps of M128 x N64 x K16, operands read in place
//   layer 4 (64 -> 1): the per-tap products P[r][tap] = sum_ci a3[r][ci] W4[ci][tap] as one
//     unshifted M128 x N16 GEMM (4 K-steps per M-block, taps along N), then the shift on the
//     output side, o[r] = b4 + sum_tap P[r + tap - 4][tap], through shared memory. (Shifting
//     the input instead takes 36 N = 16 MMAs per M-block, each reading the 4 KB A operand.)
// Activations live in the 128-byte swizzled K-major layout (row r's 64 channels in 128 bytes,
// 16-byte chunk c at position c ^ (r % 8)): a tap shift is a start address 128 bytes further.
// Each layer's epilogue (TMEM -> registers -> bias, ReLU -> BF16) writes over the layer's
// input after its MMAs have completed. (Overlapping an M-block's epilogue with the MMAs of
// the next blocks, with a dedicated issuing warp or with per-block commits, measured 10-25%
// slower on B300 than this phase-by-phase order: these N = 64 MMAs are bound by the shared-
// memory operand reads, and concurrent epilogue traffic slows them more than it hides.) A layer is exact 4 rows less deep at each end of the
// tile, so of the 384 computed rows the middle 352 (rows 16 .. 367) are final.
constexpr int kFuseUseful = kTileRows - 32;
constexpr int kFuseThreads = 512;                  // 16 warps: four per TMEM lane quarter
constexpr int kActSw = kInRows * 128;              // 50,176: swizzled activation rows
constexpr int kImPlane = kTileRows * 16;           // 6144: one 8-wide K chunk of the im2col
constexpr int kW1TBytes = 4 * kCh * 16;            // 4096
constexpr int kWSwBytes = kTaps * kCh * 128;       // 73,728: [tap][row][128 B swizzled]
constexpr int kFW2 = kActSw, kFW3 = kFW2 + kWSwBytes, kFW4 = kFW3 + kWSwBytes, kFW1 = kFW4 + 16 * 128,
              kFP = kFW1 + kW1TBytes, kFIn = kFP + kTileRows * kTaps * 4, kFBar = kFIn + kInRows * 4,
              kFBias = kFBar + 16, kFSmem = kFBias + (3 * kCh + 4) * 4;

struct FusedArgs {
  const uint32_t* in0;
  const uint4 *w1t, *w2, *w3;
  const __nv_bfloat16* w4t;  // [16 tap rows][64 ci]
  const float* master;
  float* lam;
  float* loglam;
  float* o_out;
  uint4 *a1, *a2, *a3;  // training: activations of the final rows
  int64_t R;
  int T, P, n_tiles;
  float lmin, lmax;
  unsigned* err;
};

__global__ void __launch_bounds__(kFuseThreads, 1) k_tcn_fused(const FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* act = smem;
  float* sP = reinterpret_cast<float*>(smem + kFP);    // [384][9] layer-4 per-tap products
  uint32_t* sin0 = reinterpret_cast<uint32_t*>(smem + kFIn);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kFBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kFBar + 8);
  int* sflag = reinterpret_cast<int*>(smem + kFBar + 12);
  float* sb = reinterpret_cast<float*>(smem + kFBias);  // b1 | b2 | b3 | b4
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quarter = warp & 3, part = warp >> 2;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    *sflag = 0;
  }
  if (warp == 0) {
    tmem_alloc(tslot, kTmemCols);
    tmem_relinquish();
  }
  // W2, W3: plane layout in global ([tap][chunk][row][8]) -> swizzled rows
  for (int i = tid; i < kWBytes / 16; i += kFuseThreads) {
    const int row = i & 63, chunk = (i >> 6) & 7, tap = i >> 9;
    const int dst = tap * 8192 + row * 128 + ((chunk ^ (row & 7)) << 4);
    cp_async16(smem + kFW2 + dst, a.w2 + i, true);
    cp_async16(smem + kFW3 + dst, a.w3 + i, true);
  }
  for (int i = tid; i < kW1TBytes / 16; i += kFuseThreads) cp_async16(smem + kFW1 + 16 * i, a.w1t + i, true);
  for (int i = tid; i < 16 * 8; i += kFuseThreads) {  // W4T rows (taps) of 8 chunks, swizzled
    const int row = i >> 3, chunk = i & 7;
    cp_async16(smem + kFW4 + row * 128 + ((chunk ^ (row & 7)) << 4), reinterpret_cast<const uint4*>(a.w4t) + i, true);
  }
  cp_async_commit();
  for (int i = tid; i < kActSw / 16; i += kFuseThreads) reinterpret_cast<uint4*>(act)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 3 * kCh; i += kFuseThreads)
    sb[i] = a.master[(i >> 6) == 0 ? kOB1 + i : (i >> 6) == 1 ? kOB2 + i - 64 : kOB3 + i - 128];
  if (tid == 0) sb[3 * kCh] = a.master[kOB4];
  cp_async_wait<0>();
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id64 = umma_idesc_bf16(128, 64);
  const uint32_t act_s = smem_u32(act);
  const uint64_t im_desc = umma_desc(act_s, kImPlane, 128);  // layer 1's im2col planes (no swizzle)
  const uint64_t w1d = umma_desc(smem_u32(smem + kFW1), kCh * 16, 128);
  const uint64_t act_d = umma_desc_sw128(act_s);
  const uint64_t w2d = umma_desc_sw128(smem_u32(smem + kFW2)), w3d = umma_desc_sw128(smem_u32(smem + kFW3));
  const uint64_t w4d = umma_desc_sw128(smem_u32(smem + kFW4));
  const uint32_t id16 = umma_idesc_bf16(128, 16);
  uint32_t phase = 0;

  auto wait_mma = [&]() -> bool {
    if (tid == 0 && !mbar_wait_bounded(bar, phase)) {
      atomicOr(a.err, kDevErrTimeout);
      *sflag = 1;
    }
    __syncthreads();
    phase ^= 1u;
    tc_fence_after();
    return *sflag == 0;
  };
  // 64 -> 64 layer: 3 M-blocks x 9 taps x 4 K-steps (descriptor = base + start >> 4)
  auto issue_conv = [&](uint64_t wd) {
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap)
#pragma unroll
          for (int s = 0; s < 4; ++s)
            umma_bf16(tmem + (uint32_t)(b * 64), act_d + (uint64_t)(((b * 128 + tap) * 128 + 32 * s) >> 4),
                      wd + (uint64_t)((tap * 8192 + 32 * s) >> 4), id64, (tap | s) != 0);
      umma_commit(bar);
    }
  };

  const int period = a.T + kGap;
  bool rowok[3];
  int rs[3], rt[3];
  // the next tile's input rows are loaded into a register while the current tile computes
  auto load_in0 = [&](int tl) -> uint32_t {
    const int64_t r = (int64_t)tl * kFuseUseful - 16 - kHalf + tid;
    return (tid < kInRows && tl < a.n_tiles && r >= 0 && r < a.R) ? a.in0[r] : 0u;
  };
  static_assert(kInRows <= kFuseThreads, "one staged input row per thread");
  uint32_t in_next = load_in0(blockIdx.x);
  // epilogue of a 64-channel layer: bias, ReLU, zero off-series; in place at buffer row + 4.
  // With l4, also the layer-4 partial sums of this row's 16 channels.
  auto epi64 = [&](int64_t r0, const float* bias_s, uint4* store) {
    float bias[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) bias[c] = bias_s[part * 16 + c];
    uint32_t vv[3][16];
#pragma unroll
    for (int b = 0; b < 3; ++b) tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 64 + part * 16), vv[b]);
    tmem_ld_wait();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int row = b * 128 + quarter * 32 + lane;
      const int64_t r = r0 + row;
      const uint32_t* v = vv[b];
      const bool zero = !rowok[b];
      uint4 q[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = zero ? 0.f : fmaxf(__uint_as_float(v[8 * j + e]) + bias[8 * j + e], 0.f);
        q[j] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                          pack_bf16x2(f[6], f[7]));
        const int srow = row + kHalf, chunk = part * 2 + j;
        *reinterpret_cast<uint4*>(act + srow * 128 + ((chunk ^ (srow & 7)) << 4)) = q[j];
      }
      if (store != nullptr && row >= 16 && row < 16 + kFuseUseful && r >= 0 && r < a.R)
#pragma unroll
        for (int j = 0; j < 2; ++j) store[r * 8 + part * 2 + j] = q[j];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
  };

  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * kFuseUseful - 16;  // first computed row
    {
      const int64_t rb = r0 < 0 ? 0 : r0;
      const int64_t sb0 = rb / period;  // one 64-bit division per tile, 32-bit math after
      const int tb0 = (int)(rb - sb0 * period);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int64_t r = r0 + b * 128 + quarter * 32 + lane;
        const int off = tb0 + (int)(r - rb);
        const int q = off / period;
        rs[b] = (int)(sb0 + q);
        rt[b] = off - q * period;
        rowok[b] = r >= 0 && r < a.R && rt[b] < a.T;
      }
    }
    if (tid < kInRows) sin0[tid] = in_next;
    in_next = load_in0(tile + gridDim.x);
    __syncthreads();
    // im2col of layer 1: row i, K index kk = 2 tap + c (c = 0: x, 1: w), 4 chunks of 8
    for (int e = tid; e < kTileRows * 4; e += kFuseThreads) {
      const int i = e >> 2, j = e & 3;
      uint32_t u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float f[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kk = 8 * j + 2 * q + h;
          const uint32_t src = kk < 2 * kTaps ? sin0[i + (kk >> 1)] : 0u;
          f[h] = (kk & 1) ? bf16_hi(src) : bf16_lo(src);
        }
        u[q] = pack_bf16x2(f[0], f[1]);
      }
      *reinterpret_cast<uint4*>(act + j * kImPlane + i * 16) = make_uint4(u[0], u[1], u[2], u[3]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int s = 0; s < 2; ++s)
          umma_bf16(tmem + (uint32_t)(b * 64), im_desc + (uint64_t)((2 * s * kImPlane + b * 128 * 16) >> 4),
                    w1d + (uint64_t)((2 * s * kCh * 16) >> 4), id64, s != 0);
      umma_commit(bar);
    }
    if (!wait_mma()) break;
    epi64(r0, sb, a.a1);
    issue_conv(w2d);
    if (!wait_mma()) break;
    epi64(r0, sb + kCh, a.a2);
    issue_conv(w3d);
    if (!wait_mma()) break;
    epi64(r0, sb + 2 * kCh, a.a3);
    // layer 4: P[row][tap] on the tensor cores (A = a3 rows, unshifted: buffer row + 4)
    if (tid == 0) {
      tc_fence_after();
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int s = 0; s < 4; ++s)
          umma_bf16(tmem + (uint32_t)(b * 64), act_d + (uint64_t)(((b * 128 + kHalf) * 128 + 32 * s) >> 4),
                    w4d + (uint64_t)((32 * s) >> 4), id16, s != 0);
      umma_commit(bar);
    }
    if (!wait_mma()) break;
    if (part == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int row = b * 128 + quarter * 32 + lane;
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 64), v);
        tmem_ld_wait();
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) sP[row * kTaps + tap] = __uint_as_float(v[tap]);
      }
    }
    tc_fence_before();
    __syncthreads();
    // o[row] = b4 + sum_tap P[row + tap - 4][tap] for the final rows, one row per thread
    if (tid < kFuseUseful) {
      const int row = 16 + tid;
      const int64_t r = r0 + row;
      if (r >= 0 && r < a.R) {
        const int64_t sq = r / period;
        const int t = (int)(r - sq * period);
        if (t >= a.T) {
          if (a.o_out) a.o_out[r] = 0.f;
        } else {
          float o = sb[3 * kCh];
#pragma unroll
          for (int tap = 0; tap < kTaps; ++tap) o += sP[(row + tap - kHalf) * kTaps + tap];
          const float sg = 1.f / (1.f + expf(-o));
          const float ll = a.lmin + sg * (a.lmax - a.lmin);
          a.lam[(size_t)t * a.P + sq] = expf(ll);
          if (a.loglam) a.loglam[(size_t)t * a.P + sq] = ll;
          if (a.o_out) a.o_out[r] = o;
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (*sflag && tid == 0) mbar_wait_bounded(bar, phase);  // let MMAs in flight drain before freeing TMEM
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------------------
// Backward.
// d o[r] = dL/dloglam[t][s] * (Lmax - Lmin) * sig (1 - sig), zero on gaps.
__global__ void k_tcn_dout(const float* __restrict__ gll, const float* __restrict__ o, float* __restrict__ dout,
                           int T, int P, int64_t R, float lrange) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int s = (int)(r / (T + kGap)), t = (int)(r % (T + kGap));
  float g = 0.f;
  if (t < T) {
    const float sg = 1.f / (1.f + expf(-o[r]));
    g = gll[(size_t)t * P + s] * lrange * sg * (1.f - sg);
  }
  dout[r] = g;
}

// Layer-4 data gradient through the layer-3 ReLU: dh3[r][ci] = [a3 > 0] sum_k W4[ci][k] dout[r - k + 4].
__global__ void __launch_bounds__(128) k_tcn_l4_bwd(const float* __restrict__ dout, const __nv_bfloat16* __restrict__ w4,
                                                    const uint4* __restrict__ a3, uint4* __restrict__ dh3, int64_t R) {
  __shared__ float sw[kCh * kTaps];
  for (int i = threadIdx.x; i < kCh * kTaps; i += blockDim.x) sw[i] = __bfloat162float(w4[i]);
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  float g[kTaps];
#pragma unroll
  for (int k = 0; k < kTaps; ++k) {
    const int64_t rr = r - k + kHalf;
    g[k] = (rr >= 0 && rr < R) ? dout[rr] : 0.f;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint4 m = a3[r * 8 + j];
    const uint32_t mm[4] = {m.x, m.y, m.z, m.w};
    float f[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int ci = 8 * j + e;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) acc = fmaf(sw[ci * kTaps + k], g[k], acc);
      const float mv = (e & 1) ? bf16_hi(mm[e >> 1]) : bf16_lo(mm[e >> 1]);
      f[e] = mv > 0.f ? acc : 0.f;
    }
    dh3[r * 8 + j] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                                pack_bf16x2(f[6], f[7]));
  }
}

// Weight gradient of a 64 -> 64 layer: gW[co][ci][k] += sum_r dh[r][co] a[r + k - 4][ci],
// gb[co] += sum_r dh[r][co]. 256 threads = 16 x 16 blocks of (4 co x 4 ci), 9 taps each, in
// registers over all rows of the CTA's tiles; rows staged in shared memory (FP32).
constexpr int kWgRows = 64;
__global__ void __launch_bounds__(256, 1) k_wgrad64(const uint4* __restrict__ dh, const uint4* __restrict__ act,
                                                    float* __restrict__ gW, float* __restrict__ gb, int64_t R,
                                                    int n_tiles) {
  __shared__ float sdh[kWgRows][kCh + 4];
  __shared__ float sa[kWgRows + 2 * kHalf][kCh + 4];
  const int tid = threadIdx.x, cb = tid >> 4, ib = tid & 15;  // co block, ci block
  float acc[kTaps][4][4];
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kTaps; ++k)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[k][i][j] = 0.f;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * kWgRows;
    __syncthreads();
    for (int e = tid; e < kWgRows * 8; e += 256) {
      const int i = e >> 3, j = e & 7;
      const int64_t r = r0 + i;
      const uint4 u = r < R ? dh[r * 8 + j] : make_uint4(0, 0, 0, 0);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sdh[i][8 * j + 2 * q] = bf16_lo(uu[q]);
        sdh[i][8 * j + 2 * q + 1] = bf16_hi(uu[q]);
      }
    }
    for (int e = tid; e < (kWgRows + 2 * kHalf) * 8; e += 256) {
      const int i = e >> 3, j = e & 7;
      const int64_t r = r0 - kHalf + i;
      const uint4 u = (r >= 0 && r < R) ? act[r * 8 + j] : make_uint4(0, 0, 0, 0);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sa[i][8 * j + 2 * q] = bf16_lo(uu[q]);
        sa[i][8 * j + 2 * q + 1] = bf16_hi(uu[q]);
      }
    }
    __syncthreads();
    for (int i = 0; i < kWgRows; ++i) {
      float d[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) d[c] = sdh[i][4 * cb + c];
      if (ib == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) bacc[c] += d[c];
#pragma unroll
      for (int k = 0; k < kTaps; ++k) {
        const float4 av = *reinterpret_cast<const float4*>(&sa[i + k][4 * ib]);
        const float aa[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[k][c][j] = fmaf(d[c], aa[j], acc[k][c][j]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kTaps; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) atomicAdd(&gW[((4 * cb + c) * kCh + 4 * ib + j) * kTaps + k], acc[k][c][j]);
  if (ib == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) atomicAdd(&gb[4 * cb + c], bacc[c]);
}

// Weight gradient of layer 1 (2 -> 64): gW1[co][c][k] += sum_r dh1[r][co] in0[r + k - 4][c].
// Thread per (co, c) pair (128 threads), 9 taps.
__global__ void __launch_bounds__(128) k_wgrad_l1(const uint4* __restrict__ dh, const uint32_t* __restrict__ in0,
                                                  float* __restrict__ gW, float* __restrict__ gb, int64_t R,
                                                  int n_tiles) {
  __shared__ float sdh[kWgRows][kCh + 1];
  __shared__ float sin_[kWgRows + 2 * kHalf][2];
  const int tid = threadIdx.x, co = tid >> 1, c = tid & 1;
  float acc[kTaps];
  float bacc = 0.f;
#pragma unroll
  for (int k = 0; k < kTaps; ++k) acc[k] = 0.f;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * kWgRows;
    __syncthreads();
    for (int e = tid; e < kWgRows * 8; e += 128) {
      const int i = e >> 3, j = e & 7;
      const int64_t r = r0 + i;
      const uint4 u = r < R ? dh[r * 8 + j] : make_uint4(0, 0, 0, 0);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sdh[i][8 * j + 2 * q] = bf16_lo(uu[q]);
        sdh[i][8 * j + 2 * q + 1] = bf16_hi(uu[q]);
      }
    }
    for (int i = tid; i < kWgRows + 2 * kHalf; i += 128) {
      const int64_t r = r0 - kHalf + i;
      const uint32_t u = (r >= 0 && r < R) ? in0[r] : 0u;
      sin_[i][0] = bf16_lo(u);
      sin_[i][1] = bf16_hi(u);
    }
    __syncthreads();
    for (int i = 0; i < kWgRows; ++i) {
      const float d = sdh[i][co];
      if (c == 0) bacc += d;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) acc[k] = fmaf(d, sin_[i + k][c], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < kTaps; ++k) atomicAdd(&gW[(co * 2 + c) * kTaps + k], acc[k]);
  if (c == 0) atomicAdd(&gb[co], bacc);
}

// Weight gradient of layer 4 (64 -> 1): gW4[ci][k] += sum_r dout[r] a3[r + k - 4][ci].
__global__ void __launch_bounds__(64) k_wgrad_l4(const float* __restrict__ dout, const uint4* __restrict__ a3,
                                                 float* __restrict__ gW, float* __restrict__ gb, int64_t R,
                                                 int n_tiles) {
  __shared__ float sd[kWgRows];
  __shared__ float sa[kWgRows + 2 * kHalf][kCh + 1];
  const int ci = threadIdx.x;
  float acc[kTaps];
  float bacc = 0.f;
#pragma unroll
  for (int k = 0; k < kTaps; ++k) acc[k] = 0.f;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * kWgRows;
    __syncthreads();
    for (int i = ci; i < kWgRows; i += 64) sd[i] = (r0 + i < R) ? dout[r0 + i] : 0.f;
    for (int e = ci; e < (kWgRows + 2 * kHalf) * 8; e += 64) {
      const int i = e >> 3, j = e & 7;
      const int64_t r = r0 - kHalf + i;
      const uint4 u = (r >= 0 && r < R) ? a3[r * 8 + j] : make_uint4(0, 0, 0, 0);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sa[i][8 * j + 2 * q] = bf16_lo(uu[q]);
        sa[i][8 * j + 2 * q + 1] = bf16_hi(uu[q]);
      }
    }
    __syncthreads();
    for (int i = 0; i < kWgRows; ++i) {
      const float d = sd[i];
      if (ci == 0) bacc += d;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) acc[k] = fmaf(d, sa[i + k][ci], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < kTaps; ++k) atomicAdd(&gW[ci * kTaps + k], acc[k]);
  if (ci == 0) atomicAdd(&gb[0], bacc);
}

// ---------------------------------------------------------------------------------------
// FP32 master -> BF16 packed layouts.
__global__ void k_tcn_pack(const float* __restrict__ m, __nv_bfloat16* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kCh * 2 * kTaps) p[kPW1 + i] = __float2bfloat16_rn(m[kOW1 + i]);
  if (i < kCh * kTaps) p[kPW4 + i] = __float2bfloat16_rn(m[kOW4 + i]);
  if (i < 4 * kCh * 8) {  // W1 for the tensor cores: K index kk = 2 tap + c, zero beyond 18
    const int e = i & 7, co = (i >> 3) & 63, chunk = i >> 9, kk = 8 * chunk + e;
    p[kPW1T + i] = __float2bfloat16_rn(kk < 2 * kTaps ? m[kOW1 + (co * 2 + (kk & 1)) * kTaps + (kk >> 1)] : 0.f);
  }
  if (i < 16 * kCh) {  // W4 for the tensor cores: row = tap (zero beyond 8), column = ci
    const int ci = i & 63, tap = i >> 6;
    p[kPW4T + i] = __float2bfloat16_rn(tap < kTaps ? m[kOW4 + ci * kTaps + tap] : 0.f);
  }
  if (i < kCh * kCh * kTaps) {
    // plane index i = ((tap * 8 + chunk) * 64 + row) * 8 + e
    const int e = i & 7, row = (i >> 3) & 63, chunk = (i >> 9) & 7, tap = i >> 12;
    // forward: row = co, channel = ci = 8 chunk + e, tap as is
    const int co = row, ci = 8 * chunk + e;
    p[kPW2F + i] = __float2bfloat16_rn(m[kOW2 + (co * kCh + ci) * kTaps + tap]);
    p[kPW3F + i] = __float2bfloat16_rn(m[kOW3 + (co * kCh + ci) * kTaps + tap]);
    // data gradient: row = ci of the layer, channel = co = 8 chunk + e, tap flipped
    const int bci = row, bco = 8 * chunk + e, btap = kTaps - 1 - tap;
    p[kPW2B + i] = __float2bfloat16_rn(m[kOW2 + (bco * kCh + bci) * kTaps + btap]);
    p[kPW3B + i] = __float2bfloat16_rn(m[kOW3 + (bco * kCh + bci) * kTaps + btap]);
  }
}

// Adam (Kingma & Ba 2015) with bias correction; the gradient is cleared after use.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, float* __restrict__ g,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.f;
}

// gz = scale (z - target) elementwise; loss_sum += 0.5 scale sum (z - target)^2 (block sums).
__global__ void k_mse_grad(const float* __restrict__ z, const float* __restrict__ tg, float* __restrict__ gz,
                           float* __restrict__ loss, int64_t n, float scale) {
  __shared__ float red[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n) {
    const float d = z[i] - tg[i];
    gz[i] = scale * d;
    l = 0.5f * scale * d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x < 8) {
    float s = red[threadIdx.x];
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffu, s, o);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, s);
  }
}

}  // namespace ws

using namespace ws;

// ---------------------------------------------------------------------------------------
// C-ABI

namespace {

struct TcnScratch {
  uint32_t* in0;
  uint4 *a1, *a2, *a3, *dha, *dhb;
  float *o, *dout;
  unsigned* err;
};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t tcn_rows(const ws_tcn_batch* b) { return (int64_t)b->n_series * (b->T + kGap); }

size_t tcn_scratch_bytes(const ws_tcn_batch* b, int training, TcnScratch* s, void* base) {
  const int64_t R = tcn_rows(b);
  size_t off = 256;  // error word
  char* p = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* q = p ? p + off : nullptr;
    off += round256(bytes);
    return q;
  };
  TcnScratch t;
  t.err = p ? reinterpret_cast<unsigned*>(p) : nullptr;
  t.in0 = static_cast<uint32_t*>(take((size_t)R * 4));
  t.o = static_cast<float*>(take((size_t)R * 4));
  t.a1 = t.a2 = t.a3 = nullptr;
  if (training) {  // activations of every layer for the backward pass
    t.a1 = static_cast<uint4*>(take((size_t)R * 128));
    t.a2 = static_cast<uint4*>(take((size_t)R * 128));
    t.a3 = static_cast<uint4*>(take((size_t)R * 128));
    t.dha = static_cast<uint4*>(take((size_t)R * 128));
    t.dhb = static_cast<uint4*>(take((size_t)R * 128));
    t.dout = static_cast<float*>(take((size_t)R * 4));
  } else {
    t.dha = t.dhb = nullptr;
    t.dout = nullptr;
  }
  if (s) *s = t;
  return off;
}

int check_batch(const ws_tcn_batch* b) {
  if (b == nullptr) return set_error(WS_EINVAL, "batch is NULL");
  if (b->T < 1 || b->n_series < 0) return set_error(WS_EINVAL, "T >= 1 and n_series >= 0 required");
  if ((int64_t)b->n_series * (b->T + kGap) > ((int64_t)1 << 40)) return set_error(WS_EINVAL, "batch too large");
  if (!(b->log_lam_max > b->log_lam_min)) return set_error(WS_EINVAL, "log_lam_max must exceed log_lam_min");
  return WS_OK;
}

int conv_launch(int mode, const uint4* in, const void* wp, const float* bias, const uint4* mask, uint4* out,
                int64_t R, int T, unsigned* err, cudaStream_t st) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  // + 16 KB of slack: every operand window the descriptors can describe stays inside the
  // allocation even under the other reading of LBO/SBO (a layout error then gives wrong
  // numbers, which the tests catch, rather than an out-of-range shared-memory access)
  const size_t smem = (size_t)kActBytes + kWBytes + 16 + 16384;
  const void* kern = mode == CONV_FWD ? (const void*)k_conv64<CONV_FWD> : (const void*)k_conv64<CONV_BWD>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return set_error(WS_ECUDA, "conv64: shared memory attribute");
  ConvArgs a;
  a.in = in;
  a.wp = static_cast<const uint4*>(wp);
  a.bias = bias;
  a.mask = mask;
  a.out = out;
  a.R = R;
  a.T = T;
  a.n_tiles = (int)((R + kTileRows - 1) / kTileRows);
  a.err = err;
  const int grid = std::max(1, std::min(a.n_tiles, di.sm_count));
  if (mode == CONV_FWD)
    k_conv64<CONV_FWD><<<grid, kConvThreads, smem, st>>>(a);
  else
    k_conv64<CONV_BWD><<<grid, kConvThreads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "conv64 launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

int grid_for(int64_t n, int block) { return (int)std::max<int64_t>(1, (n + block - 1) / block); }

}  // namespace

extern "C" size_t ws_tcn_scratch_size(const ws_tcn_batch* b, int training) {
  if (check_batch(b) != WS_OK) return 0;
  return tcn_scratch_bytes(b, training, nullptr, nullptr);
}

extern "C" int ws_tcn_pack(const float* master, void* packed, void* stream) {
  if (master == nullptr || packed == nullptr) return set_error(WS_EINVAL, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_tcn_pack<<<grid_for(kCh * kCh * kTaps, 256), 256, 0, st>>>(master, static_cast<__nv_bfloat16*>(packed));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "pack launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

extern "C" int ws_tcn_forward(const ws_tcn_batch* b, const void* packed, const float* master, const float* x,
                              const float* w, float* lam, float* loglam, void* scratch, size_t scratch_bytes,
                              int training, void* stream) {
  int rc = check_batch(b);
  if (rc != WS_OK) return rc;
  if (!packed || !master || !x || !w || !lam || !scratch) return set_error(WS_EINVAL, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(scratch) & 255u) != 0) return set_error(WS_EINVAL, "scratch must be 256-byte aligned");
  TcnScratch s;
  const size_t need = tcn_scratch_bytes(b, training, &s, scratch);
  if (scratch_bytes < need) return set_error(WS_ENOMEM_WS, "scratch too small: %zu < %zu", scratch_bytes, need);
  if (b->n_series == 0) return WS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t R = tcn_rows(b);
  const __nv_bfloat16* pk = static_cast<const __nv_bfloat16*>(packed);
  k_tcn_in<<<grid_for(R, 256), 256, 0, st>>>(x, w, s.in0, b->T, b->n_series, R);
  DeviceInfo di;
  if ((rc = device_info(di)) != WS_OK) return rc;
  if (cudaFuncSetAttribute(k_tcn_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmem) != cudaSuccess)
    return set_error(WS_ECUDA, "tcn: shared memory attribute");
  FusedArgs fa;
  fa.in0 = s.in0;
  fa.w1t = reinterpret_cast<const uint4*>(pk + kPW1T);
  fa.w2 = reinterpret_cast<const uint4*>(pk + kPW2F);
  fa.w3 = reinterpret_cast<const uint4*>(pk + kPW3F);
  fa.w4t = pk + kPW4T;
  fa.master = master;
  fa.lam = lam;
  fa.loglam = loglam;
  fa.o_out = s.o;
  fa.a1 = s.a1;
  fa.a2 = s.a2;
  fa.a3 = s.a3;
  fa.R = R;
  fa.T = b->T;
  fa.P = b->n_series;
  fa.n_tiles = (int)((R + kFuseUseful - 1) / kFuseUseful);
  fa.lmin = b->log_lam_min;
  fa.lmax = b->log_lam_max;
  fa.err = s.err;
  k_tcn_fused<<<std::max(1, std::min(fa.n_tiles, di.sm_count)), kFuseThreads, kFSmem, st>>>(fa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "tcn forward launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

extern "C" int ws_tcn_backward(const ws_tcn_batch* b, const void* packed, const float* g_loglam, float* grad,
                               void* scratch, size_t scratch_bytes, void* stream) {
  int rc = check_batch(b);
  if (rc != WS_OK) return rc;
  if (!packed || !g_loglam || !grad || !scratch) return set_error(WS_EINVAL, "NULL argument");
  TcnScratch s;
  const size_t need = tcn_scratch_bytes(b, 1, &s, scratch);
  if (scratch_bytes < need) return set_error(WS_ENOMEM_WS, "scratch too small: %zu < %zu", scratch_bytes, need);
  if (b->n_series == 0) return WS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t R = tcn_rows(b);
  const __nv_bfloat16* pk = static_cast<const __nv_bfloat16*>(packed);
  DeviceInfo di;
  if ((rc = device_info(di)) != WS_OK) return rc;
  const int wg_tiles = (int)((R + kWgRows - 1) / kWgRows);
  const int wg_grid = std::max(1, std::min(wg_tiles, di.sm_count * 2));
  k_tcn_dout<<<grid_for(R, 256), 256, 0, st>>>(g_loglam, s.o, s.dout, b->T, b->n_series, R,
                                               b->log_lam_max - b->log_lam_min);
  k_wgrad_l4<<<wg_grid, 64, 0, st>>>(s.dout, s.a3, grad + kOW4, grad + kOB4, R, wg_tiles);
  k_tcn_l4_bwd<<<grid_for(R, 128), 128, 0, st>>>(s.dout, pk + kPW4, s.a3, s.dha, R);  // dh3
  k_wgrad64<<<wg_grid, 256, 0, st>>>(s.dha, s.a2, grad + kOW3, grad + kOB3, R, wg_tiles);
  if ((rc = conv_launch(CONV_BWD, s.dha, pk + kPW3B, nullptr, s.a2, s.dhb, R, b->T, s.err, st)) != WS_OK) return rc;
  k_wgrad64<<<wg_grid, 256, 0, st>>>(s.dhb, s.a1, grad + kOW2, grad + kOB2, R, wg_tiles);
  if ((rc = conv_launch(CONV_BWD, s.dhb, pk + kPW2B, nullptr, s.a1, s.dha, R, b->T, s.err, st)) != WS_OK) return rc;
  k_wgrad_l1<<<wg_grid, 128, 0, st>>>(s.dha, s.in0, grad + kOW1, grad + kOB1, R, wg_tiles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "tcn backward launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

extern "C" int ws_tcn_conv64(const void* in, const void* wplanes, const float* bias, const void* mask, void* out,
                             int64_t rows, int32_t T, int32_t mode, void* err_word, void* stream) {
  if (!in || !wplanes || !out || !err_word || rows < 0 || T < 1) return set_error(WS_EINVAL, "invalid arguments");
  if (mode == CONV_FWD && bias == nullptr) return set_error(WS_EINVAL, "forward mode needs the bias");
  if (mode == CONV_BWD && mask == nullptr) return set_error(WS_EINVAL, "data-gradient mode needs the mask");
  if (mode != CONV_FWD && mode != CONV_BWD) return set_error(WS_EINVAL, "mode must be 0 or 1");
  if (rows == 0) return WS_OK;
  return conv_launch(mode, static_cast<const uint4*>(in), wplanes, bias, static_cast<const uint4*>(mask),
                     static_cast<uint4*>(out), rows, T, static_cast<unsigned*>(err_word),
                     static_cast<cudaStream_t>(stream));
}

extern "C" int ws_adam_step(float* params, float* m, float* v, float* grad, int64_t n, int32_t step, float lr,
                            float beta1, float beta2, float eps, void* stream) {
  if (!params || !m || !v || !grad || n < 0 || step < 1) return set_error(WS_EINVAL, "invalid Adam arguments");
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_adam<<<grid_for(n, 256), 256, 0, st>>>(params, m, v, grad, n, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "adam launch: %s", cudaGetErrorString(e));
  return WS_OK;
}

extern "C" int ws_mse_grad(const float* z, const float* target, float* gz, float* loss_sum, int64_t n, float scale,
                           void* stream) {
  if (!z || !target || !gz || n < 0) return set_error(WS_EINVAL, "invalid arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_mse_grad<<<grid_for(n, 256), 256, 0, st>>>(z, target, gz, loss_sum, n, scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "mse launch: %s", cudaGetErrorString(e));
  return WS_OK;
}
