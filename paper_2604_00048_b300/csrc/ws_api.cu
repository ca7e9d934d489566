// C-ABI entry points of libws_b300.so (declared in include/ws.h): argument
// validation, workspace sizing, tensor-map encoding, band groups and launch.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include <algorithm>
#include <cmath>

#include "ws_internal.h"

namespace ws {

static thread_local int g_err_code = WS_OK;
static thread_local char g_err_msg[512] = "";

int set_error(int code, const char* fmt, ...) {
  g_err_code = code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err_msg, sizeof(g_err_msg), fmt, ap);
  va_end(ap);
  return code;
}

static void clear_error() {
  g_err_code = WS_OK;
  g_err_msg[0] = '\0';
}

int device_info(DeviceInfo& info) {
  static DeviceInfo cache[64];
  static std::once_flag once[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return set_error(WS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  std::call_once(once[dev], [dev]() {
    cudaDeviceGetAttribute(&cache[dev].sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&cache[dev].smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  });
  info = cache[dev];
  if (info.sm_count <= 0 || info.smem_optin <= 0 || info.smem_per_sm <= 0) return set_error(WS_ECUDA, "device attributes unavailable");
  return WS_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int make_tmap(CUtensorMap* map, int dtype, int rank, const void* base, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box) {
  auto fn = encode_fn();
  if (fn == nullptr) return WS_EUNSUPPORTED;
  cuuint64_t gd[3];
  cuuint64_t gs[2];
  cuuint32_t bx[3], es[3] = {1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
  }
  for (int i = 0; i + 1 < rank; ++i) gs[i] = strides_bytes[i];
  CUresult r = fn(map, dtype == WS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WS_OK : WS_EUNSUPPORTED;
}

static int validate_problem(const ws_problem* pb) {
  if (pb == nullptr) return set_error(WS_EINVAL, "problem is NULL");
  if (pb->n_series < 0 || pb->n_series > 0x7fffffffLL) return set_error(WS_EINVAL, "n_series out of range");
  if (pb->T < 0) return set_error(WS_EINVAL, "T < 0");
  if (pb->d < 1 || pb->d > 4) return set_error(WS_EINVAL, "d must be 1..4 (got %d)", pb->d);
  if (pb->n_bands < 1) return set_error(WS_EINVAL, "n_bands must be >= 1");
  if (pb->layout != WS_LAYOUT_TILE) return set_error(WS_EINVAL, "layout must be WS_LAYOUT_TILE");
  if (pb->dtype != WS_F32 && pb->dtype != WS_F64) return set_error(WS_EINVAL, "dtype must be WS_F32 or WS_F64");
  if (pb->lam_mode != WS_LAM_PER_DAY && pb->lam_mode != WS_LAM_SCALAR)
    return set_error(WS_EINVAL, "lam_mode must be WS_LAM_PER_DAY or WS_LAM_SCALAR");
  return WS_OK;
}

static int elem_size(const ws_problem& pb) { return pb.dtype == WS_F64 ? 8 : 4; }

// Largest supported band-group size <= want for this dtype/order.
static int group_size(const ws_problem& pb, int want) {
  if (pb.dtype == WS_F64) return (pb.d == 2 && want >= 2) ? 2 : 1;
#ifdef WS_FAST_BUILD
  return want >= 4 ? 4 : (want >= 2 ? 2 : 1);
#else
  return want > kNbMax ? kNbMax : want;
#endif
}

static int extra_planes(int d) { return d > 2 ? d - 2 : 0; }

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

static int extra_planes_mode(int mode, int d) { return mode == MODE_ADJ ? d : extra_planes(d); }

static size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

// Checkpoint bytes of the tile kernels over all band groups and modes (the adjoint with
// and without the fused MSE loss, whose extra staged rows may shorten its chunks).
static int tile_ckpt_bytes(const ws_problem& pb, size_t& bytes) {
  bytes = 0;
  const int modes[4] = {MODE_SMOOTH, MODE_RAW, MODE_ADJ, MODE_ADJ + 8};  // + 8: with the MSE loss
  for (int mode : modes) {
    for (int b0 = 0; b0 < pb.n_bands;) {
      const int nb = group_size(pb, pb.n_bands - b0);
      TileCfg cfg;
      int rc = plan_tile(pb, mode & 7, nb, cfg, mode >> 3);
      if (rc != WS_OK) return rc;
      const size_t need = (size_t)cfg.grid * cfg.nch * cfg.fields * cfg.NP * elem_size(pb);
      if (need > bytes) bytes = need;
      b0 += nb;
    }
  }
  bytes = round256(bytes);
  return WS_OK;
}

static size_t resid_bytes(const ws_problem& pb) {
  return round256((size_t)pb.T * pb.n_bands * pb.n_series * elem_size(pb));
}

static int check_workspace(const ws_problem& pb, void* workspace, size_t ws_bytes, size_t extra,
                           size_t& ck_bytes) {
  int rc = tile_ckpt_bytes(pb, ck_bytes);
  if (rc != WS_OK) return rc;
  if (workspace == nullptr) return set_error(WS_EINVAL, "workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < kHeaderBytes + ck_bytes + extra)
    return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, kHeaderBytes + ck_bytes + extra);
  return WS_OK;
}

// The masked-MSE loss fused into the adjoint (rhs is then the target).
struct AdjMse {
  const void* mask;  // [T][P] or NULL
  double scale;
  void* loss;        // [P] or NULL
};

// One tile-kernel mode over every band group of the problem.
static int run_tile(const ws_problem& P, int mode, const void* rhs, const void* w, const void* lam,
                    const void* zin, const void* g0, void* out, void* out2, void* factor, uint8_t* status,
                    int accum, int adj_flags, void* workspace, cudaStream_t st, void* df_base = nullptr,
                    const AdjMse* mse = nullptr) {
  // adj_flags (MODE_ADJ): bit 0 gradient in log lambda, bit 1 output g instead of W g
  // pointer contract of each mode (an inconsistent internal call is an error, never a fault)
  if (rhs == nullptr || w == nullptr || lam == nullptr) return set_error(WS_EINVAL, "tile: missing input");
  if (mode != MODE_ADJ && out == nullptr) return set_error(WS_EINVAL, "tile: missing output");
  if (mode == MODE_ADJ && zin == nullptr) return set_error(WS_EINVAL, "tile: adjoint needs z");
  if (mode == MODE_ADJ && accum && g0 == nullptr) return set_error(WS_EINVAL, "tile: accumulation needs g0");
  if (mode == MODE_SMOOTH && accum) return set_error(WS_EINVAL, "tile: smooth does not accumulate");
  const int es = elem_size(P);
  const bool per_day = P.lam_mode == WS_LAM_PER_DAY;
  // the array staged into the Z region in pass 2: z (adjoint) or z0 = out (accumulating RAW)
  const void* zin_stage = mode == MODE_ADJ ? zin : ((mode == MODE_RAW && accum) ? out : nullptr);
  const bool has_m = mse != nullptr && mse->mask != nullptr;
  const bool tma_ok = ((size_t)P.n_series * es) % 16 == 0 && aligned16(rhs) && aligned16(w) &&
                      (out == nullptr || aligned16(out)) && (!per_day || aligned16(lam)) &&
                      (zin_stage == nullptr || aligned16(zin_stage)) && (!has_m || aligned16(mse->mask));
  for (int b0 = 0; b0 < P.n_bands;) {
    const int nb = group_size(P, P.n_bands - b0);
    TileCfg cfg;
    int rc = plan_tile(P, mode, nb, cfg, mse != nullptr ? 1 : 0);
    if (rc != WS_OK) return rc;
    CUtensorMap maps[6];
    memset(maps, 0, sizeof(maps));
    bool tma = tma_ok;
    if (tma) {
      const uint64_t Pn = (uint64_t)P.n_series, B = (uint64_t)P.n_bands, T = (uint64_t)P.T;
      const uint64_t dx[3] = {Pn, B, T}, sx[2] = {Pn * es, B * Pn * es};
      const uint32_t bx[3] = {(uint32_t)cfg.NP, (uint32_t)nb, (uint32_t)cfg.C};
      const uint64_t d2[2] = {Pn, T}, s2[1] = {Pn * es};
      const uint32_t bw[2] = {(uint32_t)cfg.NP, (uint32_t)(cfg.C + P.d)};
      const uint32_t bl[2] = {(uint32_t)cfg.NP, (uint32_t)cfg.C};
      tma = make_tmap(&maps[0], P.dtype, 3, rhs, dx, sx, bx) == WS_OK &&
            make_tmap(&maps[1], P.dtype, 2, w, d2, s2, bw) == WS_OK &&
            (!per_day || make_tmap(&maps[2], P.dtype, 2, lam, d2, s2, bl) == WS_OK) &&
            (out == nullptr || make_tmap(&maps[3], P.dtype, 3, out, dx, sx, bx) == WS_OK) &&
            (zin_stage == nullptr || make_tmap(&maps[4], P.dtype, 3, zin_stage, dx, sx, bx) == WS_OK) &&
            (!has_m || make_tmap(&maps[5], P.dtype, 2, mse->mask, d2, s2, bl) == WS_OK);
    }
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.T = P.T;
    a.P = (int)P.n_series;
    a.B = P.n_bands;
    a.b0 = b0;
    a.C = cfg.C;
    a.NP = cfg.NP;
    a.nch = cfg.nch;
    a.ck_group = cfg.ck_group;
    a.n_tiles = cfg.n_tiles;
    a.lam_scalar = per_day ? 0 : 1;
    a.tma = tma ? 1 : 0;
    a.write_status = b0 == 0;
    a.x = rhs;
    a.w = w;
    a.lam = lam;
    a.zin = zin_stage;
    a.g0 = g0;
    a.out = out;
    a.out2 = out2;
    a.factor = factor;
    a.status = status;
    a.ckpt = static_cast<char*>(workspace) + kHeaderBytes;
    a.err = static_cast<unsigned*>(workspace);
    a.stage_elems = cfg.stage_elems;
    a.grad_loglam = adj_flags & 1;
    a.raw_g = (adj_flags >> 1) & 1;
    a.accum = accum;
    if (df_base != nullptr) {
      char* slots = nullptr;
      adj_df_layout(P, df_base, &a.df_mark, &a.df_count, &a.df_list, &slots);
    }
    if (mse != nullptr) {
      a.mse = 1;
      a.mask = mse->mask;
      a.mse_scale = mse->scale;
      a.loss = mse->loss;
    }
    rc = launch_tile(P, mode, nb, cfg, a, maps, st);
    if (rc != WS_OK) return rc;
    b0 += nb;
  }
  return WS_OK;
}

// Smoothing of one tile problem (the ragged plan's length classes): validation is the
// caller's; the workspace is tile_workspace_bytes(P) long, 256-byte aligned, header zeroed.
int tile_smooth(const ws_problem& P, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                void* workspace, cudaStream_t st) {
  return run_tile(P, MODE_SMOOTH, x, w, lam, nullptr, nullptr, z, nullptr, nullptr, status, 0, 0, workspace, st);
}

// One refinement step of a tile problem's solution z in place (the ragged plan's length
// classes): r = W x - Omega z (double-word residual) into r, then z += Omega^{-1} r.
// Workspace as tile_smooth's.
int tile_refine(const ws_problem& P, const void* x, const void* w, const void* lam, void* z, void* r,
                void* workspace, cudaStream_t st) {
  int rc = launch_residual(P, x, w, lam, z, r, 0, static_cast<unsigned*>(workspace), st);
  if (rc != WS_OK) return rc;
  return run_tile(P, MODE_RAW, r, w, lam, nullptr, nullptr, z, nullptr, nullptr, nullptr, 1, 0, workspace, st);
}

size_t tile_workspace_bytes(const ws_problem& P) {
  size_t ck = 0;
  if (tile_ckpt_bytes(P, ck) != WS_OK) return 0;
  return kHeaderBytes + ck;
}

// GCV on sample times (ws_gcv.cu): the grid search with the rows of D formed from t.
int gcv_plan_dates(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes);
int launch_gcv_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const float* grid_vals,
                     int n_grid, float* lam_best, float* scores, void* ckpt, cudaStream_t st);

// Posterior spread on sample times (ws_post.cu): the diagonal kernel with the rows of D
// formed from t.
int post_plan_dates(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes);
int launch_posterior_dates(const ws_problem& pb, const void* t, const void* x, const void* w, const void* lam,
                           const void* z, void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den,
                           cudaStream_t st);

// Refinement on sample times (ws_dates.cu): residual into r, then the correction solve
// accumulated onto z in place.
int launch_dates_refine(const ws_problem& pb, const void* t, const void* x, const void* w, const void* lam, void* z,
                        void* r, void* ckpt, cudaStream_t st);

}  // namespace ws

using namespace ws;

// Adjoint with a stored factor: one kernel per band group, whose forward sweep writes yhat
// into the refinement region of the workspace and whose backward sweep forms g with gx and
// glam. (status is left untouched: ws_factor set it.)
static int ws_adjoint_factored(const ws_problem* pb, const void* factor, const void* w, const void* lam, const void* z,
                               const void* gz, void* gx, void* glam, uint32_t flags, uint8_t* status,
                               void* workspace, size_t ws_bytes, void* stream) {
  (void)status;
  const ws_problem& P = *pb;
  if (flags & WS_REFINE_ADJOINT) return set_error(WS_EINVAL, "refinement needs the recomputed factor (factor = NULL)");
  size_t ck_bytes = 0;
  int rc = check_workspace(P, workspace, ws_bytes, resid_bytes(P), ck_bytes);
  if (rc != WS_OK) return rc;
  void* gs = static_cast<char*>(workspace) + kHeaderBytes + ck_bytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return launch_factored(2, P, factor, nullptr, w, lam, gz, nullptr, z, gs, gx, glam, nullptr, 0,
                         ((flags & WS_GRAD_LOGLAM) ? 1 : 0) | ((flags & WS_ADJ_RAW_G) ? 2 : 0), st);
}

// ws_posterior's scratch after the header: checkpoints, then n - tr H per series.
static int post_bytes(const ws_problem& pb, size_t& bytes) {
  int grid = 0, nch = 0;
  size_t ck = 0;
  int rc = post_plan(pb, grid, nch, ck);
  if (rc != WS_OK) return rc;
  bytes = round256(ck) + round256((size_t)pb.n_series * elem_size(pb));
  return WS_OK;
}

extern "C" size_t ws_workspace_size(const ws_problem* pb, uint32_t flags) {
  clear_error();
  if (validate_problem(pb) != WS_OK) return 0;
  size_t ck = 0;
  if (pb->n_series == 0 || pb->T == 0) return kHeaderBytes;
  if (tile_ckpt_bytes(*pb, ck) != WS_OK) return 0;
  const size_t extra = (flags & WS_REFINE_ADJOINT) ? 2 * resid_bytes(*pb) + adj_df_bytes(*pb)
                                                  : ((flags & WS_REFINE) ? resid_bytes(*pb) : 0);
  size_t need = kHeaderBytes + ck + extra;
  if (flags & WS_GCV) {  // the grid search's checkpoints, then the final smooth, reuse one region
    int grid = 0, nch = 0;
    size_t gck = 0;
    if (gcv_plan(*pb, grid, nch, gck) != WS_OK) return 0;
    need = std::max(need, kHeaderBytes + round256(gck));
  }
  if ((flags & WS_GCV) && (flags & WS_DATES)) {
    int grid = 0, nch = 0;
    size_t gck = 0;
    if (gcv_plan_dates(*pb, grid, nch, gck) != WS_OK) return 0;
    need = std::max(need, kHeaderBytes + round256(gck));
  }
  if (flags & WS_DATES) {
    size_t dck = 0;
    size_t dck2 = 0;
    if (dates_plan(*pb, false, dck) != WS_OK || dates_plan(*pb, true, dck2) != WS_OK) return 0;
    dck = std::max(dck, dck2);
    need = std::max(need, kHeaderBytes + round256(dck) + ((flags & WS_REFINE) ? resid_bytes(*pb) : 0));
  }
  if (flags & WS_PARTITIONED) need = std::max(need, kHeaderBytes + part_workspace_bytes(*pb));
  if (flags & WS_POSTERIOR) {
    size_t pck = 0;
    if (post_bytes(*pb, pck) != WS_OK) return 0;
    need = std::max(need, kHeaderBytes + pck);
  }
  return need;
}

extern "C" int ws_smooth_dates(const ws_problem* pb, const void* t, const void* x, const void* w, const void* lam,
                               void* z, uint8_t* status, uint32_t flags, void* workspace, size_t ws_bytes,
                               void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~WS_REFINE) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (P.T == 0) {
    if (status != nullptr && cudaMemsetAsync(status, 0, (size_t)P.n_series, st) != cudaSuccess)
      return set_error(WS_ECUDA, "status memset failed");
    return WS_OK;
  }
  if (!t || !x || !w || !lam || !z) return set_error(WS_EINVAL, "t, x, w, lam and z must be non-NULL");
  const int es = elem_size(P);
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * es, nd = (size_t)P.T * P.n_series * es;
  const size_t nl = P.lam_mode == WS_LAM_SCALAR ? (size_t)P.n_series * es : nd;
  if (overlaps(z, nx, x, nx) || overlaps(z, nx, t, nd) || overlaps(z, nx, w, nd) || overlaps(z, nx, lam, nl))
    return set_error(WS_EINVAL, "z must not overlap the inputs");
  size_t ck = 0;
  rc = dates_plan(P, false, ck);
  if (rc != WS_OK) return rc;
  const bool refine = (flags & WS_REFINE) != 0;
  const size_t need = kHeaderBytes + round256(ck) + (refine ? resid_bytes(P) : 0);
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  char* ckpt = static_cast<char*>(workspace) + kHeaderBytes;
  rc = launch_dates(P, false, t, x, w, lam, z, nullptr, nullptr, 0, status, ckpt, st);
  if (rc != WS_OK || !refine) return rc;
  return launch_dates_refine(P, t, x, w, lam, z, ckpt + round256(ck), ckpt, st);
}

extern "C" int ws_smooth_dates_adjoint(const ws_problem* pb, const void* t, const void* w, const void* lam,
                                       const void* z, const void* gz, void* gx, void* glam, uint32_t flags,
                                       uint8_t* status, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~WS_GRAD_LOGLAM) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (P.T == 0) {
    if (status != nullptr && cudaMemsetAsync(status, 0, (size_t)P.n_series, st) != cudaSuccess)
      return set_error(WS_ECUDA, "status memset failed");
    if (glam != nullptr && P.lam_mode == WS_LAM_SCALAR &&
        cudaMemsetAsync(glam, 0, (size_t)P.n_series * elem_size(P), st) != cudaSuccess)
      return set_error(WS_ECUDA, "glam memset failed");
    return WS_OK;
  }
  if (!t || !w || !lam || !z || !gz || !gx) return set_error(WS_EINVAL, "t, w, lam, z, gz and gx must be non-NULL");
  const int es = elem_size(P);
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * es, nd = (size_t)P.T * P.n_series * es;
  const size_t nl = P.lam_mode == WS_LAM_SCALAR ? (size_t)P.n_series * es : nd;
  if (overlaps(gx, nx, gz, nx) || overlaps(gx, nx, z, nx) || overlaps(gx, nx, t, nd) || overlaps(gx, nx, w, nd) ||
      overlaps(gx, nx, lam, nl))
    return set_error(WS_EINVAL, "gx must not overlap the inputs");
  if (glam != nullptr && (overlaps(glam, nl, gz, nx) || overlaps(glam, nl, z, nx) || overlaps(glam, nl, gx, nx) ||
                          overlaps(glam, nl, lam, nl) || overlaps(glam, nl, w, nd) || overlaps(glam, nl, t, nd)))
    return set_error(WS_EINVAL, "glam must not overlap the inputs or gx");
  size_t ck = 0;
  rc = dates_plan(P, true, ck);
  if (rc != WS_OK) return rc;
  const size_t need = kHeaderBytes + round256(ck);
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  return launch_dates(P, true, t, gz, w, lam, gx, z, glam, (flags & WS_GRAD_LOGLAM) ? 1 : 0, status,
                      static_cast<char*>(workspace) + kHeaderBytes, st);
}

extern "C" int ws_weight_grad(const ws_problem* pb, const void* x, const void* w, const void* z, void* g,
                              void* gx, void* gw, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  const ws_problem& P = *pb;
  if (P.n_series == 0 || P.T == 0) return WS_OK;
  if (!x || !w || !z || !g || !gw) return set_error(WS_EINVAL, "x, w, z, g and gw must be non-NULL");
  const int es = elem_size(P);
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * es, nd = (size_t)P.T * P.n_series * es;
  if (gx != nullptr && gx != g && overlaps(gx, nx, g, nx))
    return set_error(WS_EINVAL, "gx must be g itself or not overlap it");
  const void* ins[4] = {x, w, z, g};
  const size_t nin[4] = {nx, nd, nx, nx};
  for (int i = 0; i < 4; ++i)
    if (overlaps(gw, nd, ins[i], nin[i])) return set_error(WS_EINVAL, "gw must not overlap the inputs");
  if (gx != nullptr && (overlaps(gx, nx, x, nx) || overlaps(gx, nx, w, nd) || overlaps(gx, nx, z, nx) ||
                        overlaps(gx, nx, gw, nd)))
    return set_error(WS_EINVAL, "gx must not overlap x, w, z or gw");
  return launch_wgrad(P, x, w, z, g, gx, gw, static_cast<cudaStream_t>(stream));
}

static int posterior_impl(const ws_problem* pb, const void* t_dates, const void* x, const void* w, const void* lam, const void* z,
                            void* diag, void* sigma2, void* sd, uint8_t* status, void* workspace, size_t ws_bytes,
                            void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  const int es = elem_size(P);
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * es, nd = (size_t)P.T * P.n_series * es;
  const size_t ns = (size_t)P.n_bands * P.n_series * es;
  if (!sigma2) return set_error(WS_EINVAL, "sigma2 must be non-NULL");
  if (P.T == 0) {  // no days: no valid observation, no posterior
    if (cudaMemsetAsync(sigma2, 0, ns, st) != cudaSuccess ||
        (status != nullptr && cudaMemsetAsync(status, WS_SERIES_NOT_PD, (size_t)P.n_series, st) != cudaSuccess))
      return set_error(WS_ECUDA, "memset failed");
    return WS_OK;
  }
  if (!x || !w || !lam || !z || !diag) return set_error(WS_EINVAL, "x, w, lam, z and diag must be non-NULL");
  const bool dt = t_dates != nullptr;
  const size_t nl = P.lam_mode == WS_LAM_SCALAR ? (size_t)P.n_series * es : nd;
  const void* ins[4] = {x, w, lam, z};
  const size_t nin[4] = {nx, nd, nl, nx};
  for (int i = 0; i < 4; ++i) {
    if (overlaps(diag, nd, ins[i], nin[i]) || overlaps(sigma2, ns, ins[i], nin[i]) ||
        (sd != nullptr && overlaps(sd, nx, ins[i], nin[i])))
      return set_error(WS_EINVAL, "diag, sigma2 and sd must not overlap the inputs");
  }
  if (overlaps(diag, nd, sigma2, ns) || (sd != nullptr && (overlaps(sd, nx, diag, nd) || overlaps(sd, nx, sigma2, ns))))
    return set_error(WS_EINVAL, "diag, sigma2 and sd must not overlap each other");
  size_t need = 0;
  rc = post_bytes(P, need);
  if (rc != WS_OK) return rc;
  need += kHeaderBytes;
  if (dt && overlaps(t_dates, nd, diag, nd)) return set_error(WS_EINVAL, "diag must not overlap t");
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  int grid = 0, nch = 0;
  size_t ck = 0;
  rc = dt ? post_plan_dates(P, grid, nch, ck) : post_plan(P, grid, nch, ck);
  if (rc != WS_OK) return rc;
  char* base = static_cast<char*>(workspace) + kHeaderBytes;
  return launch_posterior_dates(P, t_dates, x, w, lam, z, diag, sigma2, sd, status, base, base + round256(ck), st);
}


extern "C" int ws_posterior(const ws_problem* pb, const void* x, const void* w, const void* lam, const void* z,
                            void* diag, void* sigma2, void* sd, uint8_t* status, void* workspace, size_t ws_bytes,
                            void* stream) {
  return posterior_impl(pb, nullptr, x, w, lam, z, diag, sigma2, sd, status, workspace, ws_bytes, stream);
}

extern "C" int ws_posterior_dates(const ws_problem* pb, const void* t, const void* x, const void* w, const void* lam,
                                  const void* z, void* diag, void* sigma2, void* sd, uint8_t* status,
                                  void* workspace, size_t ws_bytes, void* stream) {
  if (pb != nullptr && pb->n_series > 0 && pb->T > 0 && t == nullptr) {
    clear_error();
    return set_error(WS_EINVAL, "t must be non-NULL");
  }
  return posterior_impl(pb, t, x, w, lam, z, diag, sigma2, sd, status, workspace, ws_bytes, stream);
}

extern "C" int ws_gcv_smooth(const ws_problem* pb, const void* x, const void* w, const float* lam_grid, int n_grid,
                             void* z, float* lam_best, float* scores, uint8_t* status, uint32_t flags,
                             void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~WS_REFINE) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  if (pb->dtype != WS_F32) return set_error(WS_EUNSUPPORTED, "GCV grid search: FP32 only");
  if (pb->n_bands != 1) return set_error(WS_EUNSUPPORTED, "GCV grid search: one band");
  if (lam_grid == nullptr || n_grid < 1 || n_grid > 16) return set_error(WS_EINVAL, "n_grid must be 1..16");
  for (int g = 0; g < n_grid; ++g)
    if (!(lam_grid[g] > 0.f) || !std::isfinite(lam_grid[g]))
      return set_error(WS_EINVAL, "lam_grid[%d] must be finite and > 0", g);
  ws_problem P = *pb;
  P.lam_mode = WS_LAM_SCALAR;  // the final smooth takes lam_best per series
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (!x || !w || !z || !lam_best) return set_error(WS_EINVAL, "x, w, z and lam_best must be non-NULL");
  if (P.T == 0) return ws_smooth_batch(&P, x, w, lam_best, z, nullptr, status, 0, workspace, ws_bytes, stream);
  const size_t need = ws_workspace_size(&P, WS_GCV | (flags & WS_REFINE));
  if (need == 0) return WS_ECUDA;
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  rc = launch_gcv(P, x, w, lam_grid, n_grid, lam_best, scores, static_cast<char*>(workspace) + kHeaderBytes, st);
  if (rc != WS_OK) return rc;
  return ws_smooth_batch(&P, x, w, lam_best, z, nullptr, status, flags & WS_REFINE, workspace, ws_bytes, stream);
}

extern "C" int ws_gcv_smooth_dates(const ws_problem* pb, const void* t, const void* x, const void* w,
                                   const float* lam_grid, int n_grid, void* z, float* lam_best, float* scores,
                                   uint8_t* status, uint32_t flags, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~WS_REFINE) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  if (pb->dtype != WS_F32) return set_error(WS_EUNSUPPORTED, "GCV grid search: FP32 only");
  if (pb->n_bands != 1) return set_error(WS_EUNSUPPORTED, "GCV grid search: one band");
  if (lam_grid == nullptr || n_grid < 1 || n_grid > 16) return set_error(WS_EINVAL, "n_grid must be 1..16");
  for (int g = 0; g < n_grid; ++g)
    if (!(lam_grid[g] > 0.f) || !std::isfinite(lam_grid[g]))
      return set_error(WS_EINVAL, "lam_grid[%d] must be finite and > 0", g);
  ws_problem P = *pb;
  P.lam_mode = WS_LAM_SCALAR;  // the final smooth takes lam_best per series
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (!t || !x || !w || !z || !lam_best) return set_error(WS_EINVAL, "t, x, w, z and lam_best must be non-NULL");
  if (P.T == 0) return ws_smooth_dates(&P, t, x, w, lam_best, z, status, 0, workspace, ws_bytes, stream);
  size_t gck = 0;
  int grid = 0, nch = 0;
  rc = gcv_plan_dates(P, grid, nch, gck);
  if (rc != WS_OK) return rc;
  const size_t need_s = ws_workspace_size(&P, WS_DATES | (flags & WS_REFINE));
  if (need_s == 0) return WS_ECUDA;
  const size_t need = std::max(need_s, kHeaderBytes + round256(gck));
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  rc = launch_gcv_dates(P, t, x, w, lam_grid, n_grid, lam_best, scores, static_cast<char*>(workspace) + kHeaderBytes,
                        st);
  if (rc != WS_OK) return rc;
  return ws_smooth_dates(&P, t, x, w, lam_best, z, status, flags & WS_REFINE, workspace, ws_bytes, stream);
}

extern "C" int ws_smooth_batch(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                               void* factor_out, uint8_t* status, uint32_t flags, void* workspace,
                               size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~WS_REFINE) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (P.T == 0) {
    if (status != nullptr && cudaMemsetAsync(status, 0, (size_t)P.n_series, st) != cudaSuccess)
      return set_error(WS_ECUDA, "status memset failed");
    return WS_OK;
  }
  if (!x || !w || !lam || !z) return set_error(WS_EINVAL, "x, w, lam and z must be non-NULL");
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * elem_size(P);
  if (overlaps(x, nx, z, nx)) return set_error(WS_EINVAL, "z must not overlap x");
  const bool refine = (flags & WS_REFINE) != 0;
  size_t ck_bytes = 0;
  rc = check_workspace(P, workspace, ws_bytes, refine ? resid_bytes(P) : 0, ck_bytes);
  if (rc != WS_OK) return rc;
  rc = run_tile(P, MODE_SMOOTH, x, w, lam, nullptr, nullptr, z, nullptr, factor_out, status, 0, 0, workspace, st);
  if (rc != WS_OK || !refine) return rc;
  void* r = static_cast<char*>(workspace) + kHeaderBytes + ck_bytes;
  rc = launch_residual(P, x, w, lam, z, r, 0, static_cast<unsigned*>(workspace), st);
  if (rc != WS_OK) return rc;
  return run_tile(P, MODE_RAW, r, w, lam, /*zin*/ nullptr, /*g0*/ nullptr, /*out*/ z, /*out2*/ nullptr,
                  /*factor*/ nullptr, /*status*/ nullptr, /*accum*/ 1, /*loglam*/ 0, workspace, st);
}

extern "C" int ws_refine(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                         void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0 || P.T == 0) return WS_OK;
  if (!x || !w || !lam || !z) return set_error(WS_EINVAL, "x, w, lam and z must be non-NULL");
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * elem_size(P);
  if (overlaps(x, nx, z, nx)) return set_error(WS_EINVAL, "z must not overlap x");
  size_t ck_bytes = 0;
  rc = check_workspace(P, workspace, ws_bytes, resid_bytes(P), ck_bytes);
  if (rc != WS_OK) return rc;
  void* r = static_cast<char*>(workspace) + kHeaderBytes + ck_bytes;
  rc = launch_residual(P, x, w, lam, z, r, 0, static_cast<unsigned*>(workspace), st);
  if (rc != WS_OK) return rc;
  return run_tile(P, MODE_RAW, r, w, lam, /*zin*/ nullptr, /*g0*/ nullptr, /*out*/ z, /*out2*/ nullptr,
                  /*factor*/ nullptr, /*status*/ nullptr, /*accum*/ 1, /*loglam*/ 0, workspace, st);
}

extern "C" int ws_factor(const ws_problem* pb, const void* w, const void* lam, void* factor, uint8_t* status,
                         void* workspace, size_t ws_bytes, void* stream) {
  (void)workspace, (void)ws_bytes;
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (pb->n_series == 0 || pb->T == 0) return WS_OK;
  if (!w || !lam || !factor) return set_error(WS_EINVAL, "w, lam and factor must be non-NULL");
  return launch_factored(0, *pb, nullptr, factor, w, lam, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                         status, 0, 0, static_cast<cudaStream_t>(stream));
}

extern "C" int ws_solve(const ws_problem* pb, const void* factor, const void* w, const void* x, void* z,
                        uint32_t flags, void* workspace, size_t ws_bytes, void* stream) {
  (void)workspace, (void)ws_bytes;
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags != 0) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  if (pb->n_series == 0 || pb->T == 0) return WS_OK;
  if (!factor || !w || !x || !z) return set_error(WS_EINVAL, "factor, w, x and z must be non-NULL");
  const size_t nx = (size_t)pb->T * pb->n_bands * pb->n_series * elem_size(*pb);
  if (overlaps(x, nx, z, nx)) return set_error(WS_EINVAL, "z must not overlap x");
  return launch_factored(1, *pb, factor, nullptr, w, nullptr, x, z, nullptr, nullptr, nullptr, nullptr, nullptr, 1,
                         0, static_cast<cudaStream_t>(stream));
}

extern "C" int ws_solve_adjoint(const ws_problem* pb, const void* factor_or_null, const void* w, const void* lam,
                                const void* z, const void* gz, void* gx, void* glam, uint32_t flags,
                                uint8_t* status, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~(WS_GRAD_LOGLAM | WS_REFINE_ADJOINT | WS_ADJ_RAW_G))
    return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (P.T == 0) {
    if (status != nullptr && cudaMemsetAsync(status, 0, (size_t)P.n_series, st) != cudaSuccess)
      return set_error(WS_ECUDA, "status memset failed");
    if (glam != nullptr && P.lam_mode == WS_LAM_SCALAR &&
        cudaMemsetAsync(glam, 0, (size_t)P.n_series * elem_size(P), st) != cudaSuccess)
      return set_error(WS_ECUDA, "glam memset failed");
    return WS_OK;
  }
  if (!w || !lam || !z || !gz) return set_error(WS_EINVAL, "w, lam, z and gz must be non-NULL");
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * elem_size(P);
  if (gx != nullptr && (overlaps(gx, nx, gz, nx) || overlaps(gx, nx, z, nx)))
    return set_error(WS_EINVAL, "gx must not overlap gz or z");
  if (factor_or_null != nullptr) return ws_adjoint_factored(pb, factor_or_null, w, lam, z, gz, gx, glam, flags,
                                                            status, workspace, ws_bytes, stream);
  const bool refine = (flags & WS_REFINE_ADJOINT) != 0;
  const int loglam = ((flags & WS_GRAD_LOGLAM) ? 1 : 0) | ((flags & WS_ADJ_RAW_G) ? 2 : 0);
  size_t ck_bytes = 0;
  const size_t df_bytes = refine ? adj_df_bytes(P) : 0;
  rc = check_workspace(P, workspace, ws_bytes, refine ? 2 * resid_bytes(P) + df_bytes : 0, ck_bytes);
  if (rc != WS_OK) return rc;
  if (!refine)
    return run_tile(P, MODE_ADJ, gz, w, lam, z, nullptr, gx, glam, nullptr, status, 0, loglam, workspace, st);
  // g0 = Omega^{-1} gz, r = gz - Omega g0 (double-word), then the adjoint pass solves
  // Omega d = r and applies the epilogue to g = g0 + d. FP32: that pass lists the series
  // whose step did not settle, and those are solved again in double-float.
  char* base = static_cast<char*>(workspace) + kHeaderBytes + ck_bytes;
  void* g0 = base;
  void* r = base + resid_bytes(P);
  void* df = df_bytes > 0 ? base + 2 * resid_bytes(P) : nullptr;
  if (df != nullptr) {  // marks and the list count start at zero
    unsigned *mark = nullptr, *count = nullptr;
    int* list = nullptr;
    char* slots = nullptr;
    adj_df_layout(P, df, &mark, &count, &list, &slots);
    if (cudaMemsetAsync(df, 0, reinterpret_cast<char*>(count) + sizeof(unsigned) - static_cast<char*>(df), st) !=
        cudaSuccess)
      return set_error(WS_ECUDA, "clearing the re-solve list failed");
  }
  rc = run_tile(P, MODE_RAW, gz, w, lam, nullptr, nullptr, g0, nullptr, nullptr, nullptr, 0, 0, workspace, st);
  if (rc != WS_OK) return rc;
  rc = launch_residual(P, gz, w, lam, g0, r, 1, static_cast<unsigned*>(workspace), st);
  if (rc != WS_OK) return rc;
  rc = run_tile(P, MODE_ADJ, r, w, lam, z, g0, gx, glam, nullptr, status, 1, loglam, workspace, st, df);
  if (rc != WS_OK || df == nullptr || (gx == nullptr && glam == nullptr)) return rc;
  return launch_adj_df(P, gz, w, lam, z, gx, glam, loglam, df, st);
}

extern "C" int ws_solve_adjoint_mse(const ws_problem* pb, const void* w, const void* lam, const void* z,
                                    const void* target, const void* mask, double scale, void* gx, void* glam,
                                    void* loss, uint32_t flags, uint8_t* status, void* workspace, size_t ws_bytes,
                                    void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  if (flags & ~(WS_GRAD_LOGLAM | WS_ADJ_RAW_G)) return set_error(WS_EINVAL, "unknown flags 0x%x", flags);
  if (!std::isfinite(scale)) return set_error(WS_EINVAL, "scale must be finite");
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  const int es = elem_size(P);
  const size_t np = (size_t)P.n_series;
  if (P.T == 0) {
    if ((status != nullptr && cudaMemsetAsync(status, 0, np, st) != cudaSuccess) ||
        (loss != nullptr && cudaMemsetAsync(loss, 0, np * es, st) != cudaSuccess) ||
        (glam != nullptr && P.lam_mode == WS_LAM_SCALAR && cudaMemsetAsync(glam, 0, np * es, st) != cudaSuccess))
      return set_error(WS_ECUDA, "memset failed");
    return WS_OK;
  }
  if (!w || !lam || !z || !target) return set_error(WS_EINVAL, "w, lam, z and target must be non-NULL");
  const size_t nx = (size_t)P.T * P.n_bands * np * es, nd = (size_t)P.T * np * es;
  const size_t nl = P.lam_mode == WS_LAM_SCALAR ? np * es : nd;
  const void* ins[5] = {w, lam, z, target, mask};
  const size_t nin[5] = {nd, nl, nx, nx, nd};
  for (int i = 0; i < 5; ++i) {
    if (ins[i] == nullptr) continue;
    if ((gx != nullptr && overlaps(gx, nx, ins[i], nin[i])) || (glam != nullptr && overlaps(glam, nl, ins[i], nin[i])) ||
        (loss != nullptr && overlaps(loss, np * es, ins[i], nin[i])))
      return set_error(WS_EINVAL, "gx, glam and loss must not overlap the inputs");
  }
  if ((gx != nullptr && glam != nullptr && overlaps(gx, nx, glam, nl)) ||
      (loss != nullptr && ((gx != nullptr && overlaps(loss, np * es, gx, nx)) ||
                           (glam != nullptr && overlaps(loss, np * es, glam, nl)))))
    return set_error(WS_EINVAL, "gx, glam and loss must not overlap each other");
  size_t ck_bytes = 0;
  rc = check_workspace(P, workspace, ws_bytes, 0, ck_bytes);
  if (rc != WS_OK) return rc;
  const int adj = ((flags & WS_GRAD_LOGLAM) ? 1 : 0) | ((flags & WS_ADJ_RAW_G) ? 2 : 0);
  const AdjMse m{mask, scale, loss};
  return run_tile(P, MODE_ADJ, target, w, lam, z, nullptr, gx, glam, nullptr, status, 0, adj, workspace, st, nullptr,
                  &m);
}

extern "C" int ws_smooth_partitioned(const ws_problem* pb, const void* x, const void* w, const void* lam, void* z,
                                     uint8_t* status, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int rc = validate_problem(pb);
  if (rc != WS_OK) return rc;
  const ws_problem& P = *pb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P.n_series == 0) return WS_OK;
  if (P.T == 0) {
    if (status != nullptr && cudaMemsetAsync(status, 0, (size_t)P.n_series, st) != cudaSuccess)
      return set_error(WS_ECUDA, "status memset failed");
    return WS_OK;
  }
  if (!x || !w || !lam || !z) return set_error(WS_EINVAL, "x, w, lam and z must be non-NULL");
  const int es = elem_size(P);
  const size_t nx = (size_t)P.T * P.n_bands * P.n_series * es, nd = (size_t)P.T * P.n_series * es;
  const size_t nl = P.lam_mode == WS_LAM_SCALAR ? (size_t)P.n_series * es : nd;
  if (overlaps(z, nx, x, nx) || overlaps(z, nx, w, nd) || overlaps(z, nx, lam, nl))
    return set_error(WS_EINVAL, "z must not overlap the inputs");
  const size_t need = kHeaderBytes + part_workspace_bytes(P);
  if (workspace == nullptr || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) return set_error(WS_ENOMEM_WS, "workspace too small: %zu < %zu", ws_bytes, need);
  return launch_partitioned(P, x, w, lam, z, status, static_cast<char*>(workspace) + kHeaderBytes, st);
}

extern "C" int ws_tune_pixels_per_cta(int32_t pixels) {
  clear_error();
  if (pixels != 0 && pixels != 64 && pixels != 128) return set_error(WS_EINVAL, "pixels per CTA must be 0, 64 or 128");
  g_tune_np = pixels;
  return WS_OK;
}

extern "C" int ws_tune_checkpoint_group(int32_t chunks) {
  clear_error();
  if (chunks < 0 || chunks > 2) return set_error(WS_EINVAL, "chunks per checkpoint must be 0, 1 or 2");
  g_tune_ckgroup = chunks;
  return WS_OK;
}

extern "C" int ws_tune_set(int32_t ctas_per_sm, int32_t chunk_days) {
  clear_error();
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return set_error(WS_EINVAL, "ctas_per_sm must be 0..32");
  if (chunk_days < 0 || chunk_days > 255) return set_error(WS_EINVAL, "chunk_days must be 0..255");
  g_tune_ctas = ctas_per_sm;
  g_tune_chunk = chunk_days;
  return WS_OK;
}

extern "C" int ws_sync_status(void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  if (workspace == nullptr || ws_bytes < kHeaderBytes) return set_error(WS_EINVAL, "workspace too small or NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  unsigned word = 0;
  e = cudaMemcpy(&word, workspace, sizeof(word), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(WS_ECUDA, "reading the device error word: %s", cudaGetErrorString(e));
  if (word != 0) {
    cudaMemset(workspace, 0, sizeof(word));
    return set_error(WS_ETIMEOUT, "a device-side wait gave up (error word 0x%x)", word);
  }
  return WS_OK;
}

extern "C" int ws_last_error(char* buf, size_t n) {
  if (buf != nullptr && n > 0) {
    strncpy(buf, g_err_msg, n - 1);
    buf[n - 1] = '\0';
  }
  return g_err_code;
}

extern "C" const char* ws_version(void) { return "ws_b300 0.1 sm_103a"; }
