// Internal declarations shared by the C-ABI layer and the kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ws.h"

namespace ws {

constexpr int kNbMax = 10;
enum { MODE_SMOOTH = 0, MODE_RAW = 1, MODE_ADJ = 2 };
constexpr int kNP = 128;  // pixels per CTA of the tile kernels (64 is the other instantiation, FP32)

// Threads per pixel of a band group: two (each owning half the bands) for 6, 8, 10 bands.
__host__ __device__ inline int band_split(int nb, bool fp64) { return (!fp64 && nb >= 6 && nb % 2 == 0) ? 2 : 1; }

// Shared-memory layout of the tile kernels, in rows of kNP elements (ws_tile_impl.cuh).
__host__ __device__ inline int tile_extra_planes(int mode, int D, int S) {
  return (mode == MODE_ADJ || S > 1) ? D : (D > 2 ? D - 2 : 0);
}
// checkpoint words per pixel per chunk: factor state + forward-substitution state
__host__ __device__ inline int tile_ckpt_fields(int NB, int D) { return D * (D + 1) + NB * D; }
// stage: X (C*NB), Z (C*NB, RAW/ADJ), W (C+d), L (C), E (extra planes * C), M (C, ADJ with
// the fused MSE loss: the day weights)
__host__ __device__ inline size_t tile_stage_rows(int mode, int C, int NB, int D, int S, int mse = 0) {
  const size_t xz = (size_t)C * NB * ((mode == MODE_RAW || mode == MODE_ADJ) ? 2 : 1);
  return xz + C + D + C + (size_t)tile_extra_planes(mode, D, S) * C + (mse ? (size_t)C : 0);
}
__host__ __device__ inline size_t tile_smem_rows(int mode, int C, int NB, int D, int S, int mse = 0) {
  size_t rows = 2 * tile_stage_rows(mode, C, NB, D, S, mse);
  if (mode == MODE_ADJ) rows += (size_t)S * C;
  return rows;
}
// rows of NP elements + 3 mbarriers (64 bytes reserved) + NP status words
__host__ __device__ inline size_t tile_smem_bytes(int mode, int C, int NB, int D, int S, int es, int NP, int mse = 0) {
  return tile_smem_rows(mode, C, NB, D, S, mse) * NP * es + 64 + NP * 4;
}         // bands per launch; more bands run as band groups
constexpr size_t kHeaderBytes = 256;  // device error word + reserved

// Staging / launch configuration of one tile launch.
struct TileCfg {
  int NP = kNP;        // pixels per CTA
  int S = 1;           // threads per pixel (band split)
  int C = 16;          // days per chunk
  int nch = 0;         // chunks per series
  int n_tiles = 0;     // ceil(P / NP)
  int grid = 0;        // CTAs (persistent over tiles)
  int stages = 2;
  size_t stage_elems = 0;
  size_t smem_bytes = 0;
  bool tma = false;
  int fields = 0;      // checkpoint words per pixel per chunk
  int ck_group = 2;    // chunks per checkpoint (1 or 2)
};

// Arguments of the tile kernels (plain pointers + sizes).
struct TileArgs {
  int T, P, B, b0;
  int C, NP, nch, n_tiles;
  int ck_group;           // chunks per checkpoint: 1, or 2 (both ring stages recomputed together)
  int lam_scalar, tma;
  int write_status;       // this launch owns the status codes (first band group)
  const void* x;          // SMOOTH: x; ADJOINT: gz
  const void* w;
  const void* lam;
  const void* zin;        // ADJOINT: forward output z
  const void* g0;         // ADJOINT with accum: first solution g0 (g = g0 + correction)
  void* out;              // SMOOTH: z; ADJOINT: gx (may be null)
  void* out2;             // ADJOINT: glam (may be null)
  void* factor;           // optional factor output (SMOOTH) / input (SOLVE)
  uint8_t* status;
  void* ckpt;
  unsigned* err;
  size_t stage_elems;
  int grad_loglam;
  int raw_g;              // ADJOINT: out receives g itself instead of W g
  int accum;              // RAW: out += solution (refinement correction)
  // ADJOINT with accum (refined adjoint, FP32): series whose step did not settle are marked
  // once (df_mark) and appended to df_list (df_count) for the double-float re-solve; NULL: off
  unsigned* df_mark;
  int* df_list;
  unsigned* df_count;
  // ADJ with the masked-MSE loss fused in (x is then the target): gz = mse_scale * m * (z - x)
  int mse;
  const void* mask;       // [T][P] day weights m, or NULL (all ones)
  double mse_scale;
  void* loss;             // [P] scale/2 * sum m (z - x)^2 (accumulated over band groups), or NULL
};

struct DeviceInfo {
  int sm_count = 0;
  int smem_optin = 0;   // max dynamic shared memory per block
  int smem_per_sm = 0;  // shared memory per SM
};
int device_info(DeviceInfo& info);

int set_error(int code, const char* fmt, ...);

// Tensor-map helper: rank-2/3 tile map over a dense row-major array (fastest dim first).
int make_tmap(CUtensorMap* map, int dtype, int rank, const void* base, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box);

// One smoothing tile launch sequence (ws_api.cu), used by the ragged plan's length classes.
int tile_smooth(const ws_problem& P, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                void* workspace, cudaStream_t st);
int tile_refine(const ws_problem& P, const void* x, const void* w, const void* lam, void* z, void* r,
                void* workspace, cudaStream_t st);
size_t tile_workspace_bytes(const ws_problem& P);

// GCV grid search (ws_gcv.cu): persistent grid, chunks and checkpoint bytes; launch.
int gcv_plan(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes);
int launch_gcv(const ws_problem& pb, const void* x, const void* w, const float* grid_vals, int n_grid,
               float* lam_best, float* scores, void* ckpt, cudaStream_t st);

// Posterior spread (ws_post.cu): persistent grid, chunks and checkpoint bytes; launch of the
// diagonal kernel and the spread kernel. den: P elements of scratch.
int post_plan(const ws_problem& pb, int& grid, int& nch, size_t& ck_bytes);
int launch_posterior(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z,
                     void* diag, void* sigma2, void* sd, uint8_t* status, void* ckpt, void* den, cudaStream_t st);

// Smoothing on uneven sample times (ws_dates.cu): checkpoint bytes; launch of the band groups.
// adj: the adjoint (x is dL/dz, out receives gx, zin the forward z, glam dL/dlambda).
int dates_plan(const ws_problem& pb, bool adj, size_t& ck_bytes);
int launch_dates(const ws_problem& pb, bool adj, const void* t, const void* x, const void* w, const void* lam,
                 void* out, const void* zin, void* glam, int loglam, uint8_t* status, void* ckpt, cudaStream_t st);

// Launchers (return WS_OK or an error code, errors recorded via set_error).
extern int g_tune_ctas, g_tune_chunk, g_tune_np, g_tune_ckgroup;  // ws_tune_* overrides (0 = automatic)
int plan_tile(const ws_problem& pb, int mode, int nb, TileCfg& cfg, int mse = 0);
int launch_tile(const ws_problem& pb, int mode, int nb, const TileCfg& cfg, const TileArgs& a,
                const CUtensorMap* maps, cudaStream_t st);
const void* tile_kernel_ptr(const ws_problem& pb, int mode, int nb, int np);
const void* tile_kernel_ptr_d1(const ws_problem& pb, int mode, int nb, int np);
const void* tile_kernel_ptr_d2(const ws_problem& pb, int mode, int nb, int np);
const void* tile_kernel_ptr_d3(const ws_problem& pb, int mode, int nb, int np);
const void* tile_kernel_ptr_d4(const ws_problem& pb, int mode, int nb, int np);
int launch_tile_d1(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d2(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d3(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d4(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
// dL/dw_t = sum_b g_tb (x_tb [w_t > 0] - z_tb) and gx = W g (ws_wgrad.cu).
int launch_wgrad(const ws_problem& pb, const void* x, const void* w, const void* z, void* g, void* gx, void* gw,
                 cudaStream_t st);
// r = W x - Omega z0 with double-word accumulation (refinement residual).
// Stored-factor kernels (ws_factored.cu): what = 0 factor, 1 solve, 2 adjoint epilogue.
int launch_factored(int what, const ws_problem& pb, const void* fac_in, void* fac_out, const void* w,
                    const void* lam, const void* x, void* out, const void* z, const void* gs, void* gx, void* glam,
                    uint8_t* status, int weighted, int loglam, cudaStream_t st);
// Double-float re-solve of the adjoint for the series the refined FP32 adjoint listed
// (ws_adjdf.cu): scratch bytes, its layout, and the launch (overwrites gx and glam of the
// listed series). adj_flags as run_tile's.
size_t adj_df_bytes(const ws_problem& pb);
void adj_df_layout(const ws_problem& pb, void* base, unsigned** mark, unsigned** count, int** list, char** slots);
int launch_adj_df(const ws_problem& pb, const void* gz, const void* w, const void* lam, const void* z, void* gx,
                  void* glam, int adj_flags, void* base, cudaStream_t st);
// Partitioned parallel-in-time solve (ws_part.cu): scratch bytes and launch.
size_t part_workspace_bytes(const ws_problem& pb);
int launch_partitioned(const ws_problem& pb, const void* x, const void* w, const void* lam, void* z, uint8_t* status,
                       void* scratch, cudaStream_t st);
// raw = 0: r = W x - Omega z0; raw = 1: r = x - Omega z0. err: the workspace's device
// error word (set when a staging wait gives up).
int launch_residual(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0,
                    void* r, int raw, unsigned* err, cudaStream_t st);

}  // namespace ws
