// Internal declarations shared by the C-ABI layer and the kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ws.h"

namespace ws {

constexpr int kNbMax = 10;
enum { MODE_SMOOTH = 0, MODE_RAW = 1, MODE_ADJ = 2 };         // bands per launch; more bands run as band groups
constexpr size_t kHeaderBytes = 256;  // device error word + reserved

// Staging / launch configuration of one tile launch.
struct TileCfg {
  int NP = 128;        // pixels (threads) per CTA
  int C = 16;          // days per chunk
  int nch = 0;         // chunks per series
  int n_tiles = 0;     // ceil(P / NP)
  int grid = 0;        // CTAs (persistent over tiles)
  int stages = 2;
  size_t stage_elems = 0;
  size_t smem_bytes = 0;
  bool tma = false;
  int fields = 0;      // checkpoint words per pixel per chunk
};

// Arguments of the tile kernels (plain pointers + sizes).
struct TileArgs {
  int T, P, B, b0;
  int C, NP, nch, n_tiles;
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
  int accum;              // RAW: out += solution (refinement correction)
};

struct DeviceInfo {
  int sm_count = 0;
  int smem_optin = 0;
};
int device_info(DeviceInfo& info);

int set_error(int code, const char* fmt, ...);

// Tensor-map helper: rank-2/3 tile map over a dense row-major array (fastest dim first).
int make_tmap(CUtensorMap* map, int dtype, int rank, const void* base, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box);

// Launchers (return WS_OK or an error code, errors recorded via set_error).
extern int g_tune_np, g_tune_chunk;  // ws_tune_set() overrides (0 = automatic)
int plan_tile(const ws_problem& pb, int nb, int D, int extra_planes, TileCfg& cfg);
int launch_tile(const ws_problem& pb, int mode, int nb, const TileCfg& cfg, const TileArgs& a,
                const CUtensorMap* maps, cudaStream_t st);
int launch_tile_d1(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d2(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d3(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
int launch_tile_d4(const ws_problem&, int, int, const TileCfg&, const TileArgs&, const CUtensorMap*, cudaStream_t);
// r = W x - Omega z0 with double-word accumulation (refinement residual).
// raw = 0: r = W x - Omega z0; raw = 1: r = x - Omega z0.
int launch_residual(const ws_problem& pb, const void* x, const void* w, const void* lam, const void* z0,
                    void* r, int raw, cudaStream_t st);

}  // namespace ws
