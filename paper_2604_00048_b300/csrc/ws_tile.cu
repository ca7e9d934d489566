// Host-side planning of the tile kernels (ws_tile_impl.cuh) and dispatch by order d.
// The kernel: z = (W + D^T Lambda D)^{-1} W x (Eq. 3) for NP pixel
// series per CTA, one series per thread, B bands as right-hand sides.
//
// Data flow per tile of NP pixels (persistent CTAs loop over tiles):
//   pass 1 (forward in time): chunks of C days of x (NB bands), w (C+d days, the
//     rotation of day i needs w_{i+d}) and lambda are staged in shared memory by TMA
//     (cp.async.bulk.tensor, two stages, mbarrier completion). Each thread runs the
//     rotation factor + forward substitution (ws_sweep.cuh) and stores its state at
//     every chunk boundary to a checkpoint area in global memory.
//   pass 2 (backward in time): for each chunk, last to first, the state is reloaded
//     from its checkpoint and the chunk is recomputed from the staged inputs,
//     writing yhat and rho in place over x, w and lambda; back substitution then
//     runs over the chunk in reverse, writing z in place over yhat, and TMA stores
//     the z box. The last two chunks of pass 1 are still resident and are reused.
// Inputs are read twice and z written once (plus d(d+1)+B*d checkpoint words per
// pixel per chunk), instead of spilling the factor and y for every day.
//
// Shared-memory stage (rows of NP elements):
//   X [C*NB rows]  x[t][b] (pass 2: yhat, then z)
//   W [C+d rows]   w       (pass 2: rho_2 over the first C rows)
//   L [C rows]     lambda  (pass 2: rho_1)
//   E [(d-2)*C]    pass 2: rho_3..rho_d (d > 2)
// When TMA cannot describe the arrays (row pitch not a multiple of 16 bytes, base
// not 16-byte aligned) every thread copies its own column with LDGSTS instead and
// stores z directly; the arithmetic is the same.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"

namespace ws {

// ----------------------------------------------------------------------------------
// host side

int g_tune_np = 0, g_tune_chunk = 0;

int plan_tile(const ws_problem& pb, int nb, int D, int extra_planes, TileCfg& cfg) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  const int es = pb.dtype == WS_F64 ? 8 : 4;
  cfg.NP = g_tune_np > 0 ? g_tune_np : 128;
  cfg.stages = 2;
  const int T = pb.T;
  // rows per stage = C * (nb + 2 + extra_planes) + D; two stages in the opt-in shared memory
  const long budget = (long)di.smem_optin - 1024;
  const long rows_max = budget / (2L * cfg.NP * es);
  long C = (rows_max - D) / (nb + 2 + extra_planes);
  if (C > 256 - D) C = 256 - D;
  if (g_tune_chunk > 0 && g_tune_chunk < C) C = g_tune_chunk;
  if (C > T) C = T > 0 ? T : 1;
  if (C < 1) C = 1;
  cfg.C = (int)C;
  cfg.nch = T > 0 ? (T + cfg.C - 1) / cfg.C : 0;
  cfg.n_tiles = (int)((pb.n_series + cfg.NP - 1) / cfg.NP);
  const size_t rows = (size_t)cfg.C * (nb + 2 + extra_planes) + D;
  cfg.stage_elems = rows * cfg.NP;
  cfg.smem_bytes = 2 * cfg.stage_elems * es + 64;
  int per_sm = (int)((long)(di.smem_optin + 1024) / (long)(cfg.smem_bytes + 1024));
  if (per_sm < 1) per_sm = 1;
  const long cap = (long)di.sm_count * per_sm;
  cfg.grid = (int)(cfg.n_tiles < cap ? cfg.n_tiles : cap);
  cfg.fields = D * (D + 1) + nb * D;
  return WS_OK;
}

int launch_tile(const ws_problem& pb, int mode, int nb, const TileCfg& cfg, const TileArgs& a,
                const CUtensorMap* maps, cudaStream_t st) {
  switch (pb.d) {
    case 1: return launch_tile_d1(pb, mode, nb, cfg, a, maps, st);
    case 2: return launch_tile_d2(pb, mode, nb, cfg, a, maps, st);
    case 3: return launch_tile_d3(pb, mode, nb, cfg, a, maps, st);
    case 4: return launch_tile_d4(pb, mode, nb, cfg, a, maps, st);
  }
  return set_error(WS_EINVAL, "unsupported order d=%d", pb.d);
}

}  // namespace ws
