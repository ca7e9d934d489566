// Host-side planning of the tile kernels (ws_tile_impl.cuh) and dispatch by order d.
// The kernel: z = (W + D^T Lambda D)^{-1} W x (Eq. 3) for NP pixel
// series per CTA, one series per thread, B bands as right-hand sides.
//
// Data flow per tile of NP pixels (persistent CTAs loop over tiles):
//   pass 1 (forward in time): chunks of C days of x (NB bands), w (C+d days, the
//     rotation of day i needs w_{i+d}) and lambda are staged in shared memory by TMA
//     (cp.async.bulk.tensor, two stages, mbarrier completion). Each thread runs the
//     rotation factor + forward substitution (ws_sweep.cuh) and stores its state at
//     the start of every group of chunks (two by default) to a checkpoint area in global
//     memory.
//   pass 2 (backward in time): group by group, last to first, the state is reloaded
//     from its checkpoint and the group's chunks (both resident) are recomputed from the
//     staged inputs, writing yhat and rho in place; back substitution then runs over
//     each chunk in reverse, writing z in place over yhat, and TMA stores the z box. The
//     last two chunks of pass 1 are still resident and are reused.
// Inputs are read twice and z written once (plus d(d+1)+B*d checkpoint words per
// pixel per group of chunks), instead of spilling the factor and y for every day.
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

int g_tune_ctas = 0, g_tune_chunk = 0, g_tune_np = 0, g_tune_ckgroup = 0;

// Largest chunk (days) whose shared memory fits `ctas` CTAs of `np` pixels on one SM.
static long chunk_for(const ws_problem& pb, int mode, int nb, int S, int ctas, int np, const DeviceInfo& di,
                      int mse) {
  const int es = pb.dtype == WS_F64 ? 8 : 4;
  const int D = pb.d;
  long per_cta = (long)di.smem_per_sm / ctas - 1024;
  if (per_cta > di.smem_optin) per_cta = di.smem_optin;
  const long rows = (per_cta - 64 - np * 4) / ((long)np * es);
  const long fixed = (long)tile_smem_rows(mode, 0, nb, D, S, mse);         // rows independent of C
  const long coef = (long)tile_smem_rows(mode, 1, nb, D, S, mse) - fixed;  // rows per day of chunk
  return (rows - fixed) / coef;
}

int plan_tile(const ws_problem& pb, int mode, int nb, TileCfg& cfg, int mse) {
  DeviceInfo di;
  int rc = device_info(di);
  if (rc != WS_OK) return rc;
  const int es = pb.dtype == WS_F64 ? 8 : 4;
  const int D = pb.d, T = pb.T;
  const int S = band_split(nb, pb.dtype == WS_F64);
  // pixels per CTA: 128, or 64 (FP32) for deeper chunks at the same CTAs per SM. FP32 band
  // groups of two or more bands default to 64: on the 10-band tile (d = 2, 3288 days) four
  // 64-pixel CTAs per SM took 31.1 / 20.6 / 44.7 ms (adjoint / smooth / smooth's refinement
  // step) against 31.6 / 21.2 / 45.2 ms for two 128-pixel ones (one CTA's barrier waits then
  // idle fewer warps); the 4-band layer workload (smooth + fused-loss adjoint) 4.1 against
  // 4.8 ms. One band keeps 128: the ragged plan's one-band length classes, 28.2 against
  // 29.2 ms (refined execute 169.5 against 173.6 ms).
  const bool np64 = g_tune_np == 64 || (g_tune_np == 0 && nb > 1);
  const int np = (pb.dtype == WS_F32 && np64) ? 64 : 128;
  cfg.NP = np;
  cfg.S = S;
  cfg.stages = 2;
  // Aim at 16 resident warps per SM (latency of the sequential recurrence), but keep
  // chunks of at least 5 days (checkpoint traffic grows as 1/C); 4 for the correction and
  // adjoint modes, whose per-day work is larger.
  int ctas = g_tune_ctas > 0 ? g_tune_ctas : (S > 1 ? 2 : 4) * (128 / np);
  const long min_chunk = (mode == MODE_RAW || mode == MODE_ADJ) ? 4 : 5;
  long C = 0;
  for (; ctas >= 1; --ctas) {
    C = chunk_for(pb, mode, nb, S, ctas, np, di, mse);
    if (C >= min_chunk || ctas == 1 || g_tune_ctas > 0) break;
  }
  // registers may allow fewer CTAs than shared memory: then give the chunk the room
  const void* kern = tile_kernel_ptr(pb, mode, nb, np);
  if (kern == nullptr) return set_error(WS_EUNSUPPORTED, "no tile kernel for %d bands", nb);
  auto fit = [&](long Cc, int* occ) -> int {
    const size_t smem = tile_smem_bytes(mode, (int)Cc, nb, D, S, es, np, mse);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(WS_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, np * S, smem);
    if (e != cudaSuccess) return set_error(WS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    return WS_OK;
  };
  auto clampC = [&](long Cc) {
    if (Cc > 256 - D) Cc = 256 - D;
    if (g_tune_chunk > 0 && g_tune_chunk < Cc) Cc = g_tune_chunk;
    if (Cc > T) Cc = T > 0 ? T : 1;
    if (Cc < 1) Cc = 1;
    return Cc;
  };
  C = clampC(C);
  int occ = 0;
  if ((rc = fit(C, &occ)) != WS_OK) return rc;
  if (occ >= 1 && occ < ctas && g_tune_chunk == 0) {
    C = clampC(chunk_for(pb, mode, nb, S, occ, np, di, mse));
    if ((rc = fit(C, &occ)) != WS_OK) return rc;
  }
  if (occ < 1) return set_error(WS_EUNSUPPORTED, "tile kernel does not fit on an SM (chunk %ld)", C);
  cfg.C = (int)C;
  cfg.nch = T > 0 ? (T + cfg.C - 1) / cfg.C : 0;
  cfg.n_tiles = (int)((pb.n_series + np - 1) / np);
  cfg.stage_elems = tile_stage_rows(mode, cfg.C, nb, D, S, mse) * np;
  cfg.smem_bytes = tile_smem_bytes(mode, cfg.C, nb, D, S, es, np, mse);
  const long cap = (long)di.sm_count * occ;
  cfg.grid = (int)(cfg.n_tiles < cap ? cfg.n_tiles : cap);
  cfg.fields = D * (D + 1) + nb * D;
  // Checkpoints every second chunk: pass 2 recomputes both resident chunks of the ring from
  // one checkpoint, halving the checkpoint words written and read.
  cfg.ck_group = g_tune_ckgroup > 0 ? g_tune_ckgroup : 2;
  return WS_OK;
}

const void* tile_kernel_ptr(const ws_problem& pb, int mode, int nb, int np) {
  switch (pb.d) {
    case 1: return tile_kernel_ptr_d1(pb, mode, nb, np);
    case 2: return tile_kernel_ptr_d2(pb, mode, nb, np);
    case 3: return tile_kernel_ptr_d3(pb, mode, nb, np);
    case 4: return tile_kernel_ptr_d4(pb, mode, nb, np);
  }
  return nullptr;
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
