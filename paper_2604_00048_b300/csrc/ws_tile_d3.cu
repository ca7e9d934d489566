// Instantiations of the tile kernels for difference order d = 3 (one translation unit
// per order so that nvcc compiles them in parallel).
#include "ws_tile_impl.cuh"

namespace ws {
int launch_tile_d3(const ws_problem& pb, int mode, int nb, const TileCfg& cfg, const TileArgs& a,
                    const CUtensorMap* maps, cudaStream_t st) {
  return dispatch_tile_d<3>(pb, mode, nb, cfg, a, maps, st);
}
const void* tile_kernel_ptr_d3(const ws_problem& pb, int mode, int nb, int np) {
  return tile_kernel_ptr_t<3>(pb, mode, nb, np);
}
}  // namespace ws
