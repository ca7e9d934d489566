// Diagnostic of the bounded device-side waits: one CTA waits on an mbarrier that no thread
// ever arrives at, with the same bounded wait the staging pipelines use. After the wait limit
// (about a second of SM cycles) it gives up, records the timeout in the workspace's error
// word and returns, leaving the context usable; ws_sync_status then reports WS_ETIMEOUT.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ws_internal.h"
#include "ws_ptx.cuh"

namespace ws {

__global__ void k_selftest_wait(unsigned* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u)) atomicOr(err, kDevErrTimeout);
}

}  // namespace ws

extern "C" int ws_selftest_wait(void* workspace, size_t ws_bytes, void* stream) {
  using namespace ws;
  if (workspace == nullptr || ws_bytes < kHeaderBytes || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return set_error(WS_EINVAL, "workspace must be non-NULL, 256-byte aligned and at least the header");
  k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<unsigned*>(workspace));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WS_ECUDA, "self-test launch: %s", cudaGetErrorString(e));
  return WS_OK;
}
