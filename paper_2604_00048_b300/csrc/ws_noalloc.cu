// ws_smooth_batch_noalloc: the smoothing entry point with its scratch in a fixed,
// file-scope device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they smooth: a host
// framework whose caching allocator already holds the device memory (a separate
// cudaMalloc would fail or fragment it), code that must not stall other streams on the
// device-wide synchronisation cudaFree implies, or a plain C caller with no device
// allocator of its own. This entry point serves them for problems whose workspace fits
// kNoallocBytes; it calls no cudaMalloc, cudaFree or allocating library routine and
// hands the static array to ws_smooth_batch, whose kernels and results it shares.
//
// Calls on the same device share the one array: calls that overlap in time (several host
// threads, or several streams without ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "ws_internal.h"

namespace {

constexpr size_t kNoallocBytes = WS_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_ws[kNoallocBytes];

std::mutex g_setup_mu;
void* g_addr[kMaxDevices] = {};

// Once per device, with that device current: the array's address, and its header (the
// device error word the kernels set when a bounded wait gives up) cleared to zero.
int noalloc_setup(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ws::set_error(WS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ws::set_error(WS_EUNSUPPORTED, "device ordinal %d", dev);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e != cudaSuccess || p == nullptr)
      return ws::set_error(WS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    e = cudaMemset(p, 0, ws::kHeaderBytes);
    if (e != cudaSuccess) return ws::set_error(WS_ECUDA, "clearing the static header: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return WS_OK;
}

}  // namespace

extern "C" int ws_smooth_batch_noalloc(const ws_problem* pb, const void* x, const void* w, const void* lam,
                                       void* z, void* factor_out, uint8_t* status, uint32_t flags,
                                       void* stream) {
  if (pb == nullptr) return ws::set_error(WS_EINVAL, "problem is NULL");
  const size_t need = ws_workspace_size(pb, flags & WS_REFINE);
  if (need == 0) return ws::set_error(WS_EINVAL, "invalid problem");
  if (need > kNoallocBytes)
    return ws::set_error(WS_ENOMEM_WS, "workspace of %zu bytes exceeds the static %zu bytes", need, kNoallocBytes);
  void* ws = nullptr;
  int rc = noalloc_setup(&ws);
  if (rc != WS_OK) return rc;
  return ws_smooth_batch(pb, x, w, lam, z, factor_out, status, flags, ws, kNoallocBytes, stream);
}
