// vc_decode_bricks_noalloc: the grid / batched decode with its scratch memory (the rANS symbol
// workspace, the size-aware order of large requests, the 64^3 decoder's scratch slices) in a
// fixed, statically reserved device array instead of stream-ordered allocations. It is meant for
// callers that must not allocate device memory while decoding: real-time loops that cannot
// afford the allocator's latency or its synchronisation, and processes whose device memory is
// reserved up front by another allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "vc_internal.h"

namespace {

constexpr size_t kNoAllocWsBytes = VC_NOALLOC_WS_BYTES;
// The early size check below compares n * ws_stride with the array size, while the launch rounds
// the symbol bytes up to 256; the two agree because the size is a multiple of 256.
static_assert(kNoAllocWsBytes % 256 == 0, "the no-alloc workspace size must be a multiple of 256 bytes");
constexpr int kMaxDevices = 64;

// Scratch of the rANS symbol kernel for every call of this entry point on a device. Nothing in it
// needs to start at zero: each item's symbols are written before they are read within one call.
__device__ __align__(256) uint8_t g_noalloc_ws[kNoAllocWsBytes];

std::mutex g_setup_mu;
uint8_t* g_ws_ptr[kMaxDevices] = {};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Once per device, with that device current: the device address of the static workspace.
vc_status workspace_for(int device, uint8_t** out) {
  if (device < 0 || device >= kMaxDevices) return VC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_ws_ptr[device]) {
    void* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (rc != cudaSuccess || !p) {
      cudaGetLastError();
      return VC_ERR_CUDA;
    }
    g_ws_ptr[device] = static_cast<uint8_t*>(p);
  }
  *out = g_ws_ptr[device];
  return VC_OK;
}

}  // namespace

extern "C" vc_status vc_decode_bricks_noalloc(vc_volume* vol, const uint32_t* brick_ids, uint32_t n,
                                             const uint32_t* cache_slots, uint32_t* cache, uint32_t lod,
                                             uint32_t mode, int32_t* status_dev, void* cuda_stream) {
  vc::Volume* v = reinterpret_cast<vc::Volume*>(vol);
  if (!v || v->kind != vc::kHandleVolume) return VC_ERR_ARG;
  if (n == 0) return VC_OK;
  if (!brick_ids || !cache_slots || !cache || !status_dev) return VC_ERR_ARG;
  const uint32_t base_mode = mode & ~VC_MODE_PALETTED;
  if (lod > v->L || (base_mode != VC_MODE_GRID && base_mode != VC_MODE_BATCHED)) return VC_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(cache) & 15u) return VC_ERR_ARG;
  if (v->coder == 1 && (size_t)n * v->dv.sm.ws_stride > kNoAllocWsBytes) return VC_ERR_ARG;  // more checks in the launch
  DeviceGuard g(v->device);
  uint8_t* ws = nullptr;
  const vc_status rc = workspace_for(v->device, &ws);
  if (rc != VC_OK) return rc;
  return vc::launch_decode_ws(*v, brick_ids, n, cache_slots, cache, lod, mode, status_dev,
                              static_cast<cudaStream_t>(cuda_stream), ws, kNoAllocWsBytes);
}
