// Fixed scratch for gp_apply_noalloc: the face outputs of one apply, held in a
// file-scope device array instead of memory the context allocates.
//
// The array is part of this library's device image: every GPU on which the
// library's code is loaded holds its GP_NOALLOC_SCRATCH_BYTES until the process
// exits.  All calls share it and it keeps the previous call's contents; the face
// kernel overwrites every entry the lift kernel reads, so nothing needs clearing.
// Calls whose kernels overlap on the GPU (different streams, or several host
// threads) race on it.
#include <mutex>

#include "gp.h"
#include "gp_launch.h"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;
static_assert(kScratchBytes == GP_NOALLOC_SCRATCH_BYTES, "the scratch size must match the documented limit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

}  // namespace

namespace gp {

size_t noalloc_scratch_bytes() { return kScratchBytes; }

// Device address of the scratch array on `device`, which must be the current
// device.  The host-side symbol is only a stand-in, so the address is looked up
// once per device with cudaGetSymbolAddress and cached.  A device reset
// (cudaDeviceReset, or a reset of the primary context) unloads the library's
// device image and invalidates the cached address: the cache is not refreshed,
// so gp_apply_noalloc must not be called after such a reset.
cudaError_t noalloc_scratch(int device, void** out) {
  *out = nullptr;
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[device] = p;
  }
  *out = g_ptr[device];
  return cudaSuccess;
}

}  // namespace gp
