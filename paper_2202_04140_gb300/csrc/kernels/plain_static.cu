// Fixed device scratch for the allocation-free variant of the plain FP64 graph
// walk (ace_eval_plain_f64_static).
//
// The array below is part of the library image: every GPU that loads libace
// holds these bytes until the process exits.  In host code the array's name
// only denotes a host-side stand-in, never a device address, so the device
// address is looked up with cudaGetSymbolAddress once per device (with that
// device current) and cached for the life of the process; kernels receive that
// address as an argument.  The cache assumes the device's primary context is
// never torn down (cudaDeviceReset would leave a stale address), which the
// entry point's documentation states.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "launch.hpp"

namespace ace {

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }

// Device address of the scratch array on the current device; the first call on
// a device performs the lookup.
cudaError_t static_scratch_ptr(void** out) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace ace
