// Fixed per-pixel scratch for lidar_simulate_noalloc.
//
// lidar_simulate keeps its per-pixel records in device memory it allocates
// (and grows) with cudaMalloc. Some callers cannot allow that: hosts whose
// memory pool reserves the whole GPU up front, and real-time loops that must
// not allocate once running (a cudaMalloc can fail, stall, or synchronise the
// device in the middle of a frame). For them the records live in the
// statically sized array below instead, which the CUDA runtime places in
// device memory when the library is loaded; every GPU that loads the library
// holds it (kNoAllocMaxPixels * 32 bytes = 32 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lidar_internal.h"

namespace gbl {

// 32-byte record per G-buffer pixel, two float4 each.
static __device__ __align__(256) float4 g_noalloc_records[2 * (size_t)kNoAllocMaxPixels];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
float4 *g_addr[kMaxDevices] = {};
}  // namespace

// Device address of the array on the current device. In host code the name
// g_noalloc_records stands for a host-side shadow, not a device address, so it
// must never be passed to a kernel directly: the address is looked up with
// cudaGetSymbolAddress, once per device (with that device current), and cached.
cudaError_t noalloc_records(float4 **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_records);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<float4 *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace gbl
