// Fixed per-pixel scratch for lidar_simulate_noalloc.
//
// lidar_simulate keeps its per-pixel records in device memory it allocates
// (and grows) with cudaMalloc. Some callers cannot allow that: hosts whose
// memory pool reserves the whole GPU up front, and real-time loops that must
// not allocate once running (a cudaMalloc can fail, stall, or synchronise the
// device in the middle of a frame). For them the records live in the
// statically sized array below instead (kNoAllocMaxPixels * 32 bytes =
// 32 MiB per GPU, held until the process exits).
//
// When the memory is committed: the CUDA runtime loads a module (and places
// its __device__ variables) on a device when the module is first used there;
// with lazy module loading, the default of recent CUDA releases, that is the
// first time the array's address is looked up. lidar_create does that lookup
// on its device, so the 32 MiB are placed while the handle is created (a call
// that allocates anyway), never inside a lidar_simulate_noalloc call.
#include <cuda_runtime.h>

#include "lidar_internal.h"

namespace gbl {

// 32-byte record per G-buffer pixel, two float4 each.
static __device__ __align__(256) float4 g_noalloc_records[2 * (size_t)kNoAllocMaxPixels];

// Device address of the array on the current device. In host code the name
// g_noalloc_records stands for a host-side shadow, not a device address, so it
// must never be passed to a kernel directly: the address comes from
// cudaGetSymbolAddress with the device current. lidar_create calls this once
// per handle and keeps the result; a device reset invalidates it together
// with the handle's other device memory.
cudaError_t noalloc_records(float4 **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_records);
    if (e != cudaSuccess) return e;
    *out = static_cast<float4 *>(p);
    return cudaSuccess;
}

}  // namespace gbl
