// Internal types of the core/tail split (lidar_tail.cu) and the tail network
// (lidar_net.cu), shared with the host API. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lidar_internal.h"

namespace gbl {

constexpr int kMipLevels = 4;     // cell sums with 4, 8, 16, 32 pixels per side
constexpr int kQuadLevels = 3;    // the annulus walk uses the 16-, 8- and 4-pixel cells
constexpr int kPrepWarps = 8;
constexpr int kPrepThreads = 32 * kPrepWarps;
constexpr int kPrepList = 512;    // refined cells per warp and level (multiple of 4)
constexpr int kNetInCells = 64 * 64 + 32 * 32 + 16 * 16 + 8 * 8;  // 2 FP16 channels each

struct MipArgs {
    int U, V;
    float az0, el0, daz, del, sv;
    const float *range, *nx, *ny, *nz, *rho, *retro, *amb;
    int ncx[kMipLevels], ncy[kMipLevels];
    float4 *s[kMipLevels];   // (sum w, sum w r, sum ambient d omega, 0)
    float2 *r[kMipLevels];   // (min r, max r) over pixels with w > 0
};

struct PrepArgs {
    int U, V, panorama;
    float daz, del;
    const BeamParam *beams;
    int n_beams;
    // radial profile, as in FootprintArgs
    float kg, trunc2, tail_amp, tc2_inv, tail_hp, invZ;
    float core, trunc;         // core and truncation radius (rad)
    float rho_top;             // radius bound of a top-level cell (rad)
    float refine[kQuadLevels]; // a cell at level l is refined when its nearest point is closer than refine[l]
    int ncx[kMipLevels], ncy[kMipLevels];
    const float4 *s[kMipLevels];
    const float2 *r[kMipLevels];
    float x_scale, x_off, inv_cf, inv_nb;
    int n_coarse;
    float *prior;              // [n_beams][n_coarse + 4]
    void *inputs;              // [n_beams][kNetInCells] half2, or NULL
};

cudaError_t launch_tail_mips(const MipArgs &a, cudaStream_t s);
cudaError_t launch_tail_prep(const PrepArgs &a, cudaStream_t s);
// Ordered list of the set flags: out[0] = count, out[1 + i] = i-th index with flags[index] != 0.
cudaError_t launch_compact(const uint8_t *flags, int n, int *out, cudaStream_t s);

}  // namespace gbl
