// Internal types shared by the host API (lidar_api.cpp) and the kernels
// (lidar_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lidar.h"

namespace gbl {

constexpr int kMaxBins = 16384;
constexpr long kNoAllocMaxPixels = 1L << 20;  // G-buffer size limit of lidar_simulate_noalloc
constexpr int kWarp = 32;
constexpr uint32_t kNoDeposit = 0xFFFFFFFFu;
constexpr int kBinBias = 8;           // bin indices in records are stored + kBinBias (>= 0)
constexpr float kMuMin = 1e-3f;       // grazing clamp of |d.n| in the range interval
constexpr float kNearRel = 1e-4f;     // threshold guard band (flag only)

// Per-beam geometry, written by the setup kernel in FP64 and stored in FP32
// relative to the pixel grid (64 bytes).
struct BeamParam {
    int ci, ri;         // integer part of the axis' pixel coordinates (centre of pixel u is u)
    float cf, rf;       // fractional part, in [0, 1)
    float sin_elb, cos_elb;
    float cg, sg;       // in-plane rotation from the G-buffer's east/north frame to the beam frame
    int row0, row1;     // candidate rows (inclusive), clamped to the G-buffer
    int col0, col1;     // candidate columns (inclusive, unwrapped for a 2 pi panorama)
    int valid;
    int pad0;
    float pad1, pad2;
};
static_assert(sizeof(BeamParam) == 64, "BeamParam layout");

struct SetupArgs {
    // pixels
    int U, V;
    float az0, el0, daz, del;
    float ch, sh, cv, sv;    // cos/sin of daz/2 and del/2
    const float *range, *nx, *ny, *nz, *rho, *retro, *amb;
    float4 *rec;             // [U*V][2]: 32-byte per-pixel records
    float x_scale, x_off;    // bin-centre coordinate X = r * x_scale + x_off
    int n_bins;
    int pad;                 // zero padding (bins) of the footprint kernel's histogram buffer
    int bin_records;         // narrow records carry the first bin index (tensor-core deposit)
                             // instead of histogram positions (shared-memory atomics)
    int pix_blocks;
    // beams
    int n_beams;
    const float *dirs;       // [n_beams][3]
    double R[9];
    double az0d, el0d, dazd, deld;
    int panorama;
    double support_rad;
    BeamParam *beams;
};

struct FootprintArgs {
    int U, V, panorama;
    float az0, el0, daz, del;
    const float4 *rec;
    const BeamParam *beams;
    int n_beams;
    // profile
    float kg;          // -log2(e) / (2 sigma^2), rad^-2 (radial)
    float trunc2;      // support radius^2, rad^2 (radial)
    float tail_amp, tc2_inv, tail_hp;  // radial tail: amp * min(1, (t2 * tc2_inv)^hp)
    float invZ;
    const float4 *quads;   // (h+1) rows of (w+1) corner quads, already divided by Z (table)
    int qw, qh;
    float tk, tcu, tcv;    // table coordinate = offset_rad * tk + tc{u,v}
    // pulse and bins
    int n_bins, nch, M, R;
    const float *taps_pad;  // length tp_len, tap m at index tp_off + m
    int tp_len, tp_off;
    int tc_split;            // tensor-core deposit: 1 = BF16 hi/lo split (3 MMAs), 0 = plain BF16
    // calibration
    float T, s_amb;
    int max_echoes;
    float c0, c1, c2;
    float rA, rB;          // range of bin-centre coordinate x: rA + x * rB
    // outputs
    float *wave;
    lidar_echo_t *echoes;
    int32_t *counts;
};

// Per-frame fields of the batched footprint kernel.
struct FrameDesc {
    int U, V, panorama, n_beams;
    float az0, el0, daz, del;
    const float4 *rec;
    const BeamParam *beams;
    float *wave;
    lidar_echo_t *echoes;
    int32_t *counts;
};

// Device address of the fixed scratch of lidar_simulate_noalloc on the current
// device (lidar_noalloc.cu); looked up on first use per device.
cudaError_t noalloc_records(float4 **out);

// Launch helpers (lidar_kernels.cu). Return cudaSuccess or the launch error.
cudaError_t launch_setup(const SetupArgs &a, cudaStream_t s);
size_t footprint_smem_bytes(int G, const FootprintArgs &a);
int footprint_pad(int M);
cudaError_t prepare_footprint(int kind, int G, bool tc, size_t smem);
cudaError_t launch_footprint(int kind, int G, bool tc, int threads, size_t smem, const FootprintArgs &a,
                             cudaStream_t s);
cudaError_t launch_setup_batch(const SetupArgs *frames, const int *pix_blk, const int *beam_blk, int n_frames,
                               int total_blocks, int *counter, cudaStream_t s);
cudaError_t prepare_footprint_batch(int kind, int G, bool tc, size_t smem);
cudaError_t launch_footprint_batch(int kind, int G, bool tc, int threads, int grid, size_t smem,
                                   const FootprintArgs &base, const FrameDesc *frames, const int2 *items,
                                   int n_items, int *counter, cudaStream_t s);

}  // namespace gbl
