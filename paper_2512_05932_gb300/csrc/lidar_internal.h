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
    // the same split for precision: x_scale = xs_hi + xs_lo, x_off = xo_int +
    // xo_fr (xo_int an integer); vh = 1 - cos(daz/2), vv = 1 - cos(del/2)
    float xs_hi, xs_lo, xo_int, xo_fr, vh, vv;
    int n_bins;
    int pad;                 // zero padding (bins) of the footprint kernel's histogram buffer
    const uint8_t *core_only;  // per beam: 1 = only the core of the profile (box radius core_rad)
    double core_rad;
    const int *beam_ids;     // beam slot b takes pattern direction beam_ids[b] (NULL: b)
    int bin_records;         // narrow records carry the first bin index (tensor-core deposit)
                             // instead of histogram positions (shared-memory atomics)
    int pix_blocks;
    long pix_begin, pix_end; // setup_kernel: the pixels [pix_begin, pix_end) only
    unsigned *wmax;          // non-NULL: atomic max of the records' deposit weights (FP32 bits)
    // beams
    int n_beams;
    const float *dirs;       // [n_beams][3]
    double R[9];
    double az0d, el0d, dazd, deld;
    int panorama;
    double support_rad;
    double sup_u, sup_v;     // half-widths (rad) of a table / separable profile's rectangle (0: radial)
    double cos_sup;          // cos(support_rad)
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
    cudaTextureObject_t nodes;  // table: (w+2) x (h+2) zero-ringed nodes divided by Z (zero outside)
    int qw, qh;
    // separable profile P = H(u) V(v) (kind LIDAR_PROFILE_SEPARABLE):
    const float2 *hpairs;  // [qw]: (H[i], H[i+1]) of the zero-padded H, divided by Z
    const float2 *vpairs;  // [qh]: (V[j], V[j+1]) of the zero-padded V
    // table coordinate = offset_rad * tk + ti{u,v} + tc{u,v}, ti an integer,
    // tc in [0, 1); ti{u,v}1 = ti{u,v} + 1 (the gather's texel coordinate)
    float tk, tcu, tcv, tiu, tiv, tiu1, tiv1;
    // pulse and bins
    int n_bins, nch, M, R;
    const float *taps_pad;  // length tp_len, tap m at index tp_off + m
    int tp_len, tp_off;
    int tc_split;            // tensor-core deposit: 1 = BF16 hi/lo split (3 MMAs), 0 = plain BF16
    // core/tail split of a radial profile (learned tail surrogate)
    float core2;             // support radius^2 (rad^2) of beams flagged core-only
    float inner2;            // samples with theta^2 <= inner2 are left out (annulus), < 0: none
    // Rows of tail_in / coarse_out have tail_stride = n_coarse + 4 floats:
    //   [0, n_coarse)  coarse histogram (n_bins / n_coarse fine bins per coarse bin)
    //   [n_coarse]     ambient sum
    //   tail_in only:  [n_coarse + 1] bound on the tail's deposited mass,
    //                  [n_coarse + 2] bound on the ambient estimate's error
    const float *tail_in;    // coarse tail of core-only beams (convolved with tail_box); NULL: none
    const float *tail_box;   // pulse averaged over cf fine bins, B(x) at index x + tb_off,
                             // x in [-M - 7, M + cf + 6] (zero outside [-M, M + cf - 1]);
                             // 16-byte aligned base, tb_off a multiple of 4
    int tb_off;
    float *coarse_out;       // coarse histogram and ambient sum of every beam; NULL: none
    int n_coarse, tail_stride;
    // acceptance test of core-only beams (pulse constants of the FP32 taps:
    // max tap, L2 norm, max |p[i+1]-p[i]|, max |p[i+2]-p[i]|, max |p[i+1]-2p[i]+p[i-1]|)
    float g_pmax, g_pl2, g_d1, g_d2, g_dd;
    float g_l2, g_dr;        // relative L2 budget of the tail error; range / EPW budget (m)
    uint8_t *fb_flags;       // [n_beams]: set to 1 for beams that fail the test (cleared by the caller)
    const int *out_ids;      // beam slot b writes output row out_ids[b] (NULL: b)
    // calibration
    float T, s_amb;
    int max_echoes;
    int strongest;           // 1: only the echo of largest intensity (first on ties) is kept
    float c0, c1, c2;
    float rA, rB;          // range of bin-centre coordinate x: rA + x * rB
    // outputs
    float *wave;             // [n_beams][n_bins] (unless slot_pool is set)
    lidar_echo_t *echoes;
    int32_t *counts;
    // echo-only simulation: each CTA keeps its beams' waveforms in a slot of
    // slot_pool (G * n_bins floats) that it claims from slot_busy (0 free,
    // 1 held) and frees at exit; n_slots >= the CTAs the GPU holds at once.
    // NULL: waveforms are outputs in `wave`.
    float *slot_pool;
    int *slot_busy;
    int n_slots;             // slot_sms * slots_per_sm
    int slot_sms, slots_per_sm;
    int *err;                // set to 1 if a slot claim or a tensor-core pipeline wait gives up
    // tcgen05 deposit (FP16 operands): the frame's largest record weight
    // (FP32 bits, from the setup kernel) and the profile's maximum
    const unsigned *umma_wmax;
    float umma_pmax;
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
    const unsigned *wmax;    // tcgen05 deposit with FP16 operands: the frame's largest record weight
};

// Device address of the fixed scratch of lidar_simulate_noalloc on the current
// device (lidar_noalloc.cu); lidar_create looks it up once per handle.
cudaError_t noalloc_records(float4 **out);

// Launch helpers (lidar_kernels.cu). Return cudaSuccess or the launch error.
cudaError_t launch_setup(const SetupArgs &a, cudaStream_t s);
size_t footprint_smem_bytes(int G, const FootprintArgs &a);
int footprint_pad(int M);
cudaError_t prepare_footprint(int kind, int G, bool tc, size_t smem);
cudaError_t footprint_occupancy(int kind, int G, bool tc, int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_footprint(int kind, int G, bool tc, int threads, size_t smem, const FootprintArgs &a,
                             cudaStream_t s);
cudaError_t launch_setup_batch(const SetupArgs *frames, const int *pix_blk, const int *beam_blk, int n_frames,
                               int total_blocks, int *counter, cudaStream_t s);
cudaError_t prepare_footprint_batch(int kind, int G, bool tc, size_t smem);
// tcgen05 deposit (16 beams per CTA, histograms in tensor memory)
size_t umma_smem_bytes(int n_bins, int M);
constexpr int kUmmaBeams = 16;
constexpr int kUmmaMaxBins = 4096;  // 32 blocks of 128 bins x 16 beams = 512 TMEM columns
cudaError_t prepare_umma(int kind, bool bf16, size_t smem);
cudaError_t launch_umma(int kind, bool bf16, size_t smem, const FootprintArgs &a, cudaStream_t s);
cudaError_t launch_umma_batch(int kind, bool bf16, int grid, size_t smem, const FootprintArgs &base,
                              const FrameDesc *frames, const int2 *items, int n_items, int *counter, cudaStream_t s);
cudaError_t launch_footprint_batch(int kind, int G, bool tc, int threads, int grid, size_t smem,
                                   const FootprintArgs &base, const FrameDesc *frames, const int2 *items,
                                   int n_items, int *counter, cudaStream_t s);

}  // namespace gbl
