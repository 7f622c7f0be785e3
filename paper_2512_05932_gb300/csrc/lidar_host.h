// Host-side state of a sensor and the helpers shared by the host API files
// (lidar_api.cpp, lidar_tail_api.cpp). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lidar_internal.h"

namespace gbl {
struct TailState;
}

struct lidar {
    // sensor
    int32_t n_beams = 0;
    int32_t kind = 0;          // lidar_profile_kind_t (the footprint kernel's KIND)
    bool separable = false;    // LIDAR_PROFILE_SEPARABLE: pairs of H and V instead of quads
    double Z = 0.0;
    double support_rad = 0.0;
    double sup_u = 0.0, sup_v = 0.0;  // rectangular support (rad) of a table / separable profile
    // radial profile
    float kg = 0.f, trunc2 = 0.f, tail_amp = 0.f, tc2_inv = 0.f, tail_hp = 0.f;
    // table profile
    int32_t qw = 0, qh = 0;
    float tk = 0.f, tcu = 0.f, tcv = 0.f;
    // pulse and calibration
    int32_t n_bins = 0, M = 0, R = 0, tp_len = 0, tp_off = 0;
    double dt = 0.0, t0 = 0.0;
    double T = 0.0, s_amb = 0.0;
    int32_t max_echoes = 0;
    double coef[3] = {0, 0, 0};
    // launch shape
    int32_t G = 16, threads = 512;
    size_t smem = 0;
    // deposit form: 0 shared-memory atomics (FP32), 1 tensor cores BF16 hi/lo
    // split (3 MMAs), 2 tensor cores plain BF16; G_tc/smem_tc: its group shape
    int32_t deposit = 0;
    int32_t echo_mode = 0;  // LIDAR_ECHOES_NEAREST or LIDAR_ECHOES_STRONGEST
    int32_t G_tc = 8;
    size_t smem_tc = 0;
    // tcgen05 deposit (LIDAR_DEPOSIT_TCGEN05_*): shared memory per CTA, the
    // profile's maximum (divided by Z) and the frame's largest record weight
    // (written by the setup kernel; FP16 operands only)
    size_t smem_um = 0;
    double pmax = 0.0;
    unsigned *d_wmax = nullptr;
    int32_t *d_perm = nullptr;  // beam slot -> pattern beam: groups of 16 nearby beams
    int device = 0;
    // device memory owned by the library
    float *d_dirs = nullptr;
    std::vector<float> h_dirs;  // host copy of the pattern (row ranges of lidar_simulate_host's beam chunks)
    cudaArray_t d_nodes = nullptr;           // table profile: zero-ringed nodes / Z ((w + 2) x (h + 2) floats)
    cudaTextureObject_t node_tex = 0;        // point-sampled, zero border, unnormalised coordinates
    float2 *d_pairs = nullptr;  // separable: qw H pairs, then qh V pairs
    float *d_taps = nullptr;
    gbl::BeamParam *d_beams = nullptr;
    float4 *d_rec = nullptr;
    size_t rec_cap = 0;  // pixels
    // lidar_simulate_noalloc: device address of the library's fixed record
    // array on this handle's device, looked up by lidar_create (or the error
    // of that lookup)
    float4 *noalloc_rec = nullptr;
    cudaError_t noalloc_err = cudaSuccess;
    // host-memory entry point buffers
    float *d_planes = nullptr;
    size_t planes_cap = 0;  // pixels
    float *d_wave = nullptr;
    lidar_echo_t *d_echo = nullptr;
    int32_t *d_counts = nullptr;
    // lidar_simulate_host on large frames (simulate_host_pipelined): uploads on
    // copy_stream (band_ev[b]: band b uploaded), set-up on setup_stream at the
    // highest priority (setup_ev[b]: band b set up), footprint launches on
    // aux_stream[0] and [1] (chunk_ev[i]: launch i finished), result copies on
    // d2h_stream[0] and [1] (two copy engines); start_ev: the caller's earlier work done; join_ev: the
    // ends of the six pipeline streams, which the caller's stream joins.
    cudaStream_t copy_stream = nullptr, d2h_stream[2] = {nullptr, nullptr}, setup_stream = nullptr;
    cudaStream_t aux_stream[2] = {nullptr, nullptr};
    cudaEvent_t chunk_ev[8] = {};
    cudaEvent_t band_ev[8] = {}, setup_ev[8] = {};
    cudaEvent_t start_ev = nullptr, join_ev[6] = {};
    // lidar_simulate_host_frames: frames of odd index use this second set of
    // frame buffers (records, beam parameters, staged planes, results), so
    // that a frame is set up while the previous one runs; done_ev[p]: the ends
    // of the six pipeline streams after the last frame that used set p.
    float4 *d_rec2 = nullptr;
    size_t rec2_cap = 0;  // pixels
    gbl::BeamParam *d_beams2 = nullptr;
    float *d_planes2 = nullptr;
    size_t planes2_cap = 0;  // pixels
    float *d_wave2 = nullptr;
    lidar_echo_t *d_echo2 = nullptr;
    int32_t *d_counts2 = nullptr;
    cudaEvent_t done_ev[2][6] = {};
    // echo-only waveform pool (lidar_simulate_echoes): n_slots slots of
    // slot_floats / n_slots floats, their busy flags, and an error word
    float *d_slot_pool = nullptr;
    int *d_slot_busy = nullptr;
    int *d_err = nullptr;
    int n_slots = 0, slots_per_sm = 0;
    size_t slot_floats = 0;
    // sensor-model fingerprint (batch compatibility) and table hash
    uint64_t model_hash = 0;
    // batched execution
    int32_t batch_G = 8, batch_cps = 0;  // beams per CTA, CTAs per SM (0 = occupancy maximum)
    float4 *d_brec = nullptr;
    size_t brec_cap = 0;  // pixels
    gbl::BeamParam *d_bbeams = nullptr;
    size_t bbeams_cap = 0;  // beams
    unsigned char *d_blob = nullptr, *h_blob = nullptr;
    size_t blob_cap = 0;
    int *d_counter = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t blob_free = nullptr;
    bool blob_pending = false;
    cudaGraphExec_t gexec = nullptr;
    std::vector<long long> gkey;
    // per-kernel timing (lidar_profile_enable)
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // 3 events per recorded simulate call
    size_t ev_used = 0;
    // core/tail split (lidar_tail_api.cpp)
    gbl::TailState *tail = nullptr;
    char err[512] = "no error";
};

namespace gblh {

constexpr double kC = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;
constexpr double kMaxSupportDeg = 10.0;
constexpr int kHostChunks = 8;  // footprint launches per frame of lidar_simulate_host (large frames)
static_assert(kHostChunks == sizeof(lidar::chunk_ev) / sizeof(cudaEvent_t), "one event per chunk");
constexpr int kHostBands = 8;  // G-buffer upload bands of lidar_simulate_host (large frames)
static_assert(kHostBands == sizeof(lidar::band_ev) / sizeof(cudaEvent_t) &&
                  kHostBands == sizeof(lidar::setup_ev) / sizeof(cudaEvent_t), "one event per band");

lidar_status_t fail(lidar_t *l, lidar_status_t st, const char *fmt, ...);
lidar_status_t cuda_fail(lidar_t *l, cudaError_t e, const char *what);
lidar_status_t check_gbuffer(lidar_t *l, const lidar_gbuffer_t *g);
lidar_status_t check_pose(lidar_t *l, const lidar_pose_t *p, double R[9]);
lidar_status_t ensure_scratch(lidar_t *l, size_t pixels);
bool is_panorama(const lidar_gbuffer_t *g);
gbl::SetupArgs setup_args(const lidar_t *l, const lidar_t *sensor, const lidar_gbuffer_t *g, const double R[9],
                          float4 *rec, gbl::BeamParam *beams);
gbl::FootprintArgs model_args(const lidar_t *l);
void tail_free(lidar_t *l);  // lidar_tail_api.cpp

}  // namespace gblh
