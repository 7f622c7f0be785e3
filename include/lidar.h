/*
 * lidar.h - C ABI of the GB300 (sm_103a) beam model library.
 *
 * The library computes, for every beam of a LiDAR steering pattern, the
 * received time-of-flight waveform and its echoes from a near-infrared
 * G-buffer, following Dudzik et al., "Physically-Based Simulation of
 * Automotive LiDAR" (IAVVC 2025, arXiv 2512.05932):
 *
 *   xi_b(r) = iint d omega (kappa eta)(Phi - Psi_b) rho_hat(Phi) delta(r - r(Phi))
 *                                          (Sec. II-B, centered-kernel equation)
 *   xi_hat  = varpi * xi + ambient,  echoes = maximal intervals xi_hat > T
 *                                          (Sec. II-C, EPW post-processing)
 *
 * discretised as the beam iteration of Alg. 1 over pixel centres, with each
 * pixel's power spread uniformly over its range interval (pixelRangeInterval
 * of Alg. 1, plane extrapolation of Sec. II-D) and projected onto linear hat
 * functions centred on the range bins.
 *
 * Conventions used throughout
 *   - Sensor frame: x forward, y left, z up. Directions are unit vectors.
 *   - G-buffer: equirectangular; pixel (u, v), 0 <= u < U along azimuth,
 *     0 <= v < V along elevation, centre at az = az0 + (u + 1/2) daz,
 *     el = el0 + (v + 1/2) del, direction (cos el cos az, cos el sin az, sin el).
 *     Planes are float32 [V][U], row v contiguous in u.
 *   - Bins: bin k covers time of flight [t0 + k dt, t0 + (k + 1) dt), centre
 *     t_k = t0 + (k + 1/2) dt, range r = c t / 2 (c = 299792458 m/s).
 *   - All intensities are relative (Sec. I-A: intensities reduce to relative
 *     values after calibration).
 *
 * Ownership: the caller owns every buffer it passes. The library copies the
 * profile table, the beam directions and the pulse at lidar_create time and
 * owns internal device scratch (per-pixel records and per-beam parameters),
 * which it grows with cudaMalloc when a larger G-buffer arrives.
 *
 * Errors: every entry point returns a lidar_status_t and never aborts; a
 * message for the last failure is available from lidar_last_error.
 * Thread safety: one lidar_t may be used by one host thread at a time.
 */
#ifndef GB300_LIDAR_H
#define GB300_LIDAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LIDAR_OK = 0,
    LIDAR_EINVAL = 1,   /* invalid argument (message says which) */
    LIDAR_ENOMEM = 2,   /* host or device allocation failed */
    LIDAR_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    LIDAR_ETIMEOUT = 4, /* a bounded device wait gave up (reported at the next sync) */
    LIDAR_ENUMERIC = 5  /* calibration fit or normalisation failed */
} lidar_status_t;

/* Beam x sensitivity profile kappa*eta of Sec. III-C, centred on the beam
 * (Sec. II-B, centered kernel). Offsets (u, v) are in degrees in the beam's
 * local tangent frame (azimuthal-equidistant): u along e1 = z x dir
 * (increasing azimuth), v along e2 = dir x e1 (increasing elevation), both
 * taken in the sensor frame and rotated with the pose. The library
 * normalises the profile to unit integral over the sphere at create time.
 *
 *   LIDAR_PROFILE_RADIAL: P(theta) = exp(-theta^2 / (2 sigma^2))
 *                         + tail_amp * min(1, (theta / tail_core)^(-tail_pow))
 *                         for theta <= trunc, 0 beyond (theta in degrees).
 *   LIDAR_PROFILE_TABLE:  bilinear interpolation of table[h][w] (row j <-> v,
 *                         column i <-> u), node (i, j) at
 *                         u = (i - (w-1)/2) pitch, v = (j - (h-1)/2) pitch,
 *                         extended by one ring of zeros (P falls linearly to 0
 *                         one pitch beyond the edge nodes). Values >= 0.
 *   LIDAR_PROFILE_SEPARABLE: P(u, v) = H(u) V(v), a separable kernel (the
 *                         measured collector sensitivity of Sec. III-C is a
 *                         product of a horizontal and a vertical profile).
 *                         table holds H (table_w nodes along u) followed by V
 *                         (table_h nodes along v), nodes placed as for TABLE;
 *                         each is interpolated linearly and falls to 0 one
 *                         pitch beyond its end nodes. This is exactly the
 *                         TABLE profile of the outer product V[j] H[i], but
 *                         stored and evaluated as two 1-D tables (w + h
 *                         values instead of w h), which stay in the L1 cache. */
typedef enum {
    LIDAR_PROFILE_RADIAL = 0,
    LIDAR_PROFILE_TABLE = 1,
    LIDAR_PROFILE_SEPARABLE = 2
} lidar_profile_kind_t;

typedef struct {
    int32_t kind;          /* lidar_profile_kind_t */
    double sigma_deg;      /* RADIAL */
    double tail_amp;
    double tail_core_deg;
    double tail_pow;
    double trunc_deg;      /* RADIAL support radius, (0, 10] degrees */
    int32_t table_w;       /* TABLE, SEPARABLE: 2..4096 */
    int32_t table_h;       /* TABLE, SEPARABLE: 2..4096 */
    double pitch_deg;      /* node spacing; half-diagonal of the support <= 10 deg */
    const float *table;    /* host pointer, copied at create: TABLE [table_h][table_w];
                              SEPARABLE H[table_w] then V[table_h] */
} lidar_profile_t;

/* Beam set B with centre directions Psi_b (Sec. II-A), sensor frame.
 * Beams are processed in groups of consecutive indices: listing spatially
 * neighbouring beams next to each other (row-major scans, curve order) keeps
 * the groups' footprints compact. */
typedef struct {
    int32_t n_beams;       /* >= 1 */
    const float *dirs;     /* host pointer, [n_beams][3], nonzero (normalised inside) */
} lidar_pattern_t;

/* Range bins and emitted pulse varpi (Sec. II-C): Gaussian of the given FWHM
 * sampled at integer bin offsets -M..M with M = ceil(trunc_sigmas * sigma/dt),
 * normalised to unit sum. */
typedef struct {
    int32_t n_bins;        /* multiple of 32, 32..16384 */
    double dt_s;           /* bin width (s), > 0 */
    double t0_s;           /* time of flight at the start of bin 0 (range gate) */
    double fwhm_s;         /* pulse FWHM (s), > 0 */
    double trunc_sigmas;   /* truncation in standard deviations, (0, 12] */
} lidar_pulse_t;

/* Detection threshold, ambient scale and EPW -> intensity conversion
 * (Sec. II-C EPW, Sec. III-C threshold calibration). The intensity of an echo
 * is exp(c0 + c1 EPW^2 + c2 EPW^4) with EPW in metres. With fit_epw != 0,
 * lidar_create fits (c0, c1, c2) in FP64 by least squares on a sweep of
 * perpendicular point targets of energy a in [50 T, 1e6 T] (64 log-spaced
 * amplitudes x 4 sub-bin phases, no ambient): ln a = c0 + c1 EPW^2 + c2 EPW^4. */
typedef struct {
    double threshold;      /* T > 0; an echo is a maximal run of bins with xi_hat > T */
    double ambient_scale;  /* s_amb >= 0: xi_hat[k] += A_b * s_amb in every bin */
    int32_t max_echoes;    /* 1..3, nearest first */
    int32_t fit_epw;       /* != 0: fit epw_coef at create time */
    double epw_coef[3];    /* used when fit_epw == 0 */
} lidar_calib_t;

/* NIR G-buffer (Alg. 1 inputs rho_hat, varrho, nu plus the material planes
 * the library turns into rho_hat). Device pointers, float32 [V][U].
 *   range: metres along the pixel-centre ray; a pixel without a hit has a
 *          non-finite or non-positive range (it still receives ambient).
 *   nx, ny, nz: unit surface normal (either orientation).
 *   rho_d: NIR diffuse reflectance (BRDF rho_d / pi, Sec. I-A).
 *   retro: retroreflective BRDF gain g (sr^-1, Sec. I-B); beta = rho_d/pi + g.
 *   ambient: ambient radiance L_amb (relative), finite >= 0.
 * The azimuth span U*daz must not exceed 2 pi (exactly 2 pi wraps around);
 * the elevation span must stay within [-pi/2, pi/2]. */
typedef struct {
    int32_t U, V;
    double az0, el0, daz, del;   /* radians */
    const float *range, *nx, *ny, *nz, *rho_d, *retro, *ambient;
} lidar_gbuffer_t;

/* Pinhole G-buffer: a rasterised rendering (Sec. II-D, rasterization), which
 * follows a pinhole projection rather than the spherical grid of
 * lidar_gbuffer_t (Sec. II-C remarks that the beam kernels are then
 * inhomogeneous). Pixel (i, j), 0 <= i < W, 0 <= j < H, has its centre at
 * image coordinates X = (i + 1/2 - cx) / fx, Y = (j + 1/2 - cy) / fy and
 * looks along the camera-frame direction (X, Y, 1); R (row-major 3x3) maps
 * camera-frame vectors to the sensor frame (its columns are the image x axis,
 * the image y axis and the optical axis). Planes are float32 [H][W], device
 * memory, with the meanings of lidar_gbuffer_t; normals in the sensor frame.
 * With depth_is_z != 0 the range plane holds z-buffer depth along the
 * optical axis (the distance along the pixel-centre ray is z |(X, Y, 1)|). */
typedef struct {
    int32_t W, H;
    double fx, fy, cx, cy;       /* pixels; fx, fy > 0 */
    double R[9];                 /* camera -> sensor frame, orthonormal (1e-3) */
    int32_t depth_is_z;
    const float *range, *nx, *ny, *nz, *rho_d, *retro, *ambient;
} lidar_pinhole_t;

/* Sensor pose: rotation R (row-major 3x3) taking sensor-frame vectors into the
 * G-buffer frame (a beam axis is R dir). Orthonormal with det +1 (1e-3). */
typedef struct {
    float R[9];
} lidar_pose_t;

enum {
    LIDAR_ECHO_CLIPPED_START = 1u,  /* run starts at bin 0 */
    LIDAR_ECHO_CLIPPED_END = 2u,    /* run ends at the last bin */
    LIDAR_ECHO_NEAR_THRESHOLD = 4u  /* a crossing bin lies within 1e-4 T of T */
};

/* One echo (32 bytes). Ranges in metres. bin_start/bin_end: first/last bin
 * above T; r0/r1 interpolate the two threshold crossings linearly, EPW =
 * r1 - r0; bin_peak = argmax in the run (lowest bin on ties); range_m is the
 * peak refined by a 3-point parabola on ln xi_hat (on xi_hat if a value is
 * <= 0); peak = xi_hat[bin_peak]. */
typedef struct {
    float range_m;
    float epw_m;
    float intensity;
    float peak;
    int32_t bin_peak;
    int32_t bin_start;
    int32_t bin_end;
    uint32_t flags;
} lidar_echo_t;

/* Echo outputs: device pointers. echoes[n_beams][max_echoes] (unused slots are
 * zero-filled), counts[n_beams] = number of echoes written (<= max_echoes). */
typedef struct {
    lidar_echo_t *echoes;
    int32_t *counts;
} lidar_echoes_t;

typedef struct lidar lidar_t;

/* Creates a simulator for one sensor: copies the profile, pattern and pulse to
 * the current CUDA device, normalises the profile (FP64) and, if asked, fits
 * the EPW -> intensity coefficients (FP64). Returns LIDAR_EINVAL for invalid
 * parameters without touching the GPU, LIDAR_ENOMEM/LIDAR_ECUDA on device
 * failures, LIDAR_ENUMERIC if the profile integrates to zero or the fit is
 * singular. On failure *out is NULL. */
lidar_status_t lidar_create(const lidar_profile_t *profile, const lidar_pattern_t *pattern,
                            const lidar_pulse_t *pulse, const lidar_calib_t *calib, lidar_t **out);

/* Reprojects a pinhole G-buffer onto the spherical grid of dst (Sec. II-C:
 * reprojection of the rendered images is one of the ways to use pinhole
 * renderings), so that lidar_simulate* can run on it. For each dst pixel with
 * centre direction v (sensor frame): v is projected through the pinhole; the
 * src pixel whose cell contains the projection (none if it falls outside the
 * image or behind the camera) gives the normal, reflectance, retro gain and
 * ambient radiance, and its range r along its own centre direction p is
 * extrapolated along the surface to v with the normal correction of
 * Sec. II-D: r_corr = (p . n) / (v . n) r (kept uncorrected where v . n is
 * below 1e-3 in magnitude or of the other sign than p . n). Pixels without a
 * source get range +inf and zeros. The projection and the cell choice are
 * FP64; the range correction forms p - v and v . n in FP64 and the small
 * remaining term in FP32 (relative error of the range about 1e-7).
 * src: pinhole planes (device, read); dst: the target grid (U, V, az0, el0,
 * daz, del as for lidar_simulate) with caller-owned device planes, all seven
 * written. Allocates nothing; asynchronous on `stream`.
 * Errors: LIDAR_EINVAL (sizes, intrinsics, rotation, NULL planes), LIDAR_ECUDA. */
lidar_status_t lidar_reproject_pinhole(const lidar_pinhole_t *src, const lidar_gbuffer_t *dst, void *stream);

/* Simulates all beams for one G-buffer and pose, enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream). Asynchronous: returns after
 * enqueueing; results are ready when the stream reaches this point.
 * out_waveforms: device float32 [n_beams][n_bins], xi_hat in beam order.
 * out_echoes: device echo arrays as described at lidar_echoes_t.
 * The first call with a larger G-buffer than before grows the internal
 * scratch with cudaMalloc (synchronising the device). Returns LIDAR_EINVAL for
 * invalid arguments (nothing is enqueued) and LIDAR_ECUDA if a launch fails. */
lidar_status_t lidar_simulate(lidar_t *lidar, const lidar_gbuffer_t *gbuffer, const lidar_pose_t *pose,
                              float *out_waveforms, lidar_echoes_t *out_echoes, void *stream);

/* Echo-only simulation: what a sensor reports (its echoes, Sec. II-C: echo
 * range, EPW and intensity per return), without the waveforms. Same
 * computation and results as lidar_simulate (up to the order of the FP32
 * deposit additions, which varies from run to run in both); the difference
 * is where each beam's waveform goes between the pulse convolution and the
 * echo scan. Each CTA of the footprint kernel
 * claims a slot of a library-owned pool that has, for every SM id below 256,
 * one slot per CTA an SM can hold (beams per CTA x n_bins floats each: 33.5 MB
 * for a 2048-bin sensor at 8 beams and 2 CTAs per SM, of which the slots of
 * the enabled SMs, about 20 MB on 152 SMs, are used), writes its beams'
 * waveforms there, scans them and frees the slot; the slots in use stay in
 * L2, so the waveform bytes (4 n_bins per beam, most of lidar_simulate's
 * output) do not reach HBM and no [n_beams][n_bins] buffer is needed.
 *   - The first call (and the first after lidar_set_deposit changes the beams
 *     per CTA) allocates the pool with cudaMalloc, synchronising the device.
 *   - Calls on several streams may overlap: slots are claimed atomically; a
 *     CTA whose SM's slots are all held takes any free slot of the pool.
 *   - A slot claim that gives up (bounded; not expected, see above) leaves
 *     that CTA's beams unwritten and is reported by lidar_sync as
 *     LIDAR_ETIMEOUT.
 * out_echoes and errors as for lidar_simulate. */
lidar_status_t lidar_simulate_echoes(lidar_t *lidar, const lidar_gbuffer_t *gbuffer, const lidar_pose_t *pose,
                                     lidar_echoes_t *out_echoes, void *stream);

/* Same computation from host memory: the G-buffer plane pointers in `gbuffer`
 * are HOST pointers, and the outputs are host arrays (waveforms
 * [n_beams][n_bins], echoes [n_beams][max_echoes], counts [n_beams]). The
 * library copies the inputs to device buffers it owns, simulates, copies the
 * results back and synchronises `stream` before returning. A frame of at
 * least 1216 beam groups is pipelined on library-owned streams that start
 * after the work already queued on `stream`: the G-buffer is set up in 8
 * bands of rows (planes in page-locked, device-mapped host memory are read in
 * place by the set-up kernel, others are first copied up band by band); the
 * beams run as 8 launches alternating between two streams (one launch's CTAs
 * fill the SMs the previous one is leaving), each started once the rows its
 * beams can reach (the profile's support radius around their elevation) are
 * set up, so that with beams ordered by elevation the first launches start
 * early; the waveforms of each launch are copied back while later ones run.
 * The planes must hold U*V floats each, the outputs the sizes above.
 * `wave` may be NULL: the echo-only form of lidar_simulate_echoes (waveforms
 * kept in L2-sized slots, only echoes and counts copied back; a slot-claim
 * timeout returns LIDAR_ETIMEOUT). */
lidar_status_t lidar_simulate_host(lidar_t *lidar, const lidar_gbuffer_t *gbuffer, const lidar_pose_t *pose,
                                   float *out_waveforms, lidar_echo_t *out_echoes, int32_t *out_counts,
                                   void *stream);

/* A sequence of frames from host memory (Alg. 1 per frame, as a sensor
 * stream of scans): frame f is described by gbuffer[f] and pose[f] (host
 * planes, as for lidar_simulate_host) and its results go to out_waveforms[f]
 * ([n_beams][n_bins] floats), out_echoes[f] and out_counts[f]. Each frame's
 * results are those of lidar_simulate_host on the same inputs (up to the order
 * of the FP32 deposit additions); the difference is that consecutive frames
 * overlap: frames alternate between two sets of library-owned device buffers,
 * so frame f + 1 is read over the host link and set up while frame f's beams
 * run and its waveforms come back, and frame f + 2 waits only for frame f.
 *   - Frames of fewer than 1216 beam groups, and a single frame, are run one
 *     after the other by lidar_simulate_host.
 *   - The frames may differ in size and field of view (each passes the checks
 *     of lidar_simulate_host); the second buffer set is allocated (cudaMalloc)
 *     on first use and grown to the largest frame.
 *   - Consecutive frames must not share output arrays (they are written
 *     concurrently); frames f and f + 2 may (f + 2 writes after f).
 *   - out_waveforms may be NULL: the echo-only form for every frame.
 *   - Per-kernel timing (lidar_profile_enable) is not recorded.
 * The pipeline starts after the work already queued on `stream` and the call
 * returns once every frame's results are in host memory. Errors: LIDAR_EINVAL
 * for n_frames < 0, a NULL array or output pointer, or a frame that fails the
 * checks of lidar_simulate_host (nothing is enqueued then); CUDA errors as for
 * lidar_simulate_host. n_frames == 0 does nothing. */
lidar_status_t lidar_simulate_host_frames(lidar_t *lidar, int n_frames, const lidar_gbuffer_t *gbuffer,
                                          const lidar_pose_t *pose, float *const *out_waveforms,
                                          lidar_echo_t *const *out_echoes, int32_t *const *out_counts,
                                          void *stream);

/* Same computation as lidar_simulate, for callers that cannot let the library
 * allocate device memory during a call: a host whose memory pool has already
 * reserved the GPU, or a real-time loop that must not allocate once running
 * (a cudaMalloc can fail, stall or synchronise the device mid-frame). The
 * paper has no counterpart; this is a property of the library only.
 * Instead of library-allocated scratch, the per-pixel records live in a fixed
 * device array of 2^20 records (32 MiB) that the library declares statically;
 * every GPU it is placed on holds it until the process exits. This call never
 * calls cudaMalloc or cudaFree.
 *   - G-buffers with more than 2^20 pixels (U * V) are rejected with
 *     LIDAR_EINVAL and a message naming the limit.
 *   - lidar_create looks up the array's device address (cudaGetSymbolAddress)
 *     on its device and keeps it in the handle. That lookup is also when the
 *     runtime places the array on the device (lazy module loading), so the
 *     32 MiB are committed by lidar_create, not by this call. If the lookup
 *     failed, this call returns LIDAR_ECUDA (or LIDAR_ENOMEM) naming it.
 *   - The call must run with the handle's device current (LIDAR_EINVAL
 *     otherwise). A device reset invalidates the handle, as it does its other
 *     device memory.
 *   - All calls, from every lidar_t in the process, share the one array on a
 *     device. Calls whose kernels overlap on the GPU (different streams or
 *     threads without ordering) race on it and give wrong results; order them
 *     on one stream or synchronise between them. Each call rewrites every
 *     record it reads, so the previous call's contents do no harm.
 *   - Profiling (lidar_profile_enable) does not record this call.
 * Arguments, outputs and errors are otherwise those of lidar_simulate. */
lidar_status_t lidar_simulate_noalloc(lidar_t *lidar, const lidar_gbuffer_t *gbuffer, const lidar_pose_t *pose,
                                      float *out_waveforms, lidar_echoes_t *out_echoes, void *stream);

/* One frame of a batch: a rendering (G-buffer) seen by one sensor at one pose.
 * A batch simulates many frames in one pass; this amortises the per-launch cost
 * the way one rendering serves all beams of a sensor (Sec. II-B). All sensors
 * of a batch must share the executor's sensor model (the same profile, pulse
 * and calibration given to lidar_create); their beam patterns may differ. */
typedef struct {
    const lidar_t *sensor;        /* beam pattern of this frame */
    lidar_gbuffer_t gbuffer;      /* device planes, as for lidar_simulate */
    lidar_pose_t pose;
    float *out_waveforms;         /* device [sensor's n_beams][n_bins] */
    lidar_echoes_t out_echoes;    /* device, as for lidar_simulate */
} lidar_frame_t;

/* Simulates n_frames frames, enqueued on `stream`, as two kernel launches: one
 * setup launch over every frame's pixels and beams, and one persistent
 * footprint launch whose CTAs take (frame, beam group) items from a device
 * counter, largest footprints first. The descriptor upload and both launches
 * are captured once into a CUDA graph per batch shape (frame count, sizes,
 * beam counts, tuning) and replayed; a new shape is captured anew. The call
 * waits (host side) until the previous batch of this executor has finished
 * reading its descriptors. Scratch for all frames (32 bytes per pixel, 64 per
 * beam) is grown with cudaMalloc when needed. Errors as lidar_simulate, plus
 * LIDAR_EINVAL if a frame's sensor has a different sensor model. */
lidar_status_t lidar_simulate_batch(lidar_t *executor, const lidar_frame_t *frames, int32_t n_frames, void *stream);

/* Autotuner for lidar_simulate_batch: times the batch (CUDA events on `stream`)
 * for every beam-group size (beams per CTA) that fits shared memory and for
 * 1 or 2 resident CTAs per SM, keeps the fastest for this executor, and
 * leaves the outputs of the last run in the frames' buffers. */
lidar_status_t lidar_autotune_batch(lidar_t *executor, const lidar_frame_t *frames, int32_t n_frames, void *stream);

/* Current batch tuning: beams per CTA and resident CTAs per SM. */
lidar_status_t lidar_batch_config(const lidar_t *executor, int32_t *beams_per_cta, int32_t *ctas_per_sm);

/* Synchronises `stream` and reports any asynchronous CUDA error as LIDAR_ECUDA,
 * and a slot claim of lidar_simulate_echoes that gave up as LIDAR_ETIMEOUT. */
lidar_status_t lidar_sync(lidar_t *lidar, void *stream);

/* Queries: number of beams, bins, echoes per beam, the profile normaliser Z
 * (integral of the raw profile over the sphere, sr) and the EPW coefficients
 * in use. Any output pointer may be NULL. */
lidar_status_t lidar_get_info(const lidar_t *lidar, int32_t *n_beams, int32_t *n_bins, int32_t *max_echoes,
                              double *profile_norm, double epw_coef[3]);

/* Number of kernel launches one lidar_simulate call enqueues. */
int32_t lidar_launches_per_simulate(const lidar_t *lidar);

/* How the footprint kernel adds a pixel's profile-weighted deposit into a
 * beam's range bins (same model, different arithmetic):
 *   LIDAR_DEPOSIT_ATOMIC   FP32 products, shared-memory atomic adds (default).
 *   LIDAR_DEPOSIT_TC_SPLIT tensor cores: for 16-pixel tiles, (bins x pixels)
 *                          hat weights times (pixels x beams) profile weights
 *                          with BF16 mma and FP32 accumulation, each factor
 *                          split into BF16 hi + lo parts (three products,
 *                          relative error ~2^-16 per product).
 *   LIDAR_DEPOSIT_TC_BF16  the same with plain BF16 factors (one product,
 *                          relative error ~2^-8 per product).
 *   LIDAR_DEPOSIT_TCGEN05_BF16  5th-generation tensor cores (tcgen05): 16
 *                          beams per CTA keep their histograms in tensor memory
 *                          (FP32); per 64-pixel tile and 128-bin block,
 *                          (bins x pixels) hat weights times (pixels x beams)
 *                          profile weights, both BF16 (relative error ~2^-8 per
 *                          product). The hat weights are built once per pixel
 *                          and tile for all 16 beams.
 *   LIDAR_DEPOSIT_TCGEN05_FP16  the same with FP16 factors, each side scaled
 *                          by a power of two (per CTA: the frame's largest
 *                          pixel weight and the profile's maximum near 2^14;
 *                          relative error ~2^-11 per product).
 * The mma.sync forms process 8 beams per CTA (4 when two CTAs of 8 would not
 * share an SM). The tcgen05 forms take n_bins <= 4096 and serve lidar_simulate,
 * lidar_simulate_noalloc and lidar_simulate_batch; the echo-only and the host
 * entry points reject them (LIDAR_EINVAL). Applies to later calls of this
 * simulator (a batch uses its executor's mode); LIDAR_EINVAL for an unknown
 * mode or one the simulator's n_bins does not allow. */
enum {
    LIDAR_DEPOSIT_ATOMIC = 0,
    LIDAR_DEPOSIT_TC_SPLIT = 1,
    LIDAR_DEPOSIT_TC_BF16 = 2,
    LIDAR_DEPOSIT_TCGEN05_BF16 = 3,
    LIDAR_DEPOSIT_TCGEN05_FP16 = 4
};
lidar_status_t lidar_set_deposit(lidar_t *lidar, int32_t mode);

/* Which echoes a beam reports (Sec. II-C: a sensor reports echoes, not the
 * waveform; the single-return mode of a sensor keeps one of them):
 *   LIDAR_ECHOES_NEAREST    the first max_echoes runs above T, nearest first
 *                           (default).
 *   LIDAR_ECHOES_STRONGEST  every run is evaluated and only the echo of largest
 *                           intensity is reported (the nearest of equal ones):
 *                           out_echoes->echoes[b][0], counts[b] 0 or 1, the
 *                           other entries zeroed.
 * Applies to later lidar_simulate*, lidar_simulate_echoes and
 * lidar_simulate_batch calls of this simulator (a batch uses its executor's
 * mode). LIDAR_EINVAL for another value. */
enum {
    LIDAR_ECHOES_NEAREST = 0,
    LIDAR_ECHOES_STRONGEST = 1
};
lidar_status_t lidar_set_echo_mode(lidar_t *lidar, int32_t mode);

/* Testing aid for the bounded wait of the echo-only form (the paper has no
 * counterpart): marks every slot of this simulator's echo-only waveform pool
 * held (held != 0) or free (held == 0), allocating the pool first if the
 * current deposit form has none yet. While the slots are held, a
 * lidar_simulate_echoes call cannot claim one: each of its CTAs polls a
 * bounded number of times (1024 passes over the pool, ~1 us apart), gives up,
 * writes nothing for its beams and sets the simulator's error word, which the
 * next lidar_sync reports as LIDAR_ETIMEOUT (and clears). Nothing waits
 * forever and no fault is raised. Synchronous: returns after the device has
 * finished the change; do not call it while a simulation of this simulator is
 * in flight. LIDAR_EINVAL for a NULL simulator, LIDAR_ECUDA / LIDAR_ENOMEM
 * from the allocation or the memset. */
lidar_status_t lidar_hold_echo_slots(lidar_t *lidar, int32_t held);

/* Per-kernel timing. While enabled, every lidar_simulate call records CUDA
 * events on its stream around each of its kernels (setup, footprint_wave).
 * lidar_profile_read synchronises those events, writes the summed device time
 * (ms) and launch count of each kernel into total_ms[2] and launches[2]
 * (either may be NULL), and clears the accumulated records. Enabling or
 * disabling clears them too. */
lidar_status_t lidar_profile_enable(lidar_t *lidar, int32_t enable);
lidar_status_t lidar_profile_read(lidar_t *lidar, double total_ms[2], int32_t launches[2]);

/* Message describing the last failure on `lidar` (or, for NULL, the last
 * failure of lidar_create on this thread). Never NULL. */
const char *lidar_last_error(const lidar_t *lidar);

/* Frees the simulator and its device memory. NULL is ignored. */
void lidar_destroy(lidar_t *lidar);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LIDAR_H */
