/*
 * Core/tail split of the beam profile and the learned tail surrogate.
 *
 * The profile of Sec. II-B's centered kernel has a narrow core and a long
 * tail (the blooming part): for a radial profile truncated at 2 degrees with
 * a 0.05 degree Gaussian core, the tail covers about 100x the pixels of a
 * 0.2 degree core while carrying a small fraction of the energy. These calls
 * let the exact footprint integration (Alg. 1's beam iteration) run on the
 * core only and take the tail's contribution from a coarse range histogram
 * (a physics estimate or a learned prediction). The result stays within the
 * accuracy of the exact method: every such beam passes an acceptance test
 * built from guaranteed bounds of the tail, or is re-run exactly.
 *
 * The paper computes the whole profile directly; the split, the bounds and the
 * network are this library's own additions.
 *
 * Radial profiles only (LIDAR_PROFILE_RADIAL); the FP32 shared-memory atomic
 * deposit is used for every pass. All pointers below are device pointers
 * unless stated otherwise; streams are cudaStream_t passed as void*.
 *
 * Coarse rows. Per beam, a row of n_coarse + 4 floats:
 *   [0, n_coarse)  mass of the histogram xi_b (before the pulse convolution)
 *                  per coarse bin; coarse bin c covers fine bins
 *                  [c * f, (c + 1) * f), f = n_bins / n_coarse
 *   [n_coarse]     ambient sum A_b (profile-weighted ambient radiance x d omega)
 *   [n_coarse + 1] bound E of the tail's deposited mass: no tail can deposit
 *                  more than E in total
 *   [n_coarse + 2] bound of the error of the ambient entry
 *   [n_coarse + 3] total of [0, n_coarse)
 */
#ifndef LIDAR_TAIL_H
#define LIDAR_TAIL_H

#include "lidar.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Net input per beam: a 4-level pyramid of 64x64, 32x32, 16x16 and 8x8 cells
 * (cells of 4, 8, 16 and 32 G-buffer pixels per side, centred on the beam's
 * axis), 2 FP16 channels per cell (channel-interleaved, levels in order). */
#define LIDAR_TAIL_INPUT_CELLS 5440

/* Enables the split on a sensor: exact core radius core_deg (0 < core_deg <
 * profile truncation), n_coarse coarse bins (n_bins % n_coarse == 0,
 * n_coarse <= 1024). Allocates per-beam device buffers (about
 * n_beams * (n_coarse + 4) * 8 bytes plus flags) and, on first use, cell sums
 * of the G-buffer. Call again to change the parameters.
 * Errors: LIDAR_EINVAL (table profile, bad sizes), LIDAR_ENOMEM, LIDAR_ECUDA. */
lidar_status_t lidar_tail_configure(lidar_t *l, double core_deg, int32_t n_coarse);

/* Per-beam tail features of one frame. Fills `rows` ([n_beams][n_coarse + 4],
 * device, written) with the physics estimate of each beam's tail (coarse rows
 * above: the estimate in [0, n_coarse] and [n_coarse + 3], the bounds in
 * [n_coarse + 1] and [n_coarse + 2]) and, if `inputs` is not NULL, the network
 * input ([n_beams][LIDAR_TAIL_INPUT_CELLS] half2, device, written).
 * Asynchronous on `stream`. Errors: LIDAR_EINVAL (not configured, bad
 * G-buffer or pose; a 2 pi panorama whose width is not a multiple of 32
 * pixels), LIDAR_ENOMEM, LIDAR_ECUDA. */
lidar_status_t lidar_tail_features(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *rows,
                                   void *inputs, void *stream);

/* The exact tail of every beam: the footprint integration restricted to the
 * annulus core < theta <= truncation, reduced to coarse rows ([n_beams]
 * [n_coarse + 4], device, written; entries [n_coarse + 1] and [n_coarse + 2]
 * are 0, [n_coarse + 3] the total). This is the training target of the
 * network. Uses internal waveform scratch (allocated on first use).
 * Asynchronous on `stream`. */
lidar_status_t lidar_tail_exact(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *rows,
                                void *stream);

/* One frame with the split: exact core of every beam plus the coarse tail
 * `tail` ([n_beams][n_coarse + 4], device, read; each coarse bin's mass spread
 * evenly over its fine bins, the ambient entry added to A_b), then the pulse
 * convolution and echo extraction. A beam is re-run with the exact full
 * profile unless its waveform passes the acceptance test: with E the tail
 * bound of its row and dA the ambient bound, (1) sqrt(2) E ||p||_2 + dA s_amb
 * sqrt(n_bins) <= 5e-4 ||xi||_2, (2) no bin within E max(p) + dA s_amb of T,
 * (3) the peak bin ahead of every other bin of its echo by more than the most
 * the tail can change their difference, (4) the worst-case movement of the
 * threshold crossings and of the log-parabola peak vertex <= 0.25 mm, and of
 * ln(intensity) and the peak value <= 3e-4. The tail entries must be
 * non-negative with total <= E (as `lidar_tail_features` and
 * `lidar_tailnet_predict` produce them). Outputs as `lidar_simulate`.
 * *n_fallback (host, may be NULL) receives the number of beams re-run.
 * Synchronises `stream` once (reads the number of re-run beams). */
lidar_status_t lidar_simulate_split(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, const float *tail,
                                    float *out_waveforms, lidar_echoes_t *out_echoes, int32_t *n_fallback,
                                    void *stream);

/* ------------------------------------------------------------------------
 * Learned tail surrogate: a small convolutional network that maps a beam's
 * input pyramid and physics prior to its coarse tail.
 *
 * Per beam, with s = max(prior mass, 0.1 E) the beam's scale (E the tail
 * bound of its row) and p = prior / s:
 *   a1 = relu(conv1(L0)), a2 = relu(conv2([a1, L1])), a3 = relu(conv3([a2, L2]))
 *        (3x3 convolutions of stride 2 with one pixel of zero padding,
 *        32 channels: 64^2 -> 32^2 -> 16^2 -> 8^2)
 *   h  = relu(W1 [a3, L3, p] + b1)            256 hidden units
 *   y  = relu(p + W2 h + b2)                  n_coarse outputs; tail = s y
 * trained with the L1 loss mean_b sum_c |y - target / s| (beams with s = 0
 * excluded). Weights and activations are FP16 with FP32 accumulation on the
 * tensor cores; the master weights and Adam state are FP32.
 *
 * Parameter vector (FP32, each tensor zero-padded to a multiple of 8 floats):
 *   conv1 [32][32] (column tap * 2 + c, tap = 3 ky + kx; columns >= 18 zero),
 *   b1 [32], conv2 [32][320] (column tap * 34 + c: c < 32 from a1, then L1;
 *   columns >= 306 zero), b2 [32], conv3 [32][320] (as conv2), b3 [32],
 *   W1 [256][2176 + n_coarse] (a3 as (y, x, c), L3 as (y, x, c), then p),
 *   b1 [256], W2 [n_coarse][256], b2 [n_coarse].
 * The paper has no counterpart of the network; the scheme is this library's.
 * ------------------------------------------------------------------------ */
typedef struct lidar_tailnet lidar_tailnet_t;

/* New network with He-uniform weights from `seed`, a zero output layer (the
 * first prediction is the prior) and zero Adam state. n_coarse: a multiple of 8
 * in [8, 1024], equal to the sensor's. Errors: LIDAR_EINVAL, LIDAR_ENOMEM,
 * LIDAR_ECUDA. */
lidar_status_t lidar_tailnet_create(int32_t n_coarse, uint64_t seed, lidar_tailnet_t **out);
void lidar_tailnet_destroy(lidar_tailnet_t *net);
const char *lidar_tailnet_last_error(const lidar_tailnet_t *net);
/* Number of floats of the parameter vector. */
int64_t lidar_tailnet_num_params(const lidar_tailnet_t *net);
/* Copies of the FP32 parameter vector (host memory, `count` floats). */
lidar_status_t lidar_tailnet_get_params(const lidar_tailnet_t *net, float *host, int64_t count);
lidar_status_t lidar_tailnet_set_params(lidar_tailnet_t *net, const float *host, int64_t count);

/* Predicted tails of n_beams beams: inputs ([n][LIDAR_TAIL_INPUT_CELLS] half2)
 * and rows ([n][n_coarse + 4], from lidar_tail_features) in, tail_out
 * ([n][n_coarse + 4]) out: s y clipped to total <= E, the ambient entry and
 * bounds copied from rows, the total in [n_coarse + 3] (the layout
 * lidar_simulate_split takes). Device pointers; asynchronous on `stream`;
 * internal scratch of about 400 MB for 65536-beam chunks is allocated on first
 * use. The three convolutions run fused per beam (one launch per chunk). */
lidar_status_t lidar_tailnet_predict(lidar_tailnet_t *net, const void *inputs, const float *rows, int32_t n_beams,
                                     float *tail_out, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on a batch:
 * inputs and rows as for predict, target ([batch][n_coarse + 4], from
 * lidar_tail_exact). *loss_host (may be NULL) receives the batch loss, which
 * synchronises `stream`. Gradients use a static loss scale of 1024; a batch
 * with a non-finite gradient leaves the weights unchanged. */
lidar_status_t lidar_tailnet_train_step(lidar_tailnet_t *net, const void *inputs, const float *rows,
                                        const float *target, int32_t batch, float lr, float *loss_host, void *stream);

/* Loss and gradient of a batch without a step (host outputs, either may be
 * NULL; grads_host holds lidar_tailnet_num_params floats). Synchronises. */
lidar_status_t lidar_tailnet_grads(lidar_tailnet_t *net, const void *inputs, const float *rows, const float *target,
                                   int32_t batch, float *grads_host, float *loss_host, void *stream);

/* Checkpoint file: header, FP32 parameters and, with with_state != 0, the
 * Adam moments and step count (resumable training). Little-endian. */
lidar_status_t lidar_tailnet_save(const lidar_tailnet_t *net, const char *path, int32_t with_state);
/* Loads a file written by lidar_tailnet_save (a file without state resets
 * the Adam state). Errors: LIDAR_EINVAL (missing, truncated, other shape). */
lidar_status_t lidar_tailnet_load(lidar_tailnet_t *net, const char *path);

/* Per-stage timing of lidar_tailnet_predict: while enabled, CUDA events are
 * recorded on the call's stream around the fused convolution launch and
 * around the dense layers (two GEMMs, output and clipping) of every chunk of
 * up to 65536 beams. _read synchronises on the last event and returns the
 * totals (ms) and counts [convolutions, dense layers] since the last read.
 * Enabling or disabling drops unread records. */
lidar_status_t lidar_tailnet_profile_enable(lidar_tailnet_t *net, int32_t enable);
lidar_status_t lidar_tailnet_profile_read(lidar_tailnet_t *net, double total_ms[2], int32_t launches[2]);

/* Which kernel runs the network's forward GEMMs: the three convolutions
 * of training (as im2col GEMMs) and both dense layers of training and
 * prediction. The fused convolutions of prediction and all gradient GEMMs
 * use the mma.sync kernels in either mode.
 *   LIDAR_DENSE_TCGEN05   (default) 5th-generation tensor cores: 256-row
 *                         tiles, FP16 operands copied by TMA into swizzled
 *                         shared memory, FP32 accumulators in tensor memory;
 *                         used when the output width is a multiple of 16 up
 *                         to 256, else the mma.sync kernel runs.
 *   LIDAR_DENSE_MMA_SYNC  64 x 64 tiles of mma.sync m16n8k16 (FP32 accumulators
 *                         in registers).
 * Both accumulate in FP32; results differ by rounding order only. */
enum { LIDAR_DENSE_TCGEN05 = 0, LIDAR_DENSE_MMA_SYNC = 1 };
lidar_status_t lidar_tailnet_set_dense(lidar_tailnet_t *net, int32_t mode);

/* Synchronises `stream` and reports errors of the network's asynchronous
 * work since the last check: LIDAR_ECUDA for a CUDA error, LIDAR_ETIMEOUT if a
 * bounded wait of the tensor-core GEMM gave up (its outputs are then
 * undefined). Clears the recorded timeout. */
lidar_status_t lidar_tailnet_sync(lidar_tailnet_t *net, void *stream);

/* One frame through the surrogate: lidar_tail_features, lidar_tailnet_predict
 * (or the physics prior when net is NULL) and lidar_simulate_split. Per-beam
 * scratch (about 22 KB per beam for the network input) is allocated on first
 * use. Synchronises `stream` once. */
lidar_status_t lidar_simulate_surrogate(lidar_t *l, lidar_tailnet_t *net, const lidar_gbuffer_t *g,
                                        const lidar_pose_t *pose, float *out_waveforms, lidar_echoes_t *out_echoes,
                                        int32_t *n_fallback, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LIDAR_TAIL_H */
