/*
 * Range stacking (the paper's Alg. 2, Sec. II-C): a pixel-dense image of the
 * nearest range slice whose kernel-weighted intensity reaches a threshold.
 *
 * Every pixel is treated as the centre of a beam. Per-pixel inputs come from
 * the same G-buffer as lidar_simulate: the intensity I = rho_hat * d omega of
 * a hit pixel (rho_hat = (rho_d / pi + g) |cos theta| / R^2, d omega the
 * pixel's exact solid angle; 0 without a hit) and the range index
 * floor(R / dr). For every slice s = s_max .. 1 the slice image (I where the
 * range index is s, else 0) is convolved with the centred kernel K[kh][kw]
 * (zero outside the image; out[v][u] = sum_{a,b} K[a][b] in[v - a + kh/2]
 * [u - b + kw/2]) and each pixel whose value is >= threshold takes s and that
 * value. Result per pixel: the smallest such s and its value, or s_max and 0.
 * s_max = floor(r_max / dr).
 *
 * The GPU takes the slices present in each 32x32-pixel output tile's region
 * nearest first and convolves each one densely over the tile, visiting only
 * the kernel rows whose region rows hold pixels of the slice, until every
 * output of the tile has its answer; the result is the same as the far-to-near
 * sweep's. Empty slices cost nothing, and so do slices too weak to reach the
 * threshold anywhere in the tile. Kernels whose tile layout does not fit
 * shared memory (square kernels from 119x119) are evaluated instead by walking
 * each output's stencil once per pass while keeping the 16 nearest slices met
 * with their sums in registers (a pass repeats above them while a nearer
 * answer is still possible).
 */
#ifndef LIDAR_STACK_H
#define LIDAR_STACK_H

#include "lidar.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lidar_stack lidar_stack_t;

typedef struct {
    int32_t kh, kw;       /* kernel height (2M + 1) and width (2N + 1): odd, 1..129 */
    const float *kernel;  /* host, [kh][kw] row-major, finite and >= 0; copied at create */
    double threshold;     /* > 0 */
    double dr;            /* range resolution (m), > 0 */
    double r_max;         /* maximum range (m); 1 <= floor(r_max / dr) <= 65535 */
} lidar_stack_params_t;

/* Validates the parameters and copies the kernel to the device.
 * Errors: LIDAR_EINVAL (message via lidar_stack_last_error(NULL)),
 * LIDAR_ENOMEM, LIDAR_ECUDA. */
lidar_status_t lidar_stack_create(const lidar_stack_params_t *p, lidar_stack_t **out);

/* A separable kernel K[a][b] = col[a] row[b] (Sec. III-C: the measured
 * collector profile is a product of a vertical and a horizontal profile;
 * Alg. 2's convolution then splits into a row pass and a column pass).
 * Same definition and results as lidar_stack_create with that K (up to FP32
 * summation order); the GPU convolves each slice present in a 32x32-pixel
 * output tile with the row vector along every row of the tile's region, then
 * with the column vector, nearest slice first, so an output costs kh + kw
 * multiply-adds per slice instead of kh kw. Slices too weak to reach the
 * threshold anywhere in the tile are skipped as in the general form. */
typedef struct {
    int32_t kh, kw;       /* odd, 1..129 */
    const float *col;     /* host, [kh] (vertical, along v), finite and >= 0; copied at create */
    const float *row;     /* host, [kw] (horizontal, along u), finite and >= 0; copied at create */
    double threshold;     /* > 0 */
    double dr;            /* range resolution (m), > 0 */
    double r_max;         /* maximum range (m); 1 <= floor(r_max / dr) <= 65535 */
} lidar_stack_sep_params_t;

/* As lidar_stack_create, for K = col row^T. Errors as lidar_stack_create. */
lidar_status_t lidar_stack_create_separable(const lidar_stack_sep_params_t *p, lidar_stack_t **out);

/* One frame: g as for lidar_simulate (device planes, not modified);
 * out_slice ([V][U] int32) and out_intensity ([V][U] float) are device
 * buffers owned by the caller. Per-pixel scratch (6 bytes per pixel) is
 * allocated on first use and grown as needed. Asynchronous on `stream`.
 * Errors: LIDAR_EINVAL (bad G-buffer, NULL outputs), LIDAR_ENOMEM, LIDAR_ECUDA. */
lidar_status_t lidar_range_stack(lidar_stack_t *h, const lidar_gbuffer_t *g, int32_t *out_slice, float *out_intensity,
                                 void *stream);

const char *lidar_stack_last_error(const lidar_stack_t *h);
void lidar_stack_destroy(lidar_stack_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LIDAR_STACK_H */
