// Internal types of the tail network kernels (lidar_net.cu) and their host
// side (lidar_net_api.cpp). Not part of the public ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace gbl {

enum { kGemmStore = 0, kGemmAtomic = 1, kGemmBiasRelu = 2, kGemmBias = 3 };

struct GemmArgs {
    int M, N, K;
    const __half *A;
    int lda;
    const __half *B;
    int ldb;
    int k_split;        // K range per blockIdx.z (multiple of 32)
    int mode;
    float *C;           // FP32 output (store / atomic / bias)
    __half *Ch;         // FP16 output (bias modes)
    int ldc;
    const float *bias;
};

struct Im2colArgs {
    int B, Hi, Wi, Ho, Wo, Ca, Kp;
    const __half *act;  // [B][Hi][Wi][Ca] or NULL (Ca = 0)
    const __half *x;    // network input, in_stride halves per beam
    long in_stride;
    long level_off;     // offset (halves) of the pyramid level within a beam's input
    __half *out;        // [B * Ho * Wo][Kp]
};

struct Col2imArgs {
    int B, Hi, Wi, Ho, Wo, Ca, Kp;
    const float *dcol;  // [B * Ho * Wo][Kp]
    const __half *act;  // activation (ReLU mask)
    __half *dact;       // [B][Hi][Wi][Ca]: gradient of the pre-activation
};

struct FlattenArgs {
    int B, F, n_a, n_l, n_coarse, row_stride;
    const __half *a3, *x;
    long in_stride, level_off;
    const float *rows;
    __half *f;
};

struct HeadArgs {
    int B, n_coarse, row_stride;
    const float *rows, *target, *d;
    float *out, *loss;      // out: rows of stride row_stride
    __half *dd;
    float grad_scale;
};

struct AdamArgs {
    size_t n;
    float *w, *m, *v;
    const float *grad;
    __half *wh;
    float lr, b1, b2, eps, c1, c2, inv_scale;
    const int *skip;
};

struct ConvArgs {
    int n;                          // beams
    const __half *x;                // [n][5440][2]
    const float *rows;              // [n][n_coarse + 4]
    int n_coarse, F;
    const __half *w1, *w2, *w3;     // conv weights [32][32], [32][320], [32][320] (parameter layout)
    const float *b1, *b2, *b3;
    __half *f;                      // [n][F]: fully connected input rows
};

// Per-beam scale of the network's input and output: the prior's mass, at
// least a tenth of the tail bound (0: no tail).
__host__ __device__ inline float net_scale(const float *row, int n_coarse)
{
    const float m = row[n_coarse + 3], e = row[n_coarse + 1];
    return m > 0.1f * e ? m : 0.1f * e;
}

// Forward GEMM on tcgen05 (lidar_umma.cu): C[m][n] = sum_k A[m][k] B[n][k]
// + bias[n] (ReLU if relu), written as FP16 (Ch) and/or FP32 (C), row
// stride ldc. N in 16..256 (multiple of 16), K and the leading dimensions
// multiples of 8, A and B 16-byte aligned. A bounded wait that gives up sets
// *err to 1 (err may be NULL).
struct UmmaArgs {
    int M, N, K;
    const __half *A;
    int lda;
    const __half *B;
    int ldb;
    const float *bias;
    int relu;
    __half *Ch;
    float *C;
    int ldc;
    int *err;
};

cudaError_t launch_gemm(bool ta, bool tb, const GemmArgs &g, int splits, cudaStream_t s);
bool umma_gemm_supported(const UmmaArgs &g);
cudaError_t launch_umma_gemm(const UmmaArgs &g, cudaStream_t s);
cudaError_t launch_im2col(const Im2colArgs &a, cudaStream_t s);
cudaError_t launch_col2im(const Col2imArgs &a, cudaStream_t s);
cudaError_t launch_flatten(const FlattenArgs &a, cudaStream_t s);
cudaError_t launch_head(const HeadArgs &a, cudaStream_t s);
cudaError_t launch_finish_rows(const float *rows, float *out, int B, int n_coarse, cudaStream_t s);
cudaError_t launch_relu_grad(const float *da, const __half *a, __half *dz, size_t n, float scale, cudaStream_t s);
cudaError_t launch_bias_grad(const __half *dz, int M, int N, float *db, cudaStream_t s);
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t s);
cudaError_t launch_finite_check(const float *g, size_t n, int *flag, cudaStream_t s);
cudaError_t launch_to_half(const float *w, __half *wh, size_t n, cudaStream_t s);
size_t conv_smem_bytes();
cudaError_t launch_conv(const ConvArgs &a, int grid, cudaStream_t s);

}  // namespace gbl
