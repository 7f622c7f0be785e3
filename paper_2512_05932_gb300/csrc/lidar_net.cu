// FP16 kernels of the tail network (training and inference): a tiled tensor-
// core GEMM (mma.sync m16n8k16, FP16 operands, FP32 accumulation) in three
// operand layouts, im2col / col2im for the 3x3 stride-2 convolutions, and the
// element-wise steps (bias, ReLU, loss, Adam).
//
// Network (per beam; x = the 4-level input pyramid, levels L0..L3 of
// 64^2, 32^2, 16^2, 8^2 cells x 2 channels):
//   a1 = relu(conv3x3/2(L0))                      32^2 x 32
//   a2 = relu(conv3x3/2([a1, L1]))                16^2 x 32
//   a3 = relu(conv3x3/2([a2, L2]))                 8^2 x 32
//   f  = [a3, L3, prior / s]                       2048 + 128 + n_coarse
//   h  = relu(W1 f + b1)                           256
//   y  = relu(prior / s + W2 h + b2)               n_coarse   (tail / s)
// with s the beam's scale (prior mass, at least 0.1 x the tail bound).
#include <cuda_fp16.h>
#include <stdint.h>

#include "lidar_net_internal.h"

namespace gbl {

// ---------------------------------------------------------------------------
// GEMM: C[m][n] = sum_k A(m, k) B(n, k)
//   A(m, k) = A[m * lda + k] (TA = false) or A[k * lda + m] (TA = true)
//   B(n, k) = B[n * ldb + k] (TB = false) or B[k * ldb + n] (TB = true)
// 64 x 64 x 32 tiles, 4 warps of 32 x 32; K a multiple of 8, leading
// dimensions multiples of 8 (16-byte rows). blockIdx.z splits K.
// ---------------------------------------------------------------------------

constexpr int kBM = 64, kBN = 64, kBK = 32, kSP = kBK + 8;  // smem row pitch (halves): conflict-free ldmatrix

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __half *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Loads a rows x 32 (k) tile of an operand into shared memory as [row][k].
template <bool T>
__device__ __forceinline__ void load_tile(__half *s, const __half *g, int ld, int r0, int nrows, int k0, int K)
{
    const int tid = threadIdx.x;
    if (!T) {
        // row-major: 4 chunks of 8 halves per row
        for (int i = tid; i < 64 * 4; i += 128) {
            const int r = i >> 2, kq = (i & 3) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r0 + r < nrows && k0 + kq < K) v = *reinterpret_cast<const uint4 *>(g + (size_t)(r0 + r) * ld + k0 + kq);
            *reinterpret_cast<uint4 *>(s + r * kSP + kq) = v;
        }
    } else {
        // k-major: 8 chunks of 8 rows per k
        for (int i = tid; i < 32 * 8; i += 128) {
            const int kk = i >> 3, rq = (i & 7) * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (k0 + kk < K) {
                if (r0 + rq + 8 <= nrows) {
                    v = *reinterpret_cast<const uint4 *>(g + (size_t)(k0 + kk) * ld + r0 + rq);
                } else {
                    __half tmp[8];
                    for (int j = 0; j < 8; ++j)
                        tmp[j] = (r0 + rq + j < nrows) ? g[(size_t)(k0 + kk) * ld + r0 + rq + j] : __float2half(0.f);
                    v = *reinterpret_cast<uint4 *>(tmp);
                }
            }
            const __half *h = reinterpret_cast<const __half *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) s[(rq + j) * kSP + kk] = h[j];
        }
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g)
{
    __shared__ __align__(16) __half sA[kBM * kSP];
    __shared__ __align__(16) __half sB[kBN * kSP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int kbeg = blockIdx.z * g.k_split;
    const int kend = min(g.K, kbeg + g.k_split);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
        __syncthreads();
        load_tile<TA>(sA, g.A, g.lda, m0, g.M, k0, kend);
        load_tile<TB>(sB, g.B, g.ldb, n0, g.N, k0, kend);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t a[2][4], b[2][4];
            const int q = lane >> 3, r = lane & 7;
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
                ldsm_x4(a[mi], sA + (wm * 32 + mi * 16 + (q & 1) * 8 + r) * kSP + kk + (q >> 1) * 8);
#pragma unroll
            for (int nj = 0; nj < 2; ++nj)
                ldsm_x4(b[nj], sB + (wn * 32 + nj * 16 + (q >> 1) * 8 + r) * kSP + kk + (q & 1) * 8);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_f16(acc[mi][ni], a[mi], b[ni >> 1][(ni & 1) * 2], b[ni >> 1][(ni & 1) * 2 + 1]);
        }
    }
    // epilogue
    const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 32 + mi * 16 + gq + 8 * h;
                const int n = n0 + wn * 32 + ni * 8 + 2 * t4;
                if (m >= g.M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (n + e >= g.N) continue;
                    float v = acc[mi][ni][2 * h + e];
                    if (g.mode == kGemmStore) {
                        g.C[(size_t)m * g.ldc + n + e] = v;
                    } else if (g.mode == kGemmAtomic) {
                        atomicAdd(g.C + (size_t)m * g.ldc + n + e, v);
                    } else {
                        v += g.bias[n + e];
                        if (g.mode == kGemmBiasRelu) v = fmaxf(v, 0.f);
                        if (g.Ch) g.Ch[(size_t)m * g.ldc + n + e] = __float2half_rn(v);
                        if (g.C && g.mode == kGemmBias) g.C[(size_t)m * g.ldc + n + e] = v;
                    }
                }
            }
}

cudaError_t launch_gemm(bool ta, bool tb, const GemmArgs &g, int splits, cudaStream_t s)
{
    dim3 grid((g.M + kBM - 1) / kBM, (g.N + kBN - 1) / kBN, splits);
    if (!ta && !tb) gemm_kernel<false, false><<<grid, 128, 0, s>>>(g);
    else if (!ta && tb) gemm_kernel<false, true><<<grid, 128, 0, s>>>(g);
    else if (ta && !tb) gemm_kernel<true, false><<<grid, 128, 0, s>>>(g);
    else gemm_kernel<true, true><<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// convolution plumbing
// ---------------------------------------------------------------------------

// im2col of a 3x3 stride-2 convolution with one pixel of zero padding:
// row (b, oy, ox) of Xc ([B * Ho * Wo][Kp]), column k = tap * Cin + c
// (tap = ky * 3 + kx), input pixel (2 oy + ky - 1, 2 ox + kx - 1); channels
// c < Ca from act ([B][Hi][Wi][Ca]), the next 2 from the pyramid level
// (x + level_off cells, [B][Hi][Wi][2] within each beam's input of
// in_stride cells); columns k >= 9 Cin are zero.
__global__ void im2col_kernel(Im2colArgs a)
{
    const int Cin = a.Ca + 2;
    const size_t total = (size_t)a.B * a.Ho * a.Wo * a.Kp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % a.Kp);
        const size_t row = i / a.Kp;
        const int ox = (int)(row % a.Wo), oy = (int)((row / a.Wo) % a.Ho);
        const int b = (int)(row / ((size_t)a.Wo * a.Ho));
        __half v = __float2half(0.f);
        if (k < 9 * Cin) {
            const int tap = k / Cin, c = k - tap * Cin;
            const int iy = 2 * oy + tap / 3 - 1, ix = 2 * ox + tap % 3 - 1;
            if (iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi) {
                if (c < a.Ca) v = a.act[(((size_t)b * a.Hi + iy) * a.Wi + ix) * a.Ca + c];
                else v = a.x[(size_t)b * a.in_stride + a.level_off + ((size_t)iy * a.Wi + ix) * 2 + (c - a.Ca)];
            }
        }
        a.out[i] = v;
    }
}

// Gradient of im2col for the activation channels: dA[b][iy][ix][c] = sum over
// the (<= 4) output pixels and taps that read (iy, ix) of dXc, times the ReLU
// mask of the activation (a > 0), scaled; written as FP16.
__global__ void col2im_kernel(Col2imArgs a)
{
    const int Cin = a.Ca + 2;
    const size_t total = (size_t)a.B * a.Hi * a.Wi * a.Ca;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % a.Ca);
        const size_t pix = i / a.Ca;
        const int ix = (int)(pix % a.Wi), iy = (int)((pix / a.Wi) % a.Hi);
        const int b = (int)(pix / ((size_t)a.Wi * a.Hi));
        float s = 0.f;
        if (__half2float(a.act[i]) > 0.f) {
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int ty = iy + 1 - ky;
                if (ty < 0 || (ty & 1) || (ty >> 1) >= a.Ho) continue;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int tx = ix + 1 - kx;
                    if (tx < 0 || (tx & 1) || (tx >> 1) >= a.Wo) continue;
                    const size_t row = ((size_t)b * a.Ho + (ty >> 1)) * a.Wo + (tx >> 1);
                    s += a.dcol[row * a.Kp + (ky * 3 + kx) * Cin + c];
                }
            }
        }
        a.dact[i] = __float2half_rn(s);
    }
}

// f = [a3 (n_a), level 3 of x (n_l), prior / s (n_coarse)] per beam, and the
// per-beam scale s.
__global__ void flatten_kernel(FlattenArgs a)
{
    const size_t total = (size_t)a.B * a.F;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % a.F);
        const int b = (int)(i / a.F);
        __half v;
        if (j < a.n_a) {
            v = a.a3[(size_t)b * a.n_a + j];
        } else if (j < a.n_a + a.n_l) {
            v = a.x[(size_t)b * a.in_stride + a.level_off + (j - a.n_a)];
        } else {
            const int c = j - a.n_a - a.n_l;
            const float *row = a.rows + (size_t)b * a.row_stride;
            const float s = net_scale(row, a.n_coarse);
            v = __float2half_rn(s > 0.f ? row[c] / s : 0.f);
        }
        a.f[i] = v;
    }
}

// Output, loss and the output gradient:
//   y_hat = relu(prior / s + d), loss = mean_b sum_c |y_hat - target / s|,
//   dd = d loss / d d x loss_scale (FP16)
__global__ void head_kernel(HeadArgs a)
{
    const size_t total = (size_t)a.B * a.n_coarse;
    float part = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % a.n_coarse);
        const int b = (int)(i / a.n_coarse);
        const float *row = a.rows + (size_t)b * a.row_stride;
        const float s = net_scale(row, a.n_coarse);
        const float pn = s > 0.f ? row[c] / s : 0.f;
        const float z = pn + a.d[i];
        const float yh = fmaxf(z, 0.f);
        if (a.out) a.out[(size_t)b * a.row_stride + c] = yh * s;
        if (a.target) {
            const float y = s > 0.f ? a.target[(size_t)b * a.row_stride + c] / s : 0.f;
            const float e = yh - y;
            part += s > 0.f ? fabsf(e) : 0.f;
            const float g = (s > 0.f && z > 0.f) ? (e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f)) : 0.f;
            a.dd[i] = __float2half_rn(g * a.grad_scale);
        }
    }
    if (a.loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(a.loss, part / (float)a.B);
    }
}

// Final rows of a prediction: clip the tail to the bound and copy the
// ambient entry and the bounds.
__global__ void finish_rows_kernel(const float *rows, float *out, int B, int n_coarse)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const float *r = rows + (size_t)b * (n_coarse + 4);
    float *o = out + (size_t)b * (n_coarse + 4);
    float s = 0.f;
    for (int c = lane; c < n_coarse; c += 32) s += fmaxf(o[c], 0.f);
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
    const float E = r[n_coarse + 1];
    const float f = (s > E && s > 0.f) ? E / s * (1.f - 1e-6f) : 1.f;
    for (int c = lane; c < n_coarse; c += 32) o[c] = fmaxf(o[c], 0.f) * f;
    if (lane == 0) {
        o[n_coarse] = r[n_coarse];
        o[n_coarse + 1] = E;
        o[n_coarse + 2] = r[n_coarse + 2];
        o[n_coarse + 3] = s * f;
    }
}

// dZ = dA * (a > 0) for a row-major activation (FP16 in, FP16 out), used
// between the fully connected layers.
__global__ void relu_grad_kernel(const float *da, const __half *a, __half *dz, size_t n, float scale)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dz[i] = __float2half_rn(__half2float(a[i]) > 0.f ? da[i] * scale : 0.f);
}

// db[n] += sum_m dz[m][n] (FP32 atomics, one thread per (m-chunk, n))
__global__ void bias_grad_kernel(const __half *dz, int M, int N, float *db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int chunk = (M + gridDim.y - 1) / gridDim.y;
    const int m0 = blockIdx.y * chunk, m1 = min(M, m0 + chunk);
    float s = 0.f;
    for (int m = m0; m < m1; ++m) s += __half2float(dz[(size_t)m * N + n]);
    atomicAdd(db + n, s);
}

// Adam with bias correction; grads are divided by the loss scale; writes the
// FP16 copy of the weights. A non-finite gradient skips the step (flag set).
__global__ void adam_kernel(AdamArgs a)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x) {
        if (*a.skip) return;
        const float g = a.grad[i] * a.inv_scale;
        const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
        const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
        a.m[i] = m;
        a.v[i] = v;
        const float w = a.w[i] - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
        a.w[i] = w;
        a.wh[i] = __float2half_rn(w);
    }
}

__global__ void finite_check_kernel(const float *g, size_t n, int *flag)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(g[i])) *flag = 1;
}

__global__ void to_half_kernel(const float *w, __half *wh, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wh[i] = __float2half_rn(w[i]);
}

namespace {
int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 32); }
}  // namespace

cudaError_t launch_im2col(const Im2colArgs &a, cudaStream_t s)
{
    im2col_kernel<<<grid_for((size_t)a.B * a.Ho * a.Wo * a.Kp), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_col2im(const Col2imArgs &a, cudaStream_t s)
{
    col2im_kernel<<<grid_for((size_t)a.B * a.Hi * a.Wi * a.Ca), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_flatten(const FlattenArgs &a, cudaStream_t s)
{
    flatten_kernel<<<grid_for((size_t)a.B * a.F), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_head(const HeadArgs &a, cudaStream_t s)
{
    head_kernel<<<grid_for((size_t)a.B * a.n_coarse), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_finish_rows(const float *rows, float *out, int B, int n_coarse, cudaStream_t s)
{
    finish_rows_kernel<<<(B + 7) / 8, 256, 0, s>>>(rows, out, B, n_coarse);
    return cudaGetLastError();
}
cudaError_t launch_relu_grad(const float *da, const __half *a, __half *dz, size_t n, float scale, cudaStream_t s)
{
    relu_grad_kernel<<<grid_for(n), 256, 0, s>>>(da, a, dz, n, scale);
    return cudaGetLastError();
}
cudaError_t launch_bias_grad(const __half *dz, int M, int N, float *db, cudaStream_t s)
{
    dim3 grid((N + 127) / 128, std::min(256, std::max(1, M / 256)));
    bias_grad_kernel<<<grid, 128, 0, s>>>(dz, M, N, db);
    return cudaGetLastError();
}
cudaError_t launch_adam(const AdamArgs &a, cudaStream_t s)
{
    adam_kernel<<<grid_for(a.n), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_finite_check(const float *g, size_t n, int *flag, cudaStream_t s)
{
    finite_check_kernel<<<grid_for(n), 256, 0, s>>>(g, n, flag);
    return cudaGetLastError();
}
cudaError_t launch_to_half(const float *w, __half *wh, size_t n, cudaStream_t s)
{
    to_half_kernel<<<grid_for(n), 256, 0, s>>>(w, wh, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused inference of the three convolutions (persistent; one beam at a time
// per CTA, 8 warps). Shared memory holds the FP16 conv weights (re-laid out
// so that every 16-column k-step is aligned), the beam's input pyramid
// (double-buffered with cp.async, levels 0-2 in zero-bordered planes so that
// window reads need no bounds tests) and the activations: a1 and a2 split by
// pixel parity into four sub-images with an 80-byte pixel pitch, so that the
// stride-2 window rows of the next layer are contiguous and ldmatrix reads
// them without bank conflicts. Every warp keeps its output tiles for the whole
// launch, so the shared-memory addresses of its A fragments are computed once.
// Writes the fully connected layer's input row f = [a3, L3, prior / s].
// ---------------------------------------------------------------------------

namespace {

constexpr int kCP = 40;                        // activation pixel pitch (halves)
constexpr int kW1P = 40, kW23P = 328;           // weight row pitches (halves)
constexpr int kInHalves = 2 * 5440;             // one beam's input
constexpr int kL1Off = 2 * 4096, kL2Off = kL1Off + 2 * 1024, kL3Off = kL2Off + 2 * 256;
// zero-bordered input planes: S + 2 rows of S + 8 pixels (4 left, 4 right), 2 halves per pixel
constexpr int kP0W = 72, kP1W = 40, kP2W = 24;
constexpr int kP0 = 66 * kP0W * 2, kP1 = 34 * kP1W * 2, kP2 = 18 * kP2W * 2, kP3 = 128;
constexpr int kXB = kP0 + kP1 + kP2 + kP3;     // halves per input buffer

struct ConvSmem {
    __half w1[32 * kW1P];
    __half w2[32 * kW23P];
    __half w3[32 * kW23P];
    float bias[96];
    __half x[2][kXB];
    __half a1[4 * 256 * kCP];
    __half a2[4 * 64 * kCP];
    __half a3[64 * 32];
    __half zero[48];
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4_addr(uint32_t (&r)[4], uint32_t a)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ uint32_t lds32(const __half *p) { return *reinterpret_cast<const uint32_t *>(p); }

// Halves offset of tap (ky, kx) = (tap / 3, tap % 3) in a zero-bordered plane of width W.
__device__ __forceinline__ int tap_off(int tap, int W) { return 2 * ((tap / 3) * W + tap % 3); }

// A fragment of the 2-channel pyramid part of K (column tap * 2 + c; taps
// 0..7 in chunk 0, tap 8 in chunk 1) for rows at plane offsets r0 and r1 (the
// window origin of each row's output pixel); t = lane % 4.
template <int W>
__device__ __forceinline__ void pyr_frag2(uint32_t (&a)[4], const __half *pl, int r0, int r1, int chunk, int t)
{
    if (chunk == 0) {
        const int o0 = tap_off(t, W), o1 = tap_off(t + 4, W);
        a[0] = lds32(pl + r0 + o0); a[1] = lds32(pl + r1 + o0);
        a[2] = lds32(pl + r0 + o1); a[3] = lds32(pl + r1 + o1);
    } else {
        const int o8 = tap_off(8, W);
        a[0] = t == 0 ? lds32(pl + r0 + o8) : 0u;
        a[1] = t == 0 ? lds32(pl + r1 + o8) : 0u;
        a[2] = 0u; a[3] = 0u;
    }
}

// Window origin (halves) of output pixel (oy, ox) in a zero-bordered plane of
// width W: input pixel (2 oy - 1, 2 ox - 1) at padded row 2 oy, column 2 ox + 3.
template <int W>
__device__ __forceinline__ int win_origin(int oy, int ox) { return 2 * ((2 * oy) * W + 2 * ox + 3); }

// Stores bias + ReLU of a 16 x 32 accumulator tile (rows g, g + 8) as FP16
// pairs at dst(row) + channel.
template <typename Dst>
__device__ __forceinline__ void store_relu(const float (&acc)[4][4], const float *bias, int g, int t, Dst dst)
{
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = ni * 8 + 2 * t;
            const float v0 = fmaxf(acc[ni][2 * h] + bias[c], 0.f), v1 = fmaxf(acc[ni][2 * h + 1] + bias[c + 1], 0.f);
            *reinterpret_cast<__half2 *>(dst(g + 8 * h) + c) = __floats2half2_rn(v0, v1);
        }
}

}  // namespace

__global__ void __launch_bounds__(256, 1) tailnet_conv_kernel(ConvArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ConvSmem &S = *reinterpret_cast<ConvSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3, q = lane >> 3, r8 = lane & 7;

    // weights: conv1 as is (columns 0..31); conv2 / conv3 reordered to
    // column tap * 32 + c for the 32 activation channels, then 288 + tap * 2 + c
    for (int i = tid; i < 32 * 32; i += 256) S.w1[(i >> 5) * kW1P + (i & 31)] = A.w1[i];
    for (int i = tid; i < 32 * 320; i += 256) {
        const int n = i / 320, k = i - n * 320;
        int src;
        if (k < 288) src = (k >> 5) * 34 + (k & 31);
        else if (k < 306) src = ((k - 288) >> 1) * 34 + 32 + ((k - 288) & 1);
        else src = -1;
        S.w2[n * kW23P + k] = src >= 0 ? A.w2[n * 320 + src] : __float2half(0.f);
        S.w3[n * kW23P + k] = src >= 0 ? A.w3[n * 320 + src] : __float2half(0.f);
    }
    for (int i = tid; i < 96; i += 256) S.bias[i] = i < 32 ? A.b1[i] : (i < 64 ? A.b2[i - 32] : A.b3[i - 64]);
    if (tid < 48) S.zero[tid] = __float2half(0.f);
    // zero borders of both input buffers (cp.async writes the interiors only)
    for (int i = tid; i < 2 * kXB / 8; i += 256) reinterpret_cast<uint4 *>(S.x)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    auto prefetch = [&](int b, int buf) {
        const __half *src = A.x + (size_t)b * kInHalves;
        __half *X = S.x[buf];
        // L0: 64 rows of 256 bytes; L1: 32 rows of 128; L2: 16 rows of 64; L3: 256 bytes
        for (int i = tid; i < 64 * 16 + 32 * 8 + 16 * 4 + 16; i += 256) {
            const __half *s;
            __half *d;
            if (i < 1024) {
                const int r = i >> 4, c = i & 15;
                s = src + r * 128 + c * 8;
                d = X + ((r + 1) * kP0W + 4) * 2 + c * 8;
            } else if (i < 1024 + 256) {
                const int j = i - 1024, r = j >> 3, c = j & 7;
                s = src + kL1Off + r * 64 + c * 8;
                d = X + kP0 + ((r + 1) * kP1W + 4) * 2 + c * 8;
            } else if (i < 1024 + 256 + 64) {
                const int j = i - 1280, r = j >> 2, c = j & 3;
                s = src + kL2Off + r * 32 + c * 8;
                d = X + kP0 + kP1 + ((r + 1) * kP2W + 4) * 2 + c * 8;
            } else {
                const int j = i - 1344;
                s = src + kL3Off + j * 8;
                d = X + kP0 + kP1 + kP2 + j * 8;
            }
            cp_async16(d, s);
        }
        cp_async_commit();
    };

    // per-warp A-fragment addresses of the activation part of conv2 (output
    // rows oy = warp, warp + 8) and conv3 (rows 2 (warp / 2), + 1), one per
    // tap: the window row of this lane's ldmatrix row, or the zero row
    uint32_t ad2[2][9], ad3[9];
    {
        const uint32_t zero = (uint32_t)__cvta_generic_to_shared(S.zero);
        const uint32_t a1s = (uint32_t)__cvta_generic_to_shared(S.a1), a2s = (uint32_t)__cvta_generic_to_shared(S.a2);
        const int koff = (q >> 1) * 8;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3, sub = ((ky + 1) & 1) * 2 + ((kx + 1) & 1);
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int oy = warp + 8 * mi, ox = (q & 1) * 8 + r8;
                const int sy = ky == 0 ? oy - 1 : oy, sx = kx == 0 ? ox - 1 : ox;
                ad2[mi][tap] = (sy < 0 || sx < 0) ? zero : a1s + 2u * (uint32_t)((sub * 256 + sy * 16 + sx) * kCP + koff);
            }
            const int oy = 2 * (warp >> 1) + (q & 1), ox = r8;
            const int sy = ky == 0 ? oy - 1 : oy, sx = kx == 0 ? ox - 1 : ox;
            ad3[tap] = (sy < 0 || sx < 0) ? zero : a2s + 2u * (uint32_t)((sub * 64 + sy * 8 + sx) * kCP + koff);
        }
    }
    const uint32_t w2s = (uint32_t)__cvta_generic_to_shared(S.w2), w3s = (uint32_t)__cvta_generic_to_shared(S.w3);
    const uint32_t bw2 = w2s + 2u * (uint32_t)(((q >> 1) * 8 + r8) * kW23P + (q & 1) * 8);
    const uint32_t bw3 = w3s + 2u * (uint32_t)((((warp & 1) * 16) + (q >> 1) * 8 + r8) * kW23P + (q & 1) * 8);

    int buf = 0;
    if ((int)blockIdx.x < A.n) prefetch(blockIdx.x, 0);

    for (int b = blockIdx.x; b < A.n; b += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        if (b + (int)gridDim.x < A.n) prefetch(b + gridDim.x, buf ^ 1);
        const __half *X = S.x[buf];

        // ---- conv1: 64^2 x 2 -> 32^2 x 32; warp w takes m-tiles w, w + 8, ...
        {
            uint32_t bw[2][2][4];  // [k-step][n-pair]
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                for (int nj = 0; nj < 2; ++nj)
                    ldsm_x4(bw[ks][nj], S.w1 + (nj * 16 + (q >> 1) * 8 + r8) * kW1P + ks * 16 + (q & 1) * 8);
#pragma unroll 2
            for (int mt = warp; mt < 64; mt += 8) {
                const int oy = mt >> 1, ox0 = (mt & 1) * 16;
                const int r0 = win_origin<kP0W>(oy, ox0 + g), r1 = r0 + 32;  // ox + 8 -> 16 pixels right
                float acc[4][4] = {};
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    uint32_t a[4];
                    pyr_frag2<kP0W>(a, X, r0, r1, ks, t);
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni)
                        mma_f16(acc[ni], a, bw[ks][ni >> 1][(ni & 1) * 2], bw[ks][ni >> 1][(ni & 1) * 2 + 1]);
                }
                store_relu(acc, S.bias, g, t, [&](int row) {
                    const int ox = ox0 + row;
                    return S.a1 + (((oy & 1) * 2 + (ox & 1)) * 256 + (oy >> 1) * 16 + (ox >> 1)) * kCP;
                });
            }
        }
        __syncthreads();

        // ---- conv2: [a1, L1] -> 16^2 x 32; warp w takes output rows w, w + 8
        {
            float acc[2][4][4] = {};
            const __half *L1 = X + kP0;
#pragma unroll
            for (int ks = 0; ks < 20; ++ks) {
                uint32_t bw[2][4];
                ldsm_x4_addr(bw[0], bw2 + 2u * (uint32_t)(ks * 16));
                ldsm_x4_addr(bw[1], bw2 + 2u * (uint32_t)(16 * kW23P + ks * 16));
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    uint32_t a[4];
                    if (ks < 18) {
                        ldsm_x4_addr(a, ad2[mi][ks >> 1] + 2u * (uint32_t)((ks & 1) * 16));
                    } else {
                        const int oy = warp + 8 * mi;
                        const int r0 = win_origin<kP1W>(oy, g);
                        pyr_frag2<kP1W>(a, L1, r0, r0 + 32, ks - 18, t);
                    }
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni)
                        mma_f16(acc[mi][ni], a, bw[ni >> 1][(ni & 1) * 2], bw[ni >> 1][(ni & 1) * 2 + 1]);
                }
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int oy = warp + 8 * mi;
                store_relu(acc[mi], S.bias + 32, g, t, [&](int ox) {
                    return S.a2 + (((oy & 1) * 2 + (ox & 1)) * 64 + (oy >> 1) * 8 + (ox >> 1)) * kCP;
                });
            }
        }
        __syncthreads();

        // ---- conv3: [a2, L2] -> 8^2 x 32; warp w: m-tile w / 2 (output rows
        // 2 mt, 2 mt + 1), n-tiles 2 (w % 2) .. + 1
        {
            const int mt = warp >> 1, nh = warp & 1;
            const __half *L2 = X + kP0 + kP1;
            float acc[2][4] = {};
#pragma unroll
            for (int ks = 0; ks < 20; ++ks) {
                uint32_t bw[4];
                ldsm_x4_addr(bw, bw3 + 2u * (uint32_t)(ks * 16));
                uint32_t a[4];
                if (ks < 18) {
                    ldsm_x4_addr(a, ad3[ks >> 1] + 2u * (uint32_t)((ks & 1) * 16));
                } else {
                    const int r0 = win_origin<kP2W>(2 * mt, g), r1 = win_origin<kP2W>(2 * mt + 1, g);
                    pyr_frag2<kP2W>(a, L2, r0, r1, ks - 18, t);
                }
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) mma_f16(acc[ni], a, bw[(ni & 1) * 2], bw[(ni & 1) * 2 + 1]);
            }
#pragma unroll
            for (int ni = 0; ni < 2; ++ni)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = nh * 16 + ni * 8 + 2 * t;
                    const int pix = (2 * mt + h) * 8 + g;  // row g (+8) of the tile = (oy, ox = g)
                    const float v0 = fmaxf(acc[ni][2 * h] + S.bias[64 + c], 0.f);
                    const float v1 = fmaxf(acc[ni][2 * h + 1] + S.bias[64 + c + 1], 0.f);
                    *reinterpret_cast<__half2 *>(S.a3 + pix * 32 + c) = __floats2half2_rn(v0, v1);
                }
        }
        __syncthreads();

        // ---- f = [a3, L3, prior / s]
        {
            __half *f = A.f + (size_t)b * A.F;
            for (int i = tid; i < 2048 / 8; i += 256)
                reinterpret_cast<uint4 *>(f)[i] = reinterpret_cast<const uint4 *>(S.a3)[i];
            for (int i = tid; i < 128 / 8; i += 256)
                reinterpret_cast<uint4 *>(f + 2048)[i] = reinterpret_cast<const uint4 *>(X + kP0 + kP1 + kP2)[i];
            const float *row = A.rows + (size_t)b * (A.n_coarse + 4);
            const float sc = net_scale(row, A.n_coarse);
            for (int c = tid; c < A.n_coarse; c += 256) f[2176 + c] = __float2half_rn(sc > 0.f ? row[c] / sc : 0.f);
        }
        buf ^= 1;
    }
    cp_async_wait_all();
}

size_t conv_smem_bytes() { return sizeof(ConvSmem); }

cudaError_t launch_conv(const ConvArgs &a, int grid, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(tailnet_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(ConvSmem));
    if (e != cudaSuccess) return e;
    tailnet_conv_kernel<<<grid, 256, sizeof(ConvSmem), s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbl
