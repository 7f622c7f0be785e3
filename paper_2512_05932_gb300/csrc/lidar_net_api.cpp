// Host side of the tail network (include/lidar_tail.h): parameters, Adam
// state, scratch, the training step (forward, L1 loss, backward, Adam) and
// batched prediction, all as launches of the kernels in lidar_net.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lidar_net_internal.h"
#include "lidar_tail.h"

namespace {

constexpr int kC = 32;          // conv channels
constexpr int kHid = 256;       // hidden units
constexpr int kK1 = 32;         // conv1 im2col width (9 taps x 2 channels, padded)
constexpr int kK2 = 320;        // conv2/3 im2col width (9 taps x 34 channels, padded)
constexpr int kNA = 64 * kC;    // flattened a3
constexpr int kNL = 8 * 8 * 2;  // flattened pyramid level 3
constexpr long kIn = 2L * LIDAR_TAIL_INPUT_CELLS;  // input halves per beam
constexpr long kOffL1 = 2L * 64 * 64, kOffL2 = kOffL1 + 2L * 32 * 32, kOffL3 = kOffL2 + 2L * 16 * 16;
constexpr float kLossScale = 1024.f;
constexpr uint32_t kMagic = 0x314E544Cu;  // "LTN1"

thread_local char g_net_err[512] = "no error";

}  // namespace

struct lidar_tailnet {
    int nc = 0, F = 0;
    // parameter tensors: offsets (floats) into w
    size_t o_w1, o_b1, o_w2, o_b2, o_w3, o_b3, o_f1, o_fb1, o_f2, o_fb2, n_par;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __half *wh = nullptr;
    int *flag = nullptr;
    float *loss = nullptr;
    int *uerr = nullptr;          // error word of the tcgen05 GEMM (bounded waits)
    int dense_mode = LIDAR_DENSE_TCGEN05;
    int64_t step = 0;
    // scratch for `cap` beams
    int cap = 0;
    __half *X1 = nullptr, *A1 = nullptr, *X2 = nullptr, *A2 = nullptr, *X3 = nullptr, *A3 = nullptr, *Fm = nullptr,
           *H = nullptr, *dD = nullptr, *dZh = nullptr, *dZ3 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *D = nullptr, *dH = nullptr, *dA3 = nullptr, *dX = nullptr;
    // prediction scratch for `pcap` beams (fused convolutions)
    int pcap = 0;
    __half *pF = nullptr, *pH = nullptr;
    float *pD = nullptr;
    int sms = 0;
    // per-stage timing of predict (lidar_tailnet_profile_enable): events around
    // the fused convolutions and the dense layers of each chunk
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    char err[512] = "no error";
};

namespace {

lidar_status_t nfail(lidar_tailnet_t *n, lidar_status_t st, const char *fmt, ...)
{
    char *buf = n ? n->err : g_net_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

lidar_status_t ncuda(lidar_tailnet_t *n, cudaError_t e, const char *what)
{
    return nfail(n, e == cudaErrorMemoryAllocation ? LIDAR_ENOMEM : LIDAR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaEvent_t next_event(lidar_tailnet_t *n)
{
    if (!n->prof) return nullptr;
    if (n->ev_used == n->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        n->ev.push_back(e);
    }
    return n->ev[n->ev_used++];
}

void free_events(lidar_tailnet_t *n)
{
    for (cudaEvent_t e : n->ev) cudaEventDestroy(e);
    n->ev.clear();
    n->ev_used = 0;
}

void free_pred(lidar_tailnet_t *n)
{
    cudaFree(n->pF); cudaFree(n->pH); cudaFree(n->pD);
    n->pF = nullptr; n->pH = nullptr; n->pD = nullptr;
    n->pcap = 0;
}

lidar_status_t ensure_pred(lidar_tailnet_t *n, int B)
{
    if (B <= n->pcap) return LIDAR_OK;
    free_pred(n);
    cudaError_t e;
    if ((e = cudaMalloc(&n->pF, (size_t)B * n->F * sizeof(__half))) != cudaSuccess ||
        (e = cudaMalloc(&n->pH, (size_t)B * 256 * sizeof(__half))) != cudaSuccess ||
        (e = cudaMalloc(&n->pD, (size_t)B * n->nc * sizeof(float))) != cudaSuccess)
        return ncuda(n, e, "cudaMalloc(prediction scratch)");
    n->pcap = B;
    return LIDAR_OK;
}

void free_scratch(lidar_tailnet_t *n)
{
    void *p[] = {n->X1, n->A1, n->X2, n->A2, n->X3, n->A3, n->Fm, n->H, n->dD, n->dZh, n->dZ3, n->dZ2, n->dZ1,
                 n->D, n->dH, n->dA3, n->dX};
    for (void *q : p) cudaFree(q);
    n->X1 = n->A1 = n->X2 = n->A2 = n->X3 = n->A3 = n->Fm = n->H = n->dD = n->dZh = n->dZ3 = n->dZ2 = n->dZ1 = nullptr;
    n->D = n->dH = n->dA3 = n->dX = nullptr;
    n->cap = 0;
}

template <typename T>
cudaError_t alloc(T **p, size_t count)
{
    return cudaMalloc(p, count * sizeof(T));
}

lidar_status_t ensure_scratch(lidar_tailnet_t *n, int B, bool train)
{
    if (B <= n->cap && (!train || n->dD)) return LIDAR_OK;
    free_scratch(n);
    const size_t b = (size_t)B;
    cudaError_t e;
    if ((e = alloc(&n->X1, b * 1024 * kK1)) != cudaSuccess || (e = alloc(&n->A1, b * 1024 * kC)) != cudaSuccess ||
        (e = alloc(&n->X2, b * 256 * kK2)) != cudaSuccess || (e = alloc(&n->A2, b * 256 * kC)) != cudaSuccess ||
        (e = alloc(&n->X3, b * 64 * kK2)) != cudaSuccess || (e = alloc(&n->A3, b * 64 * kC)) != cudaSuccess ||
        (e = alloc(&n->Fm, b * n->F)) != cudaSuccess || (e = alloc(&n->H, b * kHid)) != cudaSuccess ||
        (e = alloc(&n->D, b * n->nc)) != cudaSuccess)
        return ncuda(n, e, "cudaMalloc(network scratch)");
    if (train) {
        if ((e = alloc(&n->dD, b * n->nc)) != cudaSuccess || (e = alloc(&n->dZh, b * kHid)) != cudaSuccess ||
            (e = alloc(&n->dZ3, b * 64 * kC)) != cudaSuccess || (e = alloc(&n->dZ2, b * 256 * kC)) != cudaSuccess ||
            (e = alloc(&n->dZ1, b * 1024 * kC)) != cudaSuccess || (e = alloc(&n->dH, b * kHid)) != cudaSuccess ||
            (e = alloc(&n->dA3, b * kNA)) != cudaSuccess || (e = alloc(&n->dX, b * 256 * kK2)) != cudaSuccess)
            return ncuda(n, e, "cudaMalloc(network gradient scratch)");
    }
    n->cap = B;
    return LIDAR_OK;
}

#define NCK(call, what)                                       \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ncuda(n, e_, what);     \
    } while (0)

gbl::GemmArgs gemm(int M, int N, int K, const __half *A, int lda, const __half *B, int ldb, int mode, float *C,
                   __half *Ch, int ldc, const float *bias)
{
    gbl::GemmArgs g{};
    g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
    g.k_split = ((K + 31) / 32) * 32;
    g.mode = mode; g.C = C; g.Ch = Ch; g.ldc = ldc; g.bias = bias;
    return g;
}

// Forward GEMM with bias (+ ReLU), non-transposed operands: the tcgen05
// kernel when the network uses it and the shape allows (N a multiple of 16 up
// to 256), else the mma.sync kernel.
cudaError_t dense(lidar_tailnet_t *n, const gbl::GemmArgs &g, cudaStream_t s)
{
    if (n->dense_mode == LIDAR_DENSE_TCGEN05) {
        gbl::UmmaArgs u{g.M, g.N, g.K, g.A, g.lda, g.B, g.ldb, g.bias, g.mode == gbl::kGemmBiasRelu ? 1 : 0,
                        g.Ch, g.mode == gbl::kGemmBias ? g.C : nullptr, g.ldc, n->uerr};
        if (gbl::umma_gemm_supported(u)) return gbl::launch_umma_gemm(u, s);
    }
    return gbl::launch_gemm(false, false, g, 1, s);
}

// Weight-gradient GEMM (reduction over the batch rows) split over K with FP32 atomics.
cudaError_t gemm_splitk(bool ta, bool tb, gbl::GemmArgs g, cudaStream_t s)
{
    const long tiles = (long)((g.M + 63) / 64) * ((g.N + 63) / 64);
    int splits = (int)std::max<long>(1, std::min<long>(1024, 4 * 152 / std::max<long>(1, tiles)));
    long per = (g.K + splits - 1) / splits;
    per = ((per + 31) / 32) * 32;
    splits = (int)((g.K + per - 1) / per);
    g.k_split = (int)per;
    g.mode = gbl::kGemmAtomic;
    return gbl::launch_gemm(ta, tb, g, splits, s);
}

// Forward pass of B beams (x: inputs, rows: feature rows) up to D (FP32
// pre-activation of the output layer).
lidar_status_t forward(lidar_tailnet_t *n, const __half *x, const float *rows, int B, cudaStream_t s)
{
    const __half *wh = n->wh;
    const float *w = n->w;
    gbl::Im2colArgs ia{};
    // conv1: 64^2 x 2 -> 32^2 x 32
    ia = gbl::Im2colArgs{B, 64, 64, 32, 32, 0, kK1, nullptr, x, kIn, 0, n->X1};
    NCK(gbl::launch_im2col(ia, s), "im2col");
    NCK(dense(n,
                         gemm(B * 1024, kC, kK1, n->X1, kK1, wh + n->o_w1, kK1, gbl::kGemmBiasRelu, nullptr, n->A1, kC,
                              w + n->o_b1), s), "conv1");
    // conv2: [a1, L1] 32^2 x 34 -> 16^2 x 32
    ia = gbl::Im2colArgs{B, 32, 32, 16, 16, kC, kK2, n->A1, x, kIn, kOffL1, n->X2};
    NCK(gbl::launch_im2col(ia, s), "im2col");
    NCK(dense(n,
                         gemm(B * 256, kC, kK2, n->X2, kK2, wh + n->o_w2, kK2, gbl::kGemmBiasRelu, nullptr, n->A2, kC,
                              w + n->o_b2), s), "conv2");
    // conv3: [a2, L2] 16^2 x 34 -> 8^2 x 32
    ia = gbl::Im2colArgs{B, 16, 16, 8, 8, kC, kK2, n->A2, x, kIn, kOffL2, n->X3};
    NCK(gbl::launch_im2col(ia, s), "im2col");
    NCK(dense(n,
                         gemm(B * 64, kC, kK2, n->X3, kK2, wh + n->o_w3, kK2, gbl::kGemmBiasRelu, nullptr, n->A3, kC,
                              w + n->o_b3), s), "conv3");
    // f = [a3, L3, prior / s]; h = relu(W1 f + b1); d = W2 h + b2
    gbl::FlattenArgs fa{B, n->F, kNA, kNL, n->nc, n->nc + 4, n->A3, x, kIn, kOffL3, rows, n->Fm};
    NCK(gbl::launch_flatten(fa, s), "flatten");
    NCK(dense(n,
                         gemm(B, kHid, n->F, n->Fm, n->F, wh + n->o_f1, n->F, gbl::kGemmBiasRelu, nullptr, n->H, kHid,
                              w + n->o_fb1), s), "fc1");
    NCK(dense(n,
                         gemm(B, n->nc, kHid, n->H, kHid, wh + n->o_f2, kHid, gbl::kGemmBias, n->D, nullptr, n->nc,
                              w + n->o_fb2), s), "fc2");
    return LIDAR_OK;
}

// Backward pass from dD (set by the head kernel); accumulates into n->g.
lidar_status_t backward(lidar_tailnet_t *n, const __half *x, int B, cudaStream_t s)
{
    (void)x;
    const __half *wh = n->wh;
    float *g = n->g;
    // fc2
    NCK(gemm_splitk(true, true, gemm(n->nc, kHid, B, n->dD, n->nc, n->H, kHid, 0, g + n->o_f2, nullptr, kHid, nullptr), s),
        "dW fc2");
    NCK(gbl::launch_bias_grad(n->dD, B, n->nc, g + n->o_fb2, s), "db fc2");
    NCK(gbl::launch_gemm(false, true,
                         gemm(B, kHid, n->nc, n->dD, n->nc, wh + n->o_f2, kHid, gbl::kGemmStore, n->dH, nullptr, kHid,
                              nullptr), 1, s), "dH");
    NCK(gbl::launch_relu_grad(n->dH, n->H, n->dZh, (size_t)B * kHid, 1.f, s), "relu grad");
    // fc1
    NCK(gemm_splitk(true, true, gemm(kHid, n->F, B, n->dZh, kHid, n->Fm, n->F, 0, g + n->o_f1, nullptr, n->F, nullptr), s),
        "dW fc1");
    NCK(gbl::launch_bias_grad(n->dZh, B, kHid, g + n->o_fb1, s), "db fc1");
    NCK(gbl::launch_gemm(false, true,
                         gemm(B, kNA, kHid, n->dZh, kHid, wh + n->o_f1, n->F, gbl::kGemmStore, n->dA3, nullptr, kNA,
                              nullptr), 1, s), "dA3");
    NCK(gbl::launch_relu_grad(n->dA3, n->A3, n->dZ3, (size_t)B * kNA, 1.f, s), "relu grad");
    // conv3
    NCK(gemm_splitk(true, true, gemm(kC, kK2, B * 64, n->dZ3, kC, n->X3, kK2, 0, g + n->o_w3, nullptr, kK2, nullptr), s),
        "dW conv3");
    NCK(gbl::launch_bias_grad(n->dZ3, B * 64, kC, g + n->o_b3, s), "db conv3");
    NCK(gbl::launch_gemm(false, true,
                         gemm(B * 64, kK2, kC, n->dZ3, kC, wh + n->o_w3, kK2, gbl::kGemmStore, n->dX, nullptr, kK2,
                              nullptr), 1, s), "dX3");
    gbl::Col2imArgs ca{B, 16, 16, 8, 8, kC, kK2, n->dX, n->A2, n->dZ2};
    NCK(gbl::launch_col2im(ca, s), "col2im");
    // conv2
    NCK(gemm_splitk(true, true, gemm(kC, kK2, B * 256, n->dZ2, kC, n->X2, kK2, 0, g + n->o_w2, nullptr, kK2, nullptr), s),
        "dW conv2");
    NCK(gbl::launch_bias_grad(n->dZ2, B * 256, kC, g + n->o_b2, s), "db conv2");
    NCK(gbl::launch_gemm(false, true,
                         gemm(B * 256, kK2, kC, n->dZ2, kC, wh + n->o_w2, kK2, gbl::kGemmStore, n->dX, nullptr, kK2,
                              nullptr), 1, s), "dX2");
    ca = gbl::Col2imArgs{B, 32, 32, 16, 16, kC, kK2, n->dX, n->A1, n->dZ1};
    NCK(gbl::launch_col2im(ca, s), "col2im");
    // conv1
    NCK(gemm_splitk(true, true, gemm(kC, kK1, B * 1024, n->dZ1, kC, n->X1, kK1, 0, g + n->o_w1, nullptr, kK1, nullptr), s),
        "dW conv1");
    NCK(gbl::launch_bias_grad(n->dZ1, B * 1024, kC, g + n->o_b1, s), "db conv1");
    return LIDAR_OK;
}

// Loss and gradient of a batch into n->g (scaled by kLossScale) and n->loss.
lidar_status_t loss_grad(lidar_tailnet_t *n, const void *inputs, const float *rows, const float *target, int B,
                         cudaStream_t s)
{
    lidar_status_t st = ensure_scratch(n, B, true);
    if (st != LIDAR_OK) return st;
    const __half *x = static_cast<const __half *>(inputs);
    if ((st = forward(n, x, rows, B, s)) != LIDAR_OK) return st;
    NCK(cudaMemsetAsync(n->g, 0, n->n_par * sizeof(float), s), "cudaMemsetAsync");
    NCK(cudaMemsetAsync(n->loss, 0, sizeof(float), s), "cudaMemsetAsync");
    NCK(cudaMemsetAsync(n->flag, 0, sizeof(int), s), "cudaMemsetAsync");
    gbl::HeadArgs ha{B, n->nc, n->nc + 4, rows, target, n->D, nullptr, n->loss, n->dD, kLossScale / (float)B};
    NCK(gbl::launch_head(ha, s), "head");
    if ((st = backward(n, x, B, s)) != LIDAR_OK) return st;
    NCK(gbl::launch_finite_check(n->g, n->n_par, n->flag, s), "finite check");
    return LIDAR_OK;
}

// Reads and clears the tcgen05 GEMM's error word (synchronous copy).
lidar_status_t check_timeout(lidar_tailnet_t *n)
{
    int h = 0;
    NCK(cudaMemcpy(&h, n->uerr, sizeof(int), cudaMemcpyDeviceToHost), "error word download");
    if (h) {
        NCK(cudaMemset(n->uerr, 0, sizeof(int)), "cudaMemset");
        return nfail(n, LIDAR_ETIMEOUT, "a bounded wait of the tensor-core GEMM gave up; outputs are undefined");
    }
    return LIDAR_OK;
}

// splitmix64 -> uniform in [-1, 1)
struct Rng {
    uint64_t s;
    double next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
};

}  // namespace

extern "C" {

lidar_status_t lidar_tailnet_create(int32_t n_coarse, uint64_t seed, lidar_tailnet_t **out)
{
    if (!out) return nfail(nullptr, LIDAR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_coarse < 8 || n_coarse > 1024 || n_coarse % 8 != 0)
        return nfail(nullptr, LIDAR_EINVAL, "n_coarse must be a multiple of 8 in [8, 1024]");
    lidar_tailnet_t *n = new (std::nothrow) lidar_tailnet();
    if (!n) return nfail(nullptr, LIDAR_ENOMEM, "host allocation failed");
    n->nc = n_coarse;
    n->F = kNA + kNL + n_coarse;
    size_t o = 0;
    auto take = [&](size_t cnt) { size_t r = o; o += (cnt + 7) / 8 * 8; return r; };
    n->o_w1 = take(kC * kK1); n->o_b1 = take(kC);
    n->o_w2 = take(kC * kK2); n->o_b2 = take(kC);
    n->o_w3 = take(kC * kK2); n->o_b3 = take(kC);
    n->o_f1 = take((size_t)kHid * n->F); n->o_fb1 = take(kHid);
    n->o_f2 = take((size_t)n_coarse * kHid); n->o_fb2 = take(n_coarse);
    n->n_par = o;
    // He-uniform initialisation of the real (unpadded) weights
    std::vector<float> h(n->n_par, 0.f);
    Rng r{seed};
    auto init = [&](size_t off, int rows, int cols, int used, double fan_in, double gain) {
        const double bound = gain * std::sqrt(6.0 / fan_in);
        for (int i = 0; i < rows; ++i)
            for (int j = 0; j < used; ++j) h[off + (size_t)i * cols + j] = (float)(bound * r.next());
    };
    init(n->o_w1, kC, kK1, 18, 18, 1.0);
    init(n->o_w2, kC, kK2, 306, 306, 1.0);
    init(n->o_w3, kC, kK2, 306, 306, 1.0);
    init(n->o_f1, kHid, n->F, n->F, n->F, 1.0);
    // the output layer starts at zero: the first prediction is the prior
    cudaError_t e;
    if ((e = cudaMalloc(&n->w, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->m, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->v, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->g, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->wh, n->n_par * sizeof(__half))) != cudaSuccess ||
        (e = cudaMalloc(&n->flag, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&n->loss, sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->uerr, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(n->uerr, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(n->w, h.data(), n->n_par * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(n->m, 0, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(n->v, 0, n->n_par * sizeof(float))) != cudaSuccess ||
        (e = gbl::launch_to_half(n->w, n->wh, n->n_par, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        lidar_status_t st = ncuda(nullptr, e, "tail network allocation");
        lidar_tailnet_destroy(n);
        return st;
    }
    *out = n;
    return LIDAR_OK;
}

void lidar_tailnet_destroy(lidar_tailnet_t *n)
{
    if (!n) return;
    free_scratch(n);
    free_pred(n);
    free_events(n);
    cudaFree(n->w); cudaFree(n->m); cudaFree(n->v); cudaFree(n->g); cudaFree(n->wh);
    cudaFree(n->flag); cudaFree(n->loss); cudaFree(n->uerr);
    delete n;
}

const char *lidar_tailnet_last_error(const lidar_tailnet_t *n) { return n ? n->err : g_net_err; }

lidar_status_t lidar_tailnet_set_dense(lidar_tailnet_t *n, int32_t mode)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    if (mode != LIDAR_DENSE_TCGEN05 && mode != LIDAR_DENSE_MMA_SYNC)
        return nfail(n, LIDAR_EINVAL, "dense mode must be LIDAR_DENSE_TCGEN05 or LIDAR_DENSE_MMA_SYNC");
    n->dense_mode = mode;
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_sync(lidar_tailnet_t *n, void *stream)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    NCK(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    NCK(cudaGetLastError(), "asynchronous error");
    return check_timeout(n);
}

int64_t lidar_tailnet_num_params(const lidar_tailnet_t *n) { return n ? (int64_t)n->n_par : 0; }

lidar_status_t lidar_tailnet_get_params(const lidar_tailnet_t *n, float *host, int64_t count)
{
    if (!n || !host) return nfail(nullptr, LIDAR_EINVAL, "NULL argument");
    if (count != (int64_t)n->n_par) return nfail(const_cast<lidar_tailnet_t *>(n), LIDAR_EINVAL, "count must be %zu", n->n_par);
    cudaError_t e = cudaMemcpy(host, n->w, n->n_par * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ncuda(const_cast<lidar_tailnet_t *>(n), e, "parameter download");
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_set_params(lidar_tailnet_t *n, const float *host, int64_t count)
{
    if (!n || !host) return nfail(n, LIDAR_EINVAL, "NULL argument");
    if (count != (int64_t)n->n_par) return nfail(n, LIDAR_EINVAL, "count must be %zu", n->n_par);
    NCK(cudaMemcpy(n->w, host, n->n_par * sizeof(float), cudaMemcpyHostToDevice), "parameter upload");
    NCK(gbl::launch_to_half(n->w, n->wh, n->n_par, 0), "to half");
    NCK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_predict(lidar_tailnet_t *n, const void *inputs, const float *rows, int32_t n_beams,
                                     float *tail_out, void *stream)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    if (!inputs || !rows || !tail_out || n_beams < 0) return nfail(n, LIDAR_EINVAL, "NULL argument or negative count");
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 65536;
    lidar_status_t st = ensure_pred(n, std::min<int>(chunk, std::max(1, n_beams)));
    if (st != LIDAR_OK) return st;
    if (!n->sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int rs = n->nc + 4;
    const __half *wh = n->wh;
    const float *w = n->w;
    for (int b0 = 0; b0 < n_beams; b0 += chunk) {
        const int B = std::min(chunk, n_beams - b0);
        const __half *x = static_cast<const __half *>(inputs) + (size_t)b0 * kIn;
        const float *r = rows + (size_t)b0 * rs;
        float *o = tail_out + (size_t)b0 * rs;
        // convolutions fused per beam -> f; then the two fully connected layers
        gbl::ConvArgs ca{B, x, r, n->nc, n->F, wh + n->o_w1, wh + n->o_w2, wh + n->o_w3, w + n->o_b1, w + n->o_b2,
                         w + n->o_b3, n->pF};
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (n->prof) {
            const size_t mark = n->ev_used;
            e0 = next_event(n); e1 = next_event(n); e2 = next_event(n);
            if (!e0 || !e1 || !e2) { n->ev_used = mark; e0 = e1 = e2 = nullptr; }
        }
        if (e0) cudaEventRecord(e0, s);
        NCK(gbl::launch_conv(ca, std::min(B, n->sms), s), "fused convolutions");
        if (e1) cudaEventRecord(e1, s);
        NCK(dense(n,
                             gemm(B, kHid, n->F, n->pF, n->F, wh + n->o_f1, n->F, gbl::kGemmBiasRelu, nullptr, n->pH,
                                  kHid, w + n->o_fb1), s), "fc1");
        NCK(dense(n,
                             gemm(B, n->nc, kHid, n->pH, kHid, wh + n->o_f2, kHid, gbl::kGemmBias, n->pD, nullptr,
                                  n->nc, w + n->o_fb2), s), "fc2");
        // s * y_hat into the rows, then clip to the bound and copy the bounds
        gbl::HeadArgs hb{B, n->nc, rs, r, nullptr, n->pD, o, nullptr, nullptr, 0.f};
        NCK(gbl::launch_head(hb, s), "head");
        NCK(gbl::launch_finish_rows(r, o, B, n->nc, s), "finish rows");
        if (e2) cudaEventRecord(e2, s);
    }
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_grads(lidar_tailnet_t *n, const void *inputs, const float *rows, const float *target,
                                   int32_t batch, float *grads_host, float *loss_host, void *stream)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    if (!inputs || !rows || !target || batch < 1) return nfail(n, LIDAR_EINVAL, "NULL argument or empty batch");
    cudaStream_t s = (cudaStream_t)stream;
    lidar_status_t st = loss_grad(n, inputs, rows, target, batch, s);
    if (st != LIDAR_OK) return st;
    NCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (grads_host) {
        NCK(cudaMemcpy(grads_host, n->g, n->n_par * sizeof(float), cudaMemcpyDeviceToHost), "gradient download");
        for (size_t i = 0; i < n->n_par; ++i) grads_host[i] /= kLossScale;
    }
    if (loss_host) NCK(cudaMemcpy(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost), "loss download");
    return check_timeout(n);
}

lidar_status_t lidar_tailnet_train_step(lidar_tailnet_t *n, const void *inputs, const float *rows,
                                        const float *target, int32_t batch, float lr, float *loss_host, void *stream)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    if (!inputs || !rows || !target || batch < 1) return nfail(n, LIDAR_EINVAL, "NULL argument or empty batch");
    if (!(lr > 0.f && std::isfinite(lr))) return nfail(n, LIDAR_EINVAL, "lr must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    lidar_status_t st = loss_grad(n, inputs, rows, target, batch, s);
    if (st != LIDAR_OK) return st;
    n->step += 1;
    gbl::AdamArgs a{};
    a.n = n->n_par; a.w = n->w; a.m = n->m; a.v = n->v; a.grad = n->g; a.wh = n->wh;
    a.lr = lr; a.b1 = 0.9f; a.b2 = 0.999f; a.eps = 1e-8f;
    a.c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)n->step)));
    a.c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)n->step)));
    a.inv_scale = 1.f / kLossScale;
    a.skip = n->flag;
    NCK(gbl::launch_adam(a, s), "adam");
    if (loss_host) {
        NCK(cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s), "loss download");
        NCK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        return check_timeout(n);
    }
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_save(const lidar_tailnet_t *cn, const char *path, int32_t with_state)
{
    lidar_tailnet_t *n = const_cast<lidar_tailnet_t *>(cn);
    if (!n || !path) return nfail(n, LIDAR_EINVAL, "NULL argument");
    std::vector<float> w(n->n_par), m, v;
    NCK(cudaMemcpy(w.data(), n->w, n->n_par * sizeof(float), cudaMemcpyDeviceToHost), "parameter download");
    if (with_state) {
        m.resize(n->n_par);
        v.resize(n->n_par);
        NCK(cudaMemcpy(m.data(), n->m, n->n_par * sizeof(float), cudaMemcpyDeviceToHost), "state download");
        NCK(cudaMemcpy(v.data(), n->v, n->n_par * sizeof(float), cudaMemcpyDeviceToHost), "state download");
    }
    FILE *f = std::fopen(path, "wb");
    if (!f) return nfail(n, LIDAR_EINVAL, "cannot open %s for writing", path);
    int32_t hdr[4] = {(int32_t)kMagic, 1, n->nc, with_state ? 1 : 0};
    int64_t cnt[2] = {(int64_t)n->n_par, n->step};
    bool ok = std::fwrite(hdr, sizeof hdr, 1, f) == 1 && std::fwrite(cnt, sizeof cnt, 1, f) == 1 &&
              std::fwrite(w.data(), sizeof(float), w.size(), f) == w.size();
    if (ok && with_state)
        ok = std::fwrite(m.data(), sizeof(float), m.size(), f) == m.size() &&
             std::fwrite(v.data(), sizeof(float), v.size(), f) == v.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return nfail(n, LIDAR_EINVAL, "write to %s failed", path);
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_load(lidar_tailnet_t *n, const char *path)
{
    if (!n || !path) return nfail(n, LIDAR_EINVAL, "NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return nfail(n, LIDAR_EINVAL, "cannot open %s", path);
    int32_t hdr[4];
    int64_t cnt[2];
    bool ok = std::fread(hdr, sizeof hdr, 1, f) == 1 && std::fread(cnt, sizeof cnt, 1, f) == 1;
    if (!ok || hdr[0] != (int32_t)kMagic || hdr[1] != 1) { std::fclose(f); return nfail(n, LIDAR_EINVAL, "%s: not a tail network file", path); }
    if (hdr[2] != n->nc || cnt[0] != (int64_t)n->n_par) {
        std::fclose(f);
        return nfail(n, LIDAR_EINVAL, "%s: network shape (n_coarse %d) differs from this network's (%d)", path, hdr[2], n->nc);
    }
    std::vector<float> w(n->n_par), m, v;
    ok = std::fread(w.data(), sizeof(float), w.size(), f) == w.size();
    if (ok && hdr[3]) {
        m.resize(n->n_par);
        v.resize(n->n_par);
        ok = std::fread(m.data(), sizeof(float), m.size(), f) == m.size() &&
             std::fread(v.data(), sizeof(float), v.size(), f) == v.size();
    }
    std::fclose(f);
    if (!ok) return nfail(n, LIDAR_EINVAL, "%s: truncated", path);
    NCK(cudaMemcpy(n->w, w.data(), n->n_par * sizeof(float), cudaMemcpyHostToDevice), "parameter upload");
    if (hdr[3]) {
        NCK(cudaMemcpy(n->m, m.data(), n->n_par * sizeof(float), cudaMemcpyHostToDevice), "state upload");
        NCK(cudaMemcpy(n->v, v.data(), n->n_par * sizeof(float), cudaMemcpyHostToDevice), "state upload");
        n->step = cnt[1];
    } else {
        NCK(cudaMemset(n->m, 0, n->n_par * sizeof(float)), "cudaMemset");
        NCK(cudaMemset(n->v, 0, n->n_par * sizeof(float)), "cudaMemset");
        n->step = 0;
    }
    NCK(gbl::launch_to_half(n->w, n->wh, n->n_par, 0), "to half");
    NCK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_profile_enable(lidar_tailnet_t *n, int32_t enable)
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    free_events(n);
    n->prof = enable != 0;
    return LIDAR_OK;
}

lidar_status_t lidar_tailnet_profile_read(lidar_tailnet_t *n, double total_ms[2], int32_t launches[2])
{
    if (!n) return nfail(nullptr, LIDAR_EINVAL, "network is NULL");
    double t[2] = {0, 0};
    int32_t c[2] = {0, 0};
    for (size_t i = 0; i + 3 <= n->ev_used; i += 3) {
        NCK(cudaEventSynchronize(n->ev[i + 2]), "cudaEventSynchronize");
        float a = 0, b = 0;
        NCK(cudaEventElapsedTime(&a, n->ev[i], n->ev[i + 1]), "cudaEventElapsedTime");
        NCK(cudaEventElapsedTime(&b, n->ev[i + 1], n->ev[i + 2]), "cudaEventElapsedTime");
        t[0] += a; t[1] += b; c[0] += 1; c[1] += 1;
    }
    n->ev_used = 0;
    if (total_ms) { total_ms[0] = t[0]; total_ms[1] = t[1]; }
    if (launches) { launches[0] = c[0]; launches[1] = c[1]; }
    return LIDAR_OK;
}

}  // extern "C"
