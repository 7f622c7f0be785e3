// Dense layers of the tail network on the 5th-generation tensor cores
// (tcgen05, sm_103a): C[m][n] = epilogue(sum_k A[m][k] B[n][k]) with FP16
// operands, FP32 accumulators in tensor memory (TMEM) and a bias / ReLU
// epilogue read back with tcgen05.ld.
//
// One CTA of 4 warps owns a 256-row tile of C with all N (16..256) columns,
// as two 128 x N accumulators in TMEM (columns [0, N) and [N, 2N)), so that
// each 64-wide K slice of B (the weights) feeds 256 rows:
//   - warp 0, lane 0 (producer): per K slice, one TMA tensor copy of A
//     (256 x 64) and one of B (N x 64) into a 3-stage ring of shared-memory
//     buffers, 128-byte swizzled (the K-major SWIZZLE_128B layout of the MMA
//     descriptors); rows and columns outside the matrices arrive as zeros.
//     The copies signal the stage's "full" mbarrier by transaction bytes.
//   - warp 1, lane 0 (MMA issuer): waits for a full stage, issues 2 x 4 MMAs
//     of 128 x N x 16 and commits them to the stage's "empty" mbarrier, which
//     the producer waits on before it reuses the stage; after the last slice
//     one more commit signals "done".
//   - all 4 warps (epilogue): wait for "done"; warp w reads TMEM lanes
//     32w..32w+31 of both accumulators 16 columns at a time and writes bias
//     (+ ReLU) as FP16 and/or FP32.
// Every mbarrier wait is bounded. On expiry the kernel records an error in
// the caller's error word, waits (bounded) for its MMAs and copies in flight,
// frees its TMEM and returns without writing C.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lidar_net_internal.h"

namespace gbl {

namespace {

constexpr int kUM = 128;                      // rows of one MMA (TMEM lanes)
constexpr int kTileM = 2 * kUM;               // rows per CTA
constexpr int kUK = 64;                       // K per stage: one 128-byte swizzle span of FP16
constexpr int kStages = 3;
constexpr uint32_t kABytes = kTileM * kUK * 2;   // 32 KB
constexpr uint32_t kBBytes = 256 * kUK * 2;      // 32 KB (room for N = 256)
constexpr long kWaitLimit = 1L << 22;         // bounded mbarrier polls (after the first 1024, >= 64 ns apart)

struct UmmaSmem {  // at a 1024-byte aligned offset of the dynamic buffer (swizzle atoms)
    unsigned char a[kStages][kABytes];
    unsigned char b[kStages][kBBytes];
    uint64_t full[kStages], empty[kStages], done;
    uint32_t tmem;
    int abort, issued, consumed;
};
constexpr size_t kSmemBytes = sizeof(UmmaSmem) + 1024;  // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: start address >> 4, leading byte offset 16 (unused for
// this layout), stride byte offset 1024 (8 rows x 128 B), descriptor version
// bit, swizzle mode 2 (128-byte). A K step of 16 elements inside the swizzle
// span advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N >> 3 and M >> 4.
__device__ __forceinline__ uint32_t instr_desc(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kUM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i >= 1024) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

}  // namespace

__global__ void __launch_bounds__(128, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, UmmaArgs g)
{
    extern __shared__ unsigned char umma_smem_raw[];
    const uint32_t raw = smem_u32(umma_smem_raw);
    UmmaSmem &S = *reinterpret_cast<UmmaSmem *>(umma_smem_raw + ((1024u - (raw & 1023u)) & 1023u));
    volatile int *abort_flag = &S.abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int nch = (g.K + kUK - 1) / kUK;
    const uint32_t stage_tx = kABytes + (uint32_t)g.N * kUK * 2;
    uint32_t ncols = 32;
    while ((int)ncols < 2 * g.N) ncols <<= 1;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
        S.issued = 0;
        S.consumed = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem;

    if (warp == 0 && lane == 0) {
        // producer
        int c = 0;
        for (; c < nch; ++c) {
            const int s = c % kStages;
            if (c >= kStages && !mbar_wait(smem_u32(&S.empty[s]), (uint32_t)((c / kStages - 1) & 1))) {
                *abort_flag = 1;
                break;
            }
            if (*abort_flag) break;
            const uint32_t fb = smem_u32(&S.full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stage_tx)
                         : "memory");
            tma_load_2d(smem_u32(S.a[s]), &tmA, c * kUK, m0, fb);
            tma_load_2d(smem_u32(S.b[s]), &tmB, c * kUK, 0, fb);
        }
        S.issued = c;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(g.N);
        int c = 0;
        for (; c < nch; ++c) {
            const int s = c % kStages;
            if (!mbar_wait(smem_u32(&S.full[s]), (uint32_t)((c / kStages) & 1))) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(S.a[s]), b0 = smem_u32(S.b[s]);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < kUK / 16; ++i)
                    mma_f16(tmem + (uint32_t)(h * g.N), sw128_desc(a0 + (uint32_t)h * (kUM * 128) + 32u * i),
                            sw128_desc(b0 + 32u * i), idesc, (c > 0 || i > 0) ? 1u : 0u);
            mma_commit(smem_u32(&S.empty[s]));
        }
        S.consumed = c;
        mma_commit(smem_u32(&S.done));  // arrives once every MMA issued above has completed
    }
    __syncthreads();

    // wait for the MMAs (also after an abort, before TMEM is freed)
    bool ok = mbar_wait(smem_u32(&S.done), 0u);
    ok = __syncthreads_and(ok && !*abort_flag) != 0;
    if (!ok) {
        if (tid == 0) {
            if (g.err) atomicExch(g.err, 1);
            // copies issued but never consumed: wait for them before the buffers go away
            for (int c = S.consumed; c < S.issued; ++c)
                mbar_wait(smem_u32(&S.full[c % kStages]), (uint32_t)((c / kStages) & 1));
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int row = m0 + h * kUM + warp * 32 + lane;
            for (int n0 = 0; n0 < g.N; n0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * g.N + n0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < g.M) {
                    float y[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        y[j] = __uint_as_float(v[j]) + (g.bias ? g.bias[n0 + j] : 0.f);
                        if (g.relu) y[j] = fmaxf(y[j], 0.f);
                    }
                    if (g.Ch) {
                        __half2 *d = reinterpret_cast<__half2 *>(g.Ch + (size_t)row * g.ldc + n0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) d[j] = __floats2half2_rn(y[2 * j], y[2 * j + 1]);
                    }
                    if (g.C) {
                        float2 *d = reinterpret_cast<float2 *>(g.C + (size_t)row * g.ldc + n0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) d[j] = make_float2(y[2 * j], y[2 * j + 1]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn load_encoder()
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
}

EncodeTiledFn encoder()
{
    static EncodeTiledFn fn = load_encoder();
    return fn;
}

// Row-major FP16 matrix [rows][ld] of which the first `cols` columns are
// used, read in boxes of box_rows x 64 with 128-byte swizzling; zero fill
// outside [rows) x [cols).
bool encode(CUtensorMap *map, const __half *ptr, int rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__half)};
    const cuuint32_t box[2] = {(cuuint32_t)kUK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool umma_gemm_supported(const UmmaArgs &g)
{
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    return encoder() != nullptr && g.M >= 0 && g.N >= 16 && g.N <= 256 && g.N % 16 == 0 && g.K >= 8 &&
           g.K % 8 == 0 && g.lda >= g.K && g.ldb >= g.K && g.lda % 8 == 0 && g.ldb % 8 == 0 && g.ldc >= g.N &&
           g.ldc % 2 == 0 && g.A && g.B && al16(g.A) && al16(g.B) && (g.C || g.Ch) &&
           (!g.Ch || ((uintptr_t)g.Ch & 3u) == 0) && (!g.C || ((uintptr_t)g.C & 7u) == 0);
}

cudaError_t launch_umma_gemm(const UmmaArgs &g, cudaStream_t s)
{
    if (!umma_gemm_supported(g)) return cudaErrorInvalidValue;
    if (g.M == 0) return cudaSuccess;
    CUtensorMap ta, tb;
    if (!encode(&ta, g.A, g.M, g.K, g.lda, kTileM) || !encode(&tb, g.B, g.N, g.K, g.ldb, g.N))
        return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    umma_gemm_kernel<<<(g.M + kTileM - 1) / kTileM, 128, kSmemBytes, s>>>(ta, tb, g);
    return cudaGetLastError();
}

}  // namespace gbl
