// Range stacking (Alg. 2) on sm_103a: include/lidar_stack.h.
//
//   stack_inputs_kernel  per pixel: intensity I = rho_hat * d omega (FP32,
//                        as the beam model's per-pixel prepass computes it)
//                        and the range index floor(R / dr) (FP64 division,
//                        so that slice boundaries match the definition), or
//                        0 ("no slice") outside 1..s_max.
//   stack_tile_kernel    one CTA per 32 x 8 output tile: the kernel and the
//                        tile's input region (tile + kernel halo) are staged
//                        in shared memory; each thread walks its pixel's
//                        stencil in the same order as its warp (the kernel
//                        weight is a broadcast), keeping the 24 nearest slices
//                        it meets with their sums; the nearest one at or above
//                        the threshold is the answer. If none is and more
//                        slices were present, the walk repeats above them.
//                        Slices too weak to reach the threshold anywhere in
//                        the tile are dropped first.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <stdint.h>
#include <vector>

#include "lidar_stack.h"

namespace {

constexpr int kTW = 32, kTH = 8;  // output tile (one thread per output pixel)
constexpr int kSlots = 16;         // slices one pass of the slot walk keeps (16: 76 registers, 3 CTAs per SM)
constexpr int kMaxK = 129;
constexpr int kSpan = 2048;       // slice range of a tile's region for which weak slices are dropped (8 KB histogram)
constexpr int kDense = 4;         // at most this many remaining slices: one dense pass per slice

struct StackArgs {
    int U, V;
    float az0, el0, daz, del, sv;
    const float *range, *nx, *ny, *nz, *rho, *retro;
    double dr;
    int s_max;
    float *I;           // [V][U]
    uint16_t *S;        // [V][U], 0 = no slice
    const float *K;     // [kh][kw]
    const float *Kc, *Kr;  // separable form: K[a][b] = Kc[a] Kr[b]
    int kh, kw;
    float thr, kmax;    // threshold, largest kernel weight
    int32_t *out_slice;
    float *out_val;
};

__global__ void __launch_bounds__(256) stack_inputs_kernel(StackArgs A)
{
    const long n = (long)A.U * A.V;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        const int v = (int)(idx / A.U), u = (int)(idx - (long)v * A.U);
        float w = 0.f;
        int s = 0;
        const float rr = A.range[idx];
        if (isfinite(rr) && rr > 0.f) {
            const float az = A.az0 + ((float)u + 0.5f) * A.daz;
            const float el = A.el0 + ((float)v + 0.5f) * A.del;
            float sa, ca, se, ce;
            sincosf(az, &sa, &ca);
            sincosf(el, &se, &ce);
            const float domega = 2.f * A.daz * ce * A.sv;
            const float dn = ce * (ca * A.nx[idx] + sa * A.ny[idx]) + se * A.nz[idx];
            const float beta = A.rho[idx] * (1.f / 3.14159265358979f) + A.retro[idx];
            w = beta * fabsf(dn) / (rr * rr) * domega;
            const double q = floor((double)rr / A.dr);
            if (q >= 1.0 && q <= (double)A.s_max) s = (int)q;
        }
        A.I[idx] = w;
        A.S[idx] = (uint16_t)s;
    }
}

// hist[s - slo] += the intensities of the region's pixels of slice s (s > 0),
// for the n region pixels; called by every thread of the block (whole warps).
// Neighbouring pixels mostly share a slice: a warp whose 32 pixels all do
// adds their sum with one atomic.
__device__ __forceinline__ void region_hist(float *hist, const uint16_t *RS, const float *RI, int n, int slo)
{
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int sv = i < n ? (int)RS[i] : 0;
        const float w = sv ? RI[i] : 0.f;
        int same = 0;
        __match_all_sync(0xffffffffu, sv, &same);
        if (same) {
            float t = w;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0 && sv) atomicAdd(&hist[sv - slo], t);
        } else if (sv) {
            atomicAdd(&hist[sv - slo], w);
        }
    }
}

__global__ void __launch_bounds__(kTW * kTH, 3) stack_tile_kernel(StackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int kh = A.kh, kw = A.kw, m = kh / 2, n = kw / 2;
    const int RH = kTH + kh - 1, RW = kTW + kw - 1;
    float *Ks = reinterpret_cast<float *>(smem);
    float *RI = Ks + kh * kw;
    uint16_t *RS = reinterpret_cast<uint16_t *>(RI + RH * RW);
    const int tid = threadIdx.x, tx = tid % kTW, ty = tid / kTW;
    const int u0 = blockIdx.x * kTW, v0 = blockIdx.y * kTH;
    for (int i = tid; i < kh * kw; i += blockDim.x) Ks[i] = A.K[i];
    // region rows v0 - m .. v0 + kTH - 1 + m, columns u0 - n .. u0 + kTW - 1 + n
    for (int i = tid; i < RH * RW; i += blockDim.x) {
        const int ry = i / RW, rx = i - ry * RW;
        const int v = v0 - m + ry, u = u0 - n + rx;
        float w = 0.f;
        uint16_t s = 0;
        if (v >= 0 && v < A.V && u >= 0 && u < A.U) {
            const long idx = (long)v * A.U + u;
            w = A.I[idx];
            s = A.S[idx];
        }
        RI[i] = w;
        RS[i] = s;
    }
    __syncthreads();

    // Slice skipping: a slice whose whole intensity in the region, times the
    // largest kernel weight, stays below the threshold cannot reach it at any
    // output of the tile; its pixels are dropped (when the region's slices span
    // at most kSpan indices, so that a shared-memory histogram holds them).
    // When at most kDense slices remain, each is convolved densely in turn
    // (nearest first) instead of the slot walk.
    __shared__ int dense_n;
    __shared__ int dense_s[kDense];
    {
        __shared__ int s_lo, s_hi;
        __shared__ float hist[kSpan];
        if (tid == 0) { s_lo = INT_MAX; s_hi = 0; dense_n = -1; }
        __syncthreads();
        int lo_ = INT_MAX, hi_ = 0;
        for (int i = tid; i < RH * RW; i += blockDim.x)
            if (RS[i]) { lo_ = min(lo_, (int)RS[i]); hi_ = max(hi_, (int)RS[i]); }
        atomicMin(&s_lo, lo_);
        atomicMax(&s_hi, hi_);
        __syncthreads();
        const int slo = s_lo, shi = s_hi;
        if (shi >= slo && shi - slo < kSpan) {
            for (int i = tid; i <= shi - slo; i += blockDim.x) hist[i] = 0.f;
            __syncthreads();
            region_hist(hist, RS, RI, RH * RW, slo);
            __syncthreads();
            const float cut = A.thr * (1.f - 1e-5f);
            for (int i = tid; i < RH * RW; i += blockDim.x)
                if (RS[i] && hist[RS[i] - slo] * A.kmax < cut) RS[i] = 0;
            __syncthreads();
            // the remaining slices in ascending order (one warp), if few
            if (tid < 32) {
                int cnt = 0;
                for (int b0 = 0; b0 <= shi - slo && cnt <= kDense; b0 += 32) {
                    const int bin = b0 + tid;
                    const bool keep = bin <= shi - slo && hist[bin] > 0.f && hist[bin] * A.kmax >= cut;
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const int pos = cnt + __popc(bal & ((1u << tid) - 1u));
                    if (keep && pos < kDense) dense_s[pos] = slo + bin;
                    cnt += __popc(bal);
                }
                if (tid == 0) dense_n = cnt <= kDense ? cnt : -1;
            }
        }
        __syncthreads();
    }

    const int u = u0 + tx, v = v0 + ty;
    bool done = !(u < A.U && v < A.V);
    int lo = 0;  // slices <= lo are known to stay below the threshold
    int outS = A.s_max;
    float outX = 0.f;
    // region coordinates of input (v - a + m, u - b + n): (ty + 2m - a, tx + 2n - b)
    const int base = (ty + 2 * m) * RW + (tx + 2 * n);
    if (dense_n >= 0) {
        for (int k = 0; k < dense_n && !done; ++k) {
            const int s = dense_s[k];
            float acc = 0.f;
            for (int a = 0; a < kh; ++a) {
                const int rb = base - a * RW;
                const float *krow = Ks + a * kw;
                for (int b = 0; b < kw; ++b) {
                    const float w = RS[rb - b] == s ? RI[rb - b] : 0.f;
                    acc = fmaf(w, krow[b], acc);
                }
            }
            if (acc >= A.thr) { outS = s; outX = acc; done = true; }
        }
        done = true;
    }
    while (__syncthreads_or(!done)) {
        if (done) continue;
        int sl[kSlots];
        float sum[kSlots];
#pragma unroll
        for (int k = 0; k < kSlots; ++k) { sl[k] = INT_MAX; sum[k] = 0.f; }
        bool over = false;
        // Adds (s, w) to the slots: keeps the kSlots nearest slices; the
        // farthest is replaced when a nearer one arrives (an empty slot is
        // INT_MAX). A slice that has to leave can never come back in this
        // pass, since the farthest kept slice only moves nearer.
        auto add = [&](int s, float w) {
            bool found = false;
            int imax = 0, smax = sl[0];
#pragma unroll
            for (int k = 0; k < kSlots; ++k) {
                if (sl[k] == s) { sum[k] += w; found = true; }
                if (sl[k] > smax) { smax = sl[k]; imax = k; }
            }
            if (!found) {
                if (s < smax) {
                    if (smax != INT_MAX) over = true;
#pragma unroll
                    for (int k = 0; k < kSlots; ++k)
                        if (k == imax) { sl[k] = s; sum[k] = w; }
                } else {
                    over = true;
                }
            }
        };
        // neighbouring stencil pixels mostly share a slice (a surface seen
        // along a row): their products are summed in a run first
        int run_s = 0;
        float run_w = 0.f;
        for (int a = 0; a < kh; ++a) {
            const int rb = base - a * RW;
            const float *krow = Ks + a * kw;
            for (int b = 0; b < kw; ++b) {
                const int s = RS[rb - b];
                if (s <= lo) continue;
                const float w = RI[rb - b] * krow[b];
                if (s == run_s) { run_w += w; continue; }
                if (run_s) add(run_s, run_w);
                run_s = s;
                run_w = w;
            }
        }
        if (run_s) add(run_s, run_w);
        int best = INT_MAX, kmax = 0;
        float bx = 0.f;
#pragma unroll
        for (int k = 0; k < kSlots; ++k) {
            if (sl[k] != INT_MAX && sum[k] >= A.thr && sl[k] < best) { best = sl[k]; bx = sum[k]; }
            if (sl[k] != INT_MAX) kmax = max(kmax, sl[k]);
        }
        if (best != INT_MAX) { outS = best; outX = bx; done = true; }
        else if (!over) done = true;
        else lo = kmax;
    }
    if (u < A.U && v < A.V) {
        const long idx = (long)v * A.U + u;
        A.out_slice[idx] = outS;
        A.out_val[idx] = outX;
    }
}

// ---------------------------------------------------------------------------
// Separable kernel K[a][b] = col[a] row[b] (lidar_stack_create_separable).
// One CTA of 256 threads per 32 x 32 output tile; region = tile + halo as in
// stack_tile_kernel. The slices present in the region (and strong enough to
// reach the threshold somewhere in the tile) are taken nearest first; per
// slice s a row pass writes R[ry][x] = sum_b row[b] I_s(ry, x - b + 2n) for
// every region row ry and output column x, and a column pass gives
// out(y, x) = sum_a col[a] R[y - a + 2m][x], where I_s is I on the pixels of
// slice s and 0 elsewhere; an output takes the first slice that reaches the
// threshold. Cost per output and slice O(kh + kw) instead of O(kh kw).
//
// Both passes are register-blocked: a thread makes 4 adjacent outputs (4
// columns of one region row in the row pass, 4 rows of one column in the
// column pass) from a window read in chunks of 4 elements. Output o and window
// element q of chunk c meet at tap 2h + o - 4c - q (h = half the kernel
// length), so a chunk touches 7 consecutive taps; the taps sit in a zero-padded
// copy whose padding makes every chunk's 8-tap slice 16-byte aligned, and
// consecutive chunks share 4 of them. Per chunk: one 16-byte load of
// intensities (+ 8 bytes of slice ids) or 4 loads of row sums, one 16-byte
// load of taps, 16 FMAs.
// ---------------------------------------------------------------------------

constexpr int kSW = 32, kSH = 32;   // output tile of the separable kernel
constexpr int kList = 64;           // slices listed per round

struct SepLayout {
    int nCr, nCc;     // window chunks of the row and the column pass
    int pr, pc;       // zero taps in front of row[] and col[]
    int Lr, Lc;       // padded tap array lengths (multiples of 4)
    int RH, RW, RWp;  // region rows, columns, padded row stride (multiple of 4)
    int RHb;          // rows of the row-pass result (the column pass reads past RH)
};

__host__ __device__ inline SepLayout sep_layout(int kh, int kw)
{
    SepLayout L;
    L.nCr = (kw + 6) >> 2;  // ceil((kw + 3) / 4): 4 outputs need kw + 3 window elements
    L.nCc = (kh + 6) >> 2;
    L.pr = ((kw - 1) & 3) ? 5 : 3;  // pad + (kw - 1) - 3 = 0 mod 4
    L.pc = ((kh - 1) & 3) ? 5 : 3;
    L.Lr = (L.pr + kw + 4 + 3) & ~3;
    L.Lc = (L.pc + kh + 4 + 3) & ~3;
    L.RH = kSH + kh - 1;
    L.RW = kSW + kw - 1;
    L.RWp = kSW + 4 * L.nCr;
    L.RWp += (8 - L.RWp % 16 + 16) % 16;  // rows 4 apart: disjoint banks for a half warp's slice ids
    L.RHb = kSH + 4 * L.nCc;
    return L;
}

// Output row (of a 32-row tile) of thread `tid` in a block of 256 whose lanes
// make 4 outputs each (8 lanes a row): the quarter warps of warp w take rows
// b, b + 4, b + 1, b + 5 with b = 8 (w / 2) + 2 (w % 2), so that each half warp
// reads two region rows 4 apart.
__device__ __forceinline__ int quad_row(int tid)
{
    const int w = tid >> 5, q = (tid >> 3) & 3;
    return 8 * (w >> 1) + 2 * (w & 1) + (q >> 1) + 4 * (q & 1);
}

// acc[o] += sum_q w[q] k[3 + o - q], k = (lo, hi) the chunk's 8 taps
__device__ __forceinline__ void chunk_fma(float acc[4], const float w[4], float4 lo, float4 hi)
{
    const float k[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[o] = fmaf(w[q], k[3 + o - q], acc[o]);
}

__global__ void __launch_bounds__(256) stack_sep_kernel(StackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int kh = A.kh, kw = A.kw, m = kh / 2, n = kw / 2;
    const SepLayout L = sep_layout(kh, kw);
    const int RH = L.RH, RW = L.RW, RWp = L.RWp;
    float *Kc = reinterpret_cast<float *>(smem);   // [Lc]: col[a] at pc + a, zeros elsewhere
    float *Kr = Kc + L.Lc;                          // [Lr]: row[b] at pr + b
    float *Rb = Kr + L.Lr;                          // row-pass result [RHb][kSW]
    float *RI = Rb + L.RHb * kSW;                   // region intensity [RH][RWp]
    uint16_t *RS = reinterpret_cast<uint16_t *>(RI + RH * RWp);  // region slice [RH][RWp]
    unsigned long long *rmask = reinterpret_cast<unsigned long long *>(RS + RH * RWp);  // [RH]: listed slices on the row
    __shared__ float hist[kSpan];
    __shared__ signed char lpos[kSpan];  // list position of a slice (bin - slo), or -1
    __shared__ int lst[kList];
    __shared__ short srow[kList][2];     // first and last region row holding listed slice k
    __shared__ int s_lo, s_hi, s_cnt, s_min;
    const int tid = threadIdx.x;
    const int u0 = blockIdx.x * kSW, v0 = blockIdx.y * kSH;
    for (int i = tid; i < L.Lc; i += blockDim.x) Kc[i] = (i >= L.pc && i < L.pc + kh) ? A.Kc[i - L.pc] : 0.f;
    for (int i = tid; i < L.Lr; i += blockDim.x) Kr[i] = (i >= L.pr && i < L.pr + kw) ? A.Kr[i - L.pr] : 0.f;
    for (int i = RH * kSW + tid; i < L.RHb * kSW; i += blockDim.x) Rb[i] = 0.f;  // never written again
    for (int i = tid; i < RH * RWp; i += blockDim.x) {
        const int ry = i / RWp, rx = i - ry * RWp;
        const int v = v0 - m + ry, u = u0 - n + rx;
        float w = 0.f;
        uint16_t s = 0;
        if (rx < RW && v >= 0 && v < A.V && u >= 0 && u < A.U) {
            const long idx = (long)v * A.U + u;
            w = A.I[idx];
            s = A.S[idx];
        }
        RI[i] = w;
        RS[i] = s;
    }
    for (int i = tid; i < kSpan; i += blockDim.x) lpos[i] = -1;
    if (tid == 0) { s_lo = INT_MAX; s_hi = 0; }
    __syncthreads();
    {
        int lo_ = INT_MAX, hi_ = 0;
        for (int i = tid; i < RH * RWp; i += blockDim.x)
            if (RS[i]) { lo_ = min(lo_, (int)RS[i]); hi_ = max(hi_, (int)RS[i]); }
        atomicMin(&s_lo, lo_);
        atomicMax(&s_hi, hi_);
    }
    __syncthreads();
    const int slo = s_lo, shi = s_hi;
    const bool use_hist = shi >= slo && shi - slo < kSpan;
    const float cut = A.thr * (1.f - 1e-5f);
    if (use_hist) {
        for (int i = tid; i <= shi - slo; i += blockDim.x) hist[i] = 0.f;
        __syncthreads();
        region_hist(hist, RS, RI, RH * RWp, slo);
        __syncthreads();
    }

    // column pass: this thread's outputs are rows 4 g + o of column tx
    const int tx = tid % kSW, g = tid / kSW;
    int outS[4];
    float outX[4];
    int done = 0;  // bit o: output row 4 g + o has its answer (or is outside the image)
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        outS[o] = A.s_max;
        outX[o] = 0.f;
        if (!(u0 + tx < A.U && v0 + 4 * g + o < A.V)) done |= 1 << o;
    }
    const float4 *Kr4 = reinterpret_cast<const float4 *>(Kr + L.pr + 2 * n - 3);  // taps of chunk 0
    const float4 *Kc4 = reinterpret_cast<const float4 *>(Kc + L.pc + 2 * m - 3);
    int lo = 0;  // slices <= lo have been processed
    bool finished = __syncthreads_and(done == 0xF) != 0;
    while (!finished) {
        // the next (up to kList) slices above lo, nearest first
        if (tid == 0) { s_cnt = 0; s_min = INT_MAX; }
        __syncthreads();
        if (use_hist) {
            if (tid < 32) {
                int cnt = 0;
                for (int b0 = max(0, lo + 1 - slo); b0 <= shi - slo && cnt < kList; b0 += 32) {
                    const int bin = b0 + tid;
                    const bool keep = bin <= shi - slo && hist[bin] > 0.f && hist[bin] * A.kmax >= cut;
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const int pos = cnt + __popc(bal & ((1u << tid) - 1u));
                    if (keep && pos < kList) lst[pos] = slo + bin;
                    cnt += __popc(bal);
                }
                if (tid == 0) s_cnt = min(cnt, kList);
            }
        } else {
            int mn = INT_MAX;
            for (int i = tid; i < RH * RWp; i += blockDim.x)
                if (RS[i] > lo) mn = min(mn, (int)RS[i]);
            atomicMin(&s_min, mn);
            __syncthreads();
            if (tid == 0 && s_min != INT_MAX) { lst[0] = s_min; s_cnt = 1; }
        }
        __syncthreads();
        const int cnt = s_cnt;
        if (cnt == 0) break;
        // which listed slices lie on each region row (one warp per row), and
        // the first and last row of each
        const int lane = tid & 31, warp = tid >> 5;
        if (use_hist && tid < cnt) lpos[lst[tid] - slo] = (signed char)tid;
        __syncthreads();
        for (int r = warp; r < RH; r += (int)(blockDim.x >> 5)) {
            unsigned mlo = 0u, mhi = 0u;
            for (int x = lane; x < RW; x += 32) {
                const int sv = RS[r * RWp + x];
                int q = -1;
                if (use_hist) { if (sv >= slo && sv <= shi) q = lpos[sv - slo]; }
                else if (sv == lst[0]) q = 0;
                if (q >= 0) { if (q < 32) mlo |= 1u << q; else mhi |= 1u << (q - 32); }
            }
            mlo = __reduce_or_sync(0xffffffffu, mlo);
            mhi = __reduce_or_sync(0xffffffffu, mhi);
            if (lane == 0) rmask[r] = ((unsigned long long)mhi << 32) | mlo;
        }
        __syncthreads();
        if (tid < cnt) {
            if (use_hist) lpos[lst[tid] - slo] = -1;
            int r0 = RH, r1 = -1;
            for (int r = 0; r < RH; ++r)
                if ((rmask[r] >> tid) & 1ull) { r0 = min(r0, r); r1 = r; }
            srow[tid][0] = (short)r0;
            srow[tid][1] = (short)r1;
        }
        __syncthreads();
        for (int k = 0; k < cnt && !finished; ++k) {
            const int s = lst[k];
            const unsigned long long bit = 1ull << k;
            // row pass: item = (region row ry, column group cg of 4 outputs);
            // the 8 items of a row are adjacent threads (one 128-byte row of
            // 16-byte loads per quarter warp), blocks of 32 rows as quad_row
            for (int it = tid; it < ((RH + 31) & ~31) * (kSW / 4); it += blockDim.x) {
                const int ry = 32 * (it >> 8) + quad_row(it & 255), cg = it & 7;
                if (ry >= RH) continue;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                if (rmask[ry] & bit) {
                    const float4 *wI = reinterpret_cast<const float4 *>(RI + ry * RWp + 4 * cg);
                    const uint2 *wS = reinterpret_cast<const uint2 *>(RS + ry * RWp + 4 * cg);
                    float4 hi = Kr4[1];
                    for (int c = 0; c < L.nCr; ++c) {
                        const float4 x = wI[c];
                        const uint2 t = wS[c];
                        const float w[4] = {(int)(t.x & 0xFFFFu) == s ? x.x : 0.f, (int)(t.x >> 16) == s ? x.y : 0.f,
                                            (int)(t.y & 0xFFFFu) == s ? x.z : 0.f, (int)(t.y >> 16) == s ? x.w : 0.f};
                        const float4 lo4 = Kr4[-c];
                        chunk_fma(acc, w, lo4, hi);
                        hi = lo4;
                    }
                }
                reinterpret_cast<float4 *>(Rb + ry * kSW)[cg] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            }
            __syncthreads();
            // column pass and the threshold test, over the chunks of rows
            // 4 g + 4 c .. + 3 that meet the rows holding the slice (the row
            // sums are zero elsewhere)
            if (done != 0xF) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                const float *col = Rb + 4 * g * kSW + tx;
                const int x0 = srow[k][0] - 4 * g, x1 = srow[k][1] - 4 * g;
                const int c0 = x0 > 0 ? x0 >> 2 : 0, c1 = x1 >= 0 ? min(L.nCc - 1, x1 >> 2) : -1;
                if (c0 <= c1) {  // then 0 <= c0 <= nCc - 1: the taps Kc4[1 - c0] exist
                    float4 hi = Kc4[1 - c0];
                    for (int c = c0; c <= c1; ++c) {
                        const float *r = col + 4 * c * kSW;
                        const float w[4] = {r[0], r[kSW], r[2 * kSW], r[3 * kSW]};
                        const float4 lo4 = Kc4[-c];
                        chunk_fma(acc, w, lo4, hi);
                        hi = lo4;
                    }
                }
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    if (!((done >> o) & 1) && acc[o] >= A.thr) { outS[o] = s; outX[o] = acc[o]; done |= 1 << o; }
            }
            finished = __syncthreads_and(done == 0xF) != 0;  // also: Rb is free again
        }
        lo = lst[cnt - 1];
        __syncthreads();  // every thread has read lst before the next round overwrites it
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int u = u0 + tx, v = v0 + 4 * g + o;
        if (u < A.U && v < A.V) {
            const long idx = (long)v * A.U + u;
            A.out_slice[idx] = outS[o];
            A.out_val[idx] = outX[o];
        }
    }
}

// ---------------------------------------------------------------------------
// General kernel, dense form (kernels whose 32 x 32 tile layout fits shared
// memory). As the separable kernel: 32 x 32 output tiles, the region's strong
// slices listed 64 at a time nearest first, one pass per slice, the first
// slice reaching the threshold kept. A pass computes the full 2-D sum,
// out(y, x) = sum_a sum_b K[a][b] I_s(y + 2m - a, x + 2n - b), register-blocked
// as the separable row pass (4 outputs of a row per thread, 4-element window
// chunks, each kernel row zero-padded), and skips every kernel row whose
// region row holds no pixel of the slice (an exact bit per listed slice and
// region row): on a surface seen at grazing incidence a slice covers a few
// rows of the region, so most of the kh rows of a pass are skipped.
// ---------------------------------------------------------------------------

struct DenseLayout {
    int nC;       // window chunks per row
    int pr;       // zero taps in front of each kernel row
    int Lr;       // padded kernel row length (multiple of 4)
    int RH, RW, RWp;
};

__host__ __device__ inline DenseLayout dense_layout(int kh, int kw)
{
    DenseLayout L;
    L.nC = (kw + 6) >> 2;
    L.pr = ((kw - 1) & 3) ? 5 : 3;
    L.Lr = (L.pr + kw + 4 + 3) & ~3;
    L.RH = kSH + kh - 1;
    L.RW = kSW + kw - 1;
    // row stride = 8 (mod 16) floats: rows 4 apart are 16 (mod 32) words of
    // slice ids apart, so a half warp reading two such rows (8 bytes a lane)
    // hits each bank once
    L.RWp = kSW + 4 * L.nC;
    L.RWp += (8 - L.RWp % 16 + 16) % 16;
    return L;
}

__global__ void __launch_bounds__(256) stack_dense_kernel(StackArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int kh = A.kh, kw = A.kw, m = kh / 2, n = kw / 2;
    const DenseLayout L = dense_layout(kh, kw);
    const int RH = L.RH, RW = L.RW, RWp = L.RWp;
    float *Kp = reinterpret_cast<float *>(smem);                  // [kh][Lr]: K[a][b] at a Lr + pr + b
    float *RI = Kp + kh * L.Lr;                                    // region intensity [RH][RWp]
    uint16_t *RS = reinterpret_cast<uint16_t *>(RI + RH * RWp);    // region slice [RH][RWp]
    unsigned long long *rmask = reinterpret_cast<unsigned long long *>(RS + RH * RWp);  // [RH]: listed slices on the row
    __shared__ float hist[kSpan];
    __shared__ signed char lpos[kSpan];  // list position of a slice (bin - slo), or -1
    __shared__ int lst[kList];
    __shared__ short srow[kList][2];     // first and last region row holding listed slice k
    __shared__ int s_lo, s_hi, s_cnt, s_min;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int u0 = blockIdx.x * kSW, v0 = blockIdx.y * kSH;
    for (int i = tid; i < kh * L.Lr; i += blockDim.x) {
        const int a = i / L.Lr, c = i - a * L.Lr;
        Kp[i] = (c >= L.pr && c < L.pr + kw) ? A.K[a * kw + c - L.pr] : 0.f;
    }
    for (int i = tid; i < RH * RWp; i += blockDim.x) {
        const int ry = i / RWp, rx = i - ry * RWp;
        const int v = v0 - m + ry, u = u0 - n + rx;
        float w = 0.f;
        uint16_t s = 0;
        if (rx < RW && v >= 0 && v < A.V && u >= 0 && u < A.U) {
            const long idx = (long)v * A.U + u;
            w = A.I[idx];
            s = A.S[idx];
        }
        RI[i] = w;
        RS[i] = s;
    }
    for (int i = tid; i < kSpan; i += blockDim.x) lpos[i] = -1;
    if (tid == 0) { s_lo = INT_MAX; s_hi = 0; }
    __syncthreads();
    {
        int lo_ = INT_MAX, hi_ = 0;
        for (int i = tid; i < RH * RWp; i += blockDim.x)
            if (RS[i]) { lo_ = min(lo_, (int)RS[i]); hi_ = max(hi_, (int)RS[i]); }
        atomicMin(&s_lo, lo_);
        atomicMax(&s_hi, hi_);
    }
    __syncthreads();
    const int slo = s_lo, shi = s_hi;
    const bool use_hist = shi >= slo && shi - slo < kSpan;
    const float cut = A.thr * (1.f - 1e-5f);
    if (use_hist) {
        for (int i = tid; i <= shi - slo; i += blockDim.x) hist[i] = 0.f;
        __syncthreads();
        region_hist(hist, RS, RI, RH * RWp, slo);
        __syncthreads();
    }

    // this thread's outputs: row y, columns 4 cg + o
    const int y = quad_row(tid), cg = tid & 7;
    int outS[4];
    float outX[4];
    int done = 0;  // bit o: output (y, 4 cg + o) has its answer (or is outside the image)
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        outS[o] = A.s_max;
        outX[o] = 0.f;
        if (!(u0 + 4 * cg + o < A.U && v0 + y < A.V)) done |= 1 << o;
    }
    const int kbase = L.pr + 2 * n - 3;  // taps of chunk 0 in each padded kernel row (multiple of 4)
    int lo = 0;  // slices <= lo have been processed
    bool finished = __syncthreads_and(done == 0xF) != 0;
    while (!finished) {
        // the next (up to kList) slices above lo, nearest first
        if (tid == 0) { s_cnt = 0; s_min = INT_MAX; }
        __syncthreads();
        if (use_hist) {
            if (tid < 32) {
                int cnt = 0;
                for (int b0 = max(0, lo + 1 - slo); b0 <= shi - slo && cnt < kList; b0 += 32) {
                    const int bin = b0 + tid;
                    const bool keep = bin <= shi - slo && hist[bin] > 0.f && hist[bin] * A.kmax >= cut;
                    const unsigned bal = __ballot_sync(0xffffffffu, keep);
                    const int pos = cnt + __popc(bal & ((1u << tid) - 1u));
                    if (keep && pos < kList) lst[pos] = slo + bin;
                    cnt += __popc(bal);
                }
                if (tid == 0) s_cnt = min(cnt, kList);
            }
        } else {
            int mn = INT_MAX;
            for (int i = tid; i < RH * RWp; i += blockDim.x)
                if (RS[i] > lo) mn = min(mn, (int)RS[i]);
            atomicMin(&s_min, mn);
            __syncthreads();
            if (tid == 0 && s_min != INT_MAX) { lst[0] = s_min; s_cnt = 1; }
        }
        __syncthreads();
        const int cnt = s_cnt;
        if (cnt == 0) break;
        // which listed slices lie on each region row (one warp per row)
        if (use_hist && tid < cnt) lpos[lst[tid] - slo] = (signed char)tid;
        __syncthreads();
        for (int r = warp; r < RH; r += (int)(blockDim.x >> 5)) {
            unsigned mlo = 0u, mhi = 0u;
            for (int x = lane; x < RW; x += 32) {
                const int sv = RS[r * RWp + x];
                int k = -1;
                if (use_hist) { if (sv >= slo && sv <= shi) k = lpos[sv - slo]; }
                else if (sv == lst[0]) k = 0;
                if (k >= 0) { if (k < 32) mlo |= 1u << k; else mhi |= 1u << (k - 32); }
            }
            mlo = __reduce_or_sync(0xffffffffu, mlo);
            mhi = __reduce_or_sync(0xffffffffu, mhi);
            if (lane == 0) rmask[r] = ((unsigned long long)mhi << 32) | mlo;
        }
        __syncthreads();
        if (tid < cnt) {
            if (use_hist) lpos[lst[tid] - slo] = -1;
            int r0 = RH, r1 = -1;
            for (int r = 0; r < RH; ++r)
                if ((rmask[r] >> tid) & 1ull) { r0 = min(r0, r); r1 = r; }
            srow[tid][0] = (short)r0;
            srow[tid][1] = (short)r1;
        }
        __syncthreads();
        for (int k = 0; k < cnt && !finished; ++k) {
            const int s = lst[k];
            const unsigned long long bit = 1ull << k;
            if (done != 0xF) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                // kernel rows a whose region row y + 2m - a lies in the slice's rows
                const int a0 = max(0, y + 2 * m - srow[k][1]), a1 = min(kh - 1, y + 2 * m - srow[k][0]);
                for (int a = a0; a <= a1; ++a) {
                    const int r = y + 2 * m - a;  // region row of kernel row a for output row y
                    if (!(rmask[r] & bit)) continue;
                    const float4 *wI = reinterpret_cast<const float4 *>(RI + r * RWp + 4 * cg);
                    const uint2 *wS = reinterpret_cast<const uint2 *>(RS + r * RWp + 4 * cg);
                    const float4 *K4 = reinterpret_cast<const float4 *>(Kp + a * L.Lr + kbase);
                    float4 hi = K4[1];
                    for (int c = 0; c < L.nC; ++c) {
                        const float4 x = wI[c];
                        const uint2 t = wS[c];
                        const float w[4] = {(int)(t.x & 0xFFFFu) == s ? x.x : 0.f, (int)(t.x >> 16) == s ? x.y : 0.f,
                                            (int)(t.y & 0xFFFFu) == s ? x.z : 0.f, (int)(t.y >> 16) == s ? x.w : 0.f};
                        const float4 lo4 = K4[-c];
                        chunk_fma(acc, w, lo4, hi);
                        hi = lo4;
                    }
                }
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    if (!((done >> o) & 1) && acc[o] >= A.thr) { outS[o] = s; outX[o] = acc[o]; done |= 1 << o; }
            }
            finished = __syncthreads_and(done == 0xF) != 0;
        }
        lo = lst[cnt - 1];
        __syncthreads();  // every thread has read lst (and rmask) before the next round overwrites them
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int u = u0 + 4 * cg + o, v = v0 + y;
        if (u < A.U && v < A.V) {
            const long idx = (long)v * A.U + u;
            A.out_slice[idx] = outS[o];
            A.out_val[idx] = outX[o];
        }
    }
}

thread_local char g_stack_err[512] = "no error";

}  // namespace

struct lidar_stack {
    int kh = 0, kw = 0, s_max = 0;
    double dr = 0, thr = 0;
    float kmax = 0.f;
    bool sep = false;           // separable kernel: row/column passes
    bool dense = false;         // general kernel in the dense form (its tile layout fits shared memory)
    float *d_K = nullptr;       // [kh][kw], or col[kh] then row[kw] when sep
    float *d_I = nullptr;
    uint16_t *d_S = nullptr;
    size_t cap = 0;
    char err[512] = "no error";
};

namespace {

lidar_status_t sfail(lidar_stack_t *h, lidar_status_t st, const char *fmt, ...)
{
    char *buf = h ? h->err : g_stack_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

lidar_status_t scuda(lidar_stack_t *h, cudaError_t e, const char *what)
{
    return sfail(h, e == cudaErrorMemoryAllocation ? LIDAR_ENOMEM : LIDAR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t tile_smem(int kh, int kw)
{
    const size_t RH = kTH + kh - 1, RW = kTW + kw - 1;
    return (size_t)kh * kw * 4 + RH * RW * 4 + RH * RW * 2;
}

// dynamic shared memory of stack_dense_kernel: padded kernel rows, region
// (float + uint16), per-row slice masks
size_t dense_smem(int kh, int kw)
{
    const DenseLayout L = dense_layout(kh, kw);
    return (size_t)kh * L.Lr * 4 + (size_t)L.RH * L.RWp * 6 + (size_t)L.RH * 8;
}

// dynamic shared memory of stack_sep_kernel: padded taps, row-pass result,
// region (float + uint16), per-row slice range
size_t sep_smem(int kh, int kw)
{
    const SepLayout L = sep_layout(kh, kw);
    return (size_t)(L.Lc + L.Lr) * 4 + (size_t)L.RHb * kSW * 4 + (size_t)L.RH * L.RWp * 6 + (size_t)L.RH * 8;
}

lidar_status_t check_common(int kh, int kw, double thr, double dr, double r_max, double *sm)
{
    if (kh < 1 || kw < 1 || kh > kMaxK || kw > kMaxK || !(kh & 1) || !(kw & 1))
        return sfail(nullptr, LIDAR_EINVAL, "kernel sizes must be odd and in [1, %d]", kMaxK);
    if (!(std::isfinite(thr) && thr > 0)) return sfail(nullptr, LIDAR_EINVAL, "threshold must be > 0");
    if (!(std::isfinite(dr) && dr > 0)) return sfail(nullptr, LIDAR_EINVAL, "dr must be > 0");
    if (!std::isfinite(r_max)) return sfail(nullptr, LIDAR_EINVAL, "r_max must be finite");
    *sm = std::floor(r_max / dr);
    if (!(*sm >= 1 && *sm <= 65535)) return sfail(nullptr, LIDAR_EINVAL, "floor(r_max / dr) must be in [1, 65535]");
    return LIDAR_OK;
}

}  // namespace

extern "C" {

lidar_status_t lidar_stack_create(const lidar_stack_params_t *p, lidar_stack_t **out)
{
    if (!out) return sfail(nullptr, LIDAR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p || !p->kernel) return sfail(nullptr, LIDAR_EINVAL, "params or kernel is NULL");
    if (p->kh < 1 || p->kw < 1 || p->kh > kMaxK || p->kw > kMaxK || !(p->kh & 1) || !(p->kw & 1))
        return sfail(nullptr, LIDAR_EINVAL, "kernel sizes must be odd and in [1, %d]", kMaxK);
    if (!(std::isfinite(p->threshold) && p->threshold > 0)) return sfail(nullptr, LIDAR_EINVAL, "threshold must be > 0");
    if (!(std::isfinite(p->dr) && p->dr > 0)) return sfail(nullptr, LIDAR_EINVAL, "dr must be > 0");
    if (!std::isfinite(p->r_max)) return sfail(nullptr, LIDAR_EINVAL, "r_max must be finite");
    const double sm = std::floor(p->r_max / p->dr);
    if (!(sm >= 1 && sm <= 65535)) return sfail(nullptr, LIDAR_EINVAL, "floor(r_max / dr) must be in [1, 65535]");
    for (int i = 0; i < p->kh * p->kw; ++i)
        if (!(std::isfinite(p->kernel[i]) && p->kernel[i] >= 0.f))
            return sfail(nullptr, LIDAR_EINVAL, "kernel[%d] is negative or not finite", i);
    // dynamic shared memory next to the kernel's 16 KB histogram (227 KB per block)
    if (tile_smem(p->kh, p->kw) > 210 * 1024) return sfail(nullptr, LIDAR_EINVAL, "kernel too large");
    lidar_stack_t *h = new (std::nothrow) lidar_stack();
    if (!h) return sfail(nullptr, LIDAR_ENOMEM, "host allocation failed");
    h->kh = p->kh; h->kw = p->kw; h->s_max = (int)sm; h->dr = p->dr; h->thr = p->threshold;
    for (int i = 0; i < p->kh * p->kw; ++i) h->kmax = std::max(h->kmax, p->kernel[i]);
    cudaError_t e;
    // the dense form where its layout leaves room for the static arrays (~10 KB)
    h->dense = dense_smem(p->kh, p->kw) <= 200 * 1024;
    if ((e = cudaMalloc(&h->d_K, (size_t)p->kh * p->kw * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(h->d_K, p->kernel, (size_t)p->kh * p->kw * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(stack_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tile_smem(p->kh, p->kw))) != cudaSuccess ||
        (h->dense && (e = cudaFuncSetAttribute(stack_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)dense_smem(p->kh, p->kw))) != cudaSuccess)) {
        lidar_status_t st = scuda(nullptr, e, "range stacking set-up");
        lidar_stack_destroy(h);
        return st;
    }
    *out = h;
    return LIDAR_OK;
}

lidar_status_t lidar_range_stack(lidar_stack_t *h, const lidar_gbuffer_t *g, int32_t *out_slice, float *out_intensity,
                                 void *stream)
{
    if (!h) return sfail(nullptr, LIDAR_EINVAL, "handle is NULL");
    if (!g || !out_slice || !out_intensity) return sfail(h, LIDAR_EINVAL, "gbuffer or output pointer is NULL");
    if (g->U < 1 || g->V < 1 || (long long)g->U * g->V > (1LL << 30))
        return sfail(h, LIDAR_EINVAL, "gbuffer size must be 1..2^30 pixels");
    if (!(std::isfinite(g->daz) && g->daz > 0 && std::isfinite(g->del) && g->del > 0))
        return sfail(h, LIDAR_EINVAL, "gbuffer daz, del must be > 0");
    if (!g->range || !g->nx || !g->ny || !g->nz || !g->rho_d || !g->retro)
        return sfail(h, LIDAR_EINVAL, "gbuffer plane pointer is NULL");
    const size_t np = (size_t)g->U * g->V;
    cudaError_t e;
    if (np > h->cap) {
        cudaFree(h->d_I);
        cudaFree(h->d_S);
        h->d_I = nullptr; h->d_S = nullptr; h->cap = 0;
        if ((e = cudaMalloc(&h->d_I, np * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&h->d_S, np * sizeof(uint16_t))) != cudaSuccess)
            return scuda(h, e, "cudaMalloc(range stacking scratch)");
        h->cap = np;
    }
    StackArgs a{};
    a.U = g->U; a.V = g->V;
    a.az0 = (float)g->az0; a.el0 = (float)g->el0; a.daz = (float)g->daz; a.del = (float)g->del;
    a.sv = (float)std::sin(0.5 * g->del);
    a.range = g->range; a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.rho = g->rho_d; a.retro = g->retro;
    a.dr = h->dr; a.s_max = h->s_max;
    a.I = h->d_I; a.S = h->d_S; a.K = h->d_K; a.kh = h->kh; a.kw = h->kw; a.thr = (float)h->thr;
    if (h->sep) { a.Kc = h->d_K; a.Kr = h->d_K + h->kh; }
    a.kmax = h->kmax;
    a.out_slice = out_slice; a.out_val = out_intensity;
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = (int)std::min<size_t>((np + 255) / 256, 152 * 16);
    stack_inputs_kernel<<<grid, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return scuda(h, e, "range stacking input kernel launch");
    if (h->sep) {
        dim3 sg((g->U + kSW - 1) / kSW, (g->V + kSH - 1) / kSH);
        stack_sep_kernel<<<sg, 256, sep_smem(h->kh, h->kw), s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return scuda(h, e, "range stacking separable kernel launch");
        return LIDAR_OK;
    }
    if (h->dense) {
        dim3 dg((g->U + kSW - 1) / kSW, (g->V + kSH - 1) / kSH);
        stack_dense_kernel<<<dg, 256, dense_smem(h->kh, h->kw), s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return scuda(h, e, "range stacking dense kernel launch");
        return LIDAR_OK;
    }
    dim3 tg((g->U + kTW - 1) / kTW, (g->V + kTH - 1) / kTH);
    stack_tile_kernel<<<tg, kTW * kTH, tile_smem(h->kh, h->kw), s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return scuda(h, e, "range stacking tile kernel launch");
    return LIDAR_OK;
}

lidar_status_t lidar_stack_create_separable(const lidar_stack_sep_params_t *p, lidar_stack_t **out)
{
    if (!out) return sfail(nullptr, LIDAR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p || !p->col || !p->row) return sfail(nullptr, LIDAR_EINVAL, "params, col or row is NULL");
    double sm = 0;
    lidar_status_t st = check_common(p->kh, p->kw, p->threshold, p->dr, p->r_max, &sm);
    if (st != LIDAR_OK) return st;
    float cmax = 0.f, rmax = 0.f;
    for (int i = 0; i < p->kh; ++i) {
        if (!(std::isfinite(p->col[i]) && p->col[i] >= 0.f))
            return sfail(nullptr, LIDAR_EINVAL, "col[%d] is negative or not finite", i);
        cmax = std::max(cmax, p->col[i]);
    }
    for (int i = 0; i < p->kw; ++i) {
        if (!(std::isfinite(p->row[i]) && p->row[i] >= 0.f))
            return sfail(nullptr, LIDAR_EINVAL, "row[%d] is negative or not finite", i);
        rmax = std::max(rmax, p->row[i]);
    }
    lidar_stack_t *h = new (std::nothrow) lidar_stack();
    if (!h) return sfail(nullptr, LIDAR_ENOMEM, "host allocation failed");
    h->kh = p->kh; h->kw = p->kw; h->s_max = (int)sm; h->dr = p->dr; h->thr = p->threshold;
    h->sep = true;
    h->kmax = (float)((double)cmax * rmax);
    std::vector<float> k(p->col, p->col + p->kh);
    k.insert(k.end(), p->row, p->row + p->kw);
    cudaError_t e;
    if ((e = cudaMalloc(&h->d_K, k.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(h->d_K, k.data(), k.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(stack_sep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sep_smem(p->kh, p->kw))) != cudaSuccess) {
        st = scuda(nullptr, e, "range stacking set-up");
        lidar_stack_destroy(h);
        return st;
    }
    *out = h;
    return LIDAR_OK;
}

const char *lidar_stack_last_error(const lidar_stack_t *h) { return h ? h->err : g_stack_err; }

void lidar_stack_destroy(lidar_stack_t *h)
{
    if (!h) return;
    cudaFree(h->d_K);
    cudaFree(h->d_I);
    cudaFree(h->d_S);
    delete h;
}

}  // extern "C"
