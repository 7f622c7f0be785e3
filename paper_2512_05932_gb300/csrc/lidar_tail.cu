// Kernels of the core/tail split used by the learned tail surrogate.
//
// The profile of a radial beam is split at a core radius theta_c: the core
// (theta <= theta_c) is always deposited exactly by the footprint kernel; the
// tail (theta_c < theta <= truncation) is the blooming part of Sec. II-B's
// centered kernel, whose pixels far outnumber the core's. Its per-beam
// contribution is replaced by a coarse range histogram (a prediction), and a
// beam is re-run exactly when the bounds below cannot guarantee the result.
//
//   tail_mip_kernel   G-buffer cell sums at 4 levels (4, 8, 16, 32 pixels per
//                     side): sum of rho_hat |cos| / R^2 d omega (the deposit
//                     mass of the pixel before the profile weight), the same
//                     weighted by range, ambient * d omega, and the range
//                     extremes. One pass over the planes, then 2x2 reductions.
//   tail_prep_kernel  one warp per beam: walks the tail annulus over a
//                     quadtree of those cells (16-pixel cells, refined to 8 and
//                     4 pixels near the axis) and forms
//                       - E_ub: an upper bound of the tail's deposited mass,
//                         sum over cells of (cell mass) x (profile maximum over
//                         the cell's part of the annulus);
//                       - bounds of the tail's ambient sum, and an estimate;
//                       - the prior: each cell's mass x profile at its pixels,
//                         spread over the cell's range interval, on the coarse
//                         bins;
//                     and gathers the network input: a 4-level pyramid of
//                     64^2 ... 8^2 cells around the axis (FP16, 2 channels:
//                     range and log tail mass).
#include <cuda_fp16.h>

#include <algorithm>
#include <math_constants.h>
#include <stdint.h>

#include "lidar_internal.h"
#include "lidar_tail_internal.h"

namespace gbl {

// ---------------------------------------------------------------------------
// cell sums
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) tail_mip_base_kernel(MipArgs A)
{
    const int L = 2, side = 1 << L;
    const int ncx = A.ncx[0], ncy = A.ncy[0];
    const int n = ncx * ncy;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int cy = c / ncx, cx = c - cy * ncx;
        float sw = 0.f, swr = 0.f, sa = 0.f, rmin = CUDART_INF_F, rmax = -CUDART_INF_F;
        for (int dy = 0; dy < side; ++dy) {
            const int v = cy * side + dy;
            if (v >= A.V) break;
            const float el = A.el0 + ((float)v + 0.5f) * A.del;
            float se, ce;
            sincosf(el, &se, &ce);
            const float domega = 2.f * A.daz * ce * A.sv;
            for (int dx = 0; dx < side; ++dx) {
                const int u = cx * side + dx;
                if (u >= A.U) break;
                const size_t idx = (size_t)v * A.U + u;
                const float Lm = A.amb[idx];
                if (isfinite(Lm)) sa += Lm * domega;
                const float rr = A.range[idx];
                if (isfinite(rr) && rr > 0.f) {
                    const float az = A.az0 + ((float)u + 0.5f) * A.daz;
                    float sa_, ca_;
                    sincosf(az, &sa_, &ca_);
                    const float dn = ce * (ca_ * A.nx[idx] + sa_ * A.ny[idx]) + se * A.nz[idx];
                    const float beta = A.rho[idx] * (1.f / CUDART_PI_F) + A.retro[idx];
                    const float w = beta * fabsf(dn) / (rr * rr) * domega;
                    if (w > 0.f) {
                        sw += w;
                        swr += w * rr;
                        rmin = fminf(rmin, rr);
                        rmax = fmaxf(rmax, rr);
                    }
                }
            }
        }
        A.s[0][c] = make_float4(sw, swr, sa, 0.f);
        A.r[0][c] = make_float2(rmin, rmax);
    }
}

__global__ void __launch_bounds__(256) tail_mip_reduce_kernel(MipArgs A, int lvl)
{
    const int ncx = A.ncx[lvl], ncy = A.ncy[lvl];
    const int px = A.ncx[lvl - 1], py = A.ncy[lvl - 1];
    const float4 *S = A.s[lvl - 1];
    const float2 *R = A.r[lvl - 1];
    const int n = ncx * ncy;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int cy = c / ncx, cx = c - cy * ncx;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 r = make_float2(CUDART_INF_F, -CUDART_INF_F);
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int x = 2 * cx + dx, y = 2 * cy + dy;
                if (x >= px || y >= py) continue;
                const float4 q = S[(size_t)y * px + x];
                const float2 rq = R[(size_t)y * px + x];
                s.x += q.x; s.y += q.y; s.z += q.z;
                r.x = fminf(r.x, rq.x);
                r.y = fmaxf(r.y, rq.y);
            }
        A.s[lvl][c] = s;
        A.r[lvl][c] = r;
    }
}

cudaError_t launch_tail_mips(const MipArgs &a, cudaStream_t s)
{
    for (int l = 0; l < kMipLevels; ++l) {
        const int n = a.ncx[l] * a.ncy[l];
        const int grid = (int)std::min<long>((n + 255) / 256, 152L * 16);
        if (l == 0) tail_mip_base_kernel<<<grid, 256, 0, s>>>(a);
        else tail_mip_reduce_kernel<<<grid, 256, 0, s>>>(a, l);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// per-beam bounds, prior and network input
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2f(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Normalised radial profile at theta^2 (rad^2), as the footprint kernel
// evaluates it (Gaussian + power-law tail); relative error ~1e-6 (hardware
// base-2 exponential and logarithm), covered by the bounds' slack.
__device__ __forceinline__ float tail_profile(const PrepArgs &A, float t2)
{
    if (!(t2 <= A.trunc2)) return 0.f;
    const float x = fmaxf(t2 * A.tc2_inv, 1e-30f);
    const float tl = A.tail_amp * fminf(1.f, ex2f(A.tail_hp * lg2f(x)));
    return A.invZ * (ex2f(t2 * A.kg) + tl);
}

struct CellGeom {
    float th;    // angular distance of the cell centre from the axis (rad)
    float rel;   // bound of the relative error of th
    float rho;   // bound of the distance from the centre to any pixel centre of the cell
    int u0, v0, nu, nv;  // pixel box
};

// Angular distance between the axis and pixel coordinates (x, y) (pixel u's
// centre at x = u). For |dAz| <= 0.1 rad: theta^2 = dEl^2 + cos(el_b) cos(el)
// dAz^2, the haversine formula with sin x = x and asin y = y, whose relative
// error is below max(dEl^2, dAz^2) / 24 + theta^2 / 24 (returned in *rel with
// a 1.5x margin); beyond, the haversine formula itself.
__device__ __forceinline__ float ang_dist(const PrepArgs &A, const BeamParam &P, float x, float y, float *rel)
{
    const float dAz = (x - (float)P.ci - P.cf) * A.daz;
    const float dEl = (y - (float)P.ri - P.rf) * A.del;
    float sEl, cEl;
    if (fabsf(dEl) <= 0.1f) {
        // Taylor series, error below |dEl|^5 / 120 (1e-7)
        const float e2 = dEl * dEl;
        sEl = dEl * fmaf(-e2, 1.f / 6.f, 1.f);
        cEl = fmaf(e2, fmaf(e2, 1.f / 24.f, -0.5f), 1.f);
    } else {
        sincosf(dEl, &sEl, &cEl);
    }
    const float cos_c = fmaxf(0.f, P.cos_elb * cEl - P.sin_elb * sEl);  // cos(el_b + dEl)
    if (fabsf(dAz) <= 0.1f && fabsf(dEl) <= 0.1f) {
        const float t2 = fmaf(dEl, dEl, P.cos_elb * cos_c * dAz * dAz);
        *rel = 1.5f * (fmaxf(dEl * dEl, dAz * dAz) + t2) * (1.f / 24.f) + 2e-6f;
        return sqrtf(t2);
    }
    const float sa = sinf(0.5f * dAz), se = sinf(0.5f * dEl);
    const float hav = se * se + P.cos_elb * cos_c * sa * sa;
    *rel = 2e-6f;
    return 2.f * asinf(fminf(1.f, sqrtf(fmaxf(hav, 0.f))));
}

__device__ __forceinline__ bool cell_geom(const PrepArgs &A, const BeamParam &P, int lvl, int cx, int cy, CellGeom &g)
{
    const int side = 4 << lvl;
    int u0 = cx * side;
    if (cy < 0 || cy * side >= A.V) return false;
    if (A.panorama) {
        // unwrapped column index: pixel coordinates stay continuous around the beam
    } else if (cx < 0 || u0 >= A.U) {
        return false;
    }
    g.u0 = u0;
    g.v0 = cy * side;
    g.nu = A.panorama ? side : min(side, A.U - u0);
    g.nv = min(side, A.V - g.v0);
    const float xc = (float)g.u0 + 0.5f * (float)(g.nu - 1);
    const float yc = (float)g.v0 + 0.5f * (float)(g.nv - 1);
    g.th = ang_dist(A, P, xc, yc, &g.rel);
    const float hx = 0.5f * (float)(g.nu - 1) * A.daz, hy = 0.5f * (float)(g.nv - 1) * A.del;
    g.rho = 1.0001f * sqrtf(hx * hx + hy * hy) + 1e-7f;
    return true;
}

__device__ __forceinline__ int wrap_cell(const PrepArgs &A, int lvl, int cx)
{
    const int n = A.ncx[lvl];
    if (!A.panorama) return cx;
    cx %= n;
    return cx < 0 ? cx + n : cx;
}

// Spreads mass m uniformly over the coarse coordinate interval [a, b] of the
// warp's coarse histogram h (coarse bin c covers [c, c + 1)).
__device__ __forceinline__ void spread(float *h, int nc, float a, float b, float m)
{
    if (!(m > 0.f)) return;
    if (!(b > a + 1e-6f)) {
        const int c = (int)floorf(fminf(fmaxf(a, -1.f), (float)nc + 1.f));
        if (c >= 0 && c < nc) atomicAdd(h + c, m);
        return;
    }
    const float inv = m / (b - a);  // the part outside the window is dropped
    a = fminf(fmaxf(a, -1.f), (float)nc + 1.f);
    b = fminf(fmaxf(b, -1.f), (float)nc + 1.f);
    int c0 = max(0, (int)floorf(a)), c1 = min(nc - 1, (int)floorf(b));
    for (int c = c0; c <= c1; ++c) {
        const float lo = fmaxf(a, (float)c), hi = fminf(b, (float)(c + 1));
        if (hi > lo) atomicAdd(h + c, (hi - lo) * inv);
    }
}

struct PrepAcc {
    float eub, ahi, alo, aest;
};

// Estimate part of a leaf: the cell's ambient and mass times the mean profile
// pm over its pixels, the mass spread over the cell's range interval.
__device__ __forceinline__ void prep_estimate(const PrepArgs &A, int lvl, size_t ci, const float4 &s, float pm,
                                              float *hc, PrepAcc &acc)
{
    if (!(pm > 0.f)) return;
    acc.aest += s.z * pm;
    if (s.x > 0.f) {
        const float2 r = A.r[lvl][ci];
        const float a = fmaf(r.x, A.x_scale, A.x_off + 0.5f) * A.inv_cf;
        const float b = fmaf(r.y, A.x_scale, A.x_off + 0.5f) * A.inv_cf;
        spread(hc, A.n_coarse, a, b, s.x * pm);
    }
}

__device__ __forceinline__ size_t cell_index(const PrepArgs &A, int lvl, int cxw, const CellGeom &g)
{
    return (size_t)(g.v0 >> (2 + lvl)) * A.ncx[lvl] + cxw;
}

// Mean of the annulus profile over the pixel centres of a cell (one thread).
__device__ __forceinline__ float pixel_mean_profile(const PrepArgs &A, const BeamParam &P, const CellGeom &g)
{
    float acc_p = 0.f;
    for (int dy = 0; dy < g.nv; ++dy)
        for (int dx = 0; dx < g.nu; ++dx) {
            float r_;
            const float th = ang_dist(A, P, (float)(g.u0 + dx), (float)(g.v0 + dy), &r_);
            if (th > A.core) acc_p += tail_profile(A, th * th);
        }
    return acc_p / (float)(g.nu * g.nv);
}

// One leaf cell of the quadtree: bounds, ambient estimate and prior. The
// estimate takes the profile at the cell centre, except in 4-pixel cells that
// cross the core or truncation radius, where it is the mean over the cell's
// pixels (zero outside the annulus): with defer, such a cell returns true and
// its estimate is left to the caller (evaluated pixel-parallel by the warp).
__device__ __forceinline__ bool prep_leaf(const PrepArgs &A, const BeamParam &P, int lvl, int cxw, const CellGeom &g,
                                          float *hc, PrepAcc &acc, bool defer)
{
    const size_t ci = cell_index(A, lvl, cxw, g);
    const float4 s = A.s[lvl][ci];
    if (!(s.x > 0.f) && !(s.z > 0.f)) return false;
    const float tmin = fmaxf(0.f, g.th * (1.f - g.rel) - g.rho), tmax = g.th * (1.f + g.rel) + g.rho;
    if (!(tmax * (1.f + 1e-5f) > A.core) || !(tmin <= A.trunc * (1.f + 1e-5f))) return false;
    const float tb = fmaxf(tmin, A.core * (1.f - 1e-5f));
    const float pmax = tail_profile(A, tb * tb) * (1.f + 1e-4f);
    acc.eub += s.x * pmax;
    acc.ahi += s.z * pmax;
    if (tmin > A.core * (1.f + 1e-5f) && tmax < A.trunc * (1.f - 1e-5f)) acc.alo += s.z * tail_profile(A, tmax * tmax) * (1.f - 1e-4f);
    float pm;
    if (lvl == 0 && (tmin < A.core || tmax > A.trunc)) {
        if (defer) return true;
        pm = pixel_mean_profile(A, P, g);
    } else {
        pm = (g.th > A.core) ? tail_profile(A, g.th * g.th) : 0.f;
    }
    prep_estimate(A, lvl, ci, s, pm, hc, acc);
    return false;
}

__global__ void __launch_bounds__(kPrepThreads) tail_prep_kernel(PrepArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int beam = blockIdx.x * kPrepWarps + warp;
    float *hc = reinterpret_cast<float *>(smem) + (size_t)warp * A.n_coarse;
    int *list = reinterpret_cast<int *>(smem + (size_t)kPrepWarps * A.n_coarse * 4) + (size_t)warp * 2 * kPrepList;
    int *l3 = list, *l2 = list + kPrepList;
    __shared__ int n3s[kPrepWarps], n2s[kPrepWarps];
    if (beam >= A.n_beams) return;  // warp-uniform: no block barrier follows
    const BeamParam P = A.beams[beam];
    for (int c = lane; c < A.n_coarse; c += 32) hc[c] = 0.f;
    if (lane == 0) { n3s[warp] = 0; n2s[warp] = 0; }
    __syncwarp();
    PrepAcc acc{0.f, 0.f, 0.f, 0.f};
    // bounding box of the support (radius trunc + the largest cell radius) in 32-pixel cells
    const float R = A.trunc + A.rho_top;
    const float bx = (float)P.ci + P.cf + 0.5f, by = (float)P.ri + P.rf + 0.5f;  // continuous pixel position
    const int side = 4 << (kQuadLevels - 1);
    const float elb = asinf(fmaxf(-1.f, fminf(1.f, P.sin_elb)));
    const bool polar = fabsf(elb) + R >= 0.5f * CUDART_PI_F - 1e-6f;
    const float dl = polar ? CUDART_PI_F : asinf(fminf(1.f, sinf(R) / P.cos_elb));
    int cx0 = (int)floorf((bx - dl / A.daz) / side), cx1 = (int)floorf((bx + dl / A.daz) / side);
    int cy0 = (int)floorf((by - R / A.del) / side), cy1 = (int)floorf((by + R / A.del) / side);
    if (A.panorama && (cx1 - cx0 + 1) * side >= A.U) { cx0 = (int)floorf(bx / side) - A.ncx[kQuadLevels - 1] / 2; cx1 = cx0 + A.ncx[kQuadLevels - 1] - 1; }
    const int nx = cx1 - cx0 + 1, ny = cy1 - cy0 + 1;
    // top level: leaf or refine
    for (int i = lane; i < nx * ny; i += 32) {
        const int cy = cy0 + i / nx, cx = cx0 + i % nx;
        const int lvl = kQuadLevels - 1;
        CellGeom g;
        if (!cell_geom(A, P, lvl, cx, cy, g)) continue;
        if (g.th * (1.f - g.rel) - g.rho > A.trunc * (1.f + 1e-5f) ||
            g.th * (1.f + g.rel) + g.rho < A.core * (1.f - 1e-5f))
            continue;
        if (g.th - g.rho < A.refine[lvl]) {
            int k = atomicAdd(n3s + warp, 4);
            if (k + 4 <= kPrepList) {
                for (int q = 0; q < 4; ++q) l3[k + q] = ((2 * cy + (q >> 1)) << 16) ^ ((2 * cx + (q & 1)) & 0xFFFF);
                continue;
            }
        }
        prep_leaf(A, P, lvl, wrap_cell(A, lvl, cx), g, hc, acc, false);
    }
    __syncwarp();
    const int n3 = min(n3s[warp], kPrepList);
    for (int i = lane; i < n3; i += 32) {
        const int lvl = kQuadLevels - 2;
        const int cy = l3[i] >> 16, cx = (int)(short)(l3[i] & 0xFFFF);
        CellGeom g;
        if (!cell_geom(A, P, lvl, cx, cy, g)) continue;
        if (g.th * (1.f - g.rel) - g.rho > A.trunc * (1.f + 1e-5f) ||
            g.th * (1.f + g.rel) + g.rho < A.core * (1.f - 1e-5f))
            continue;
        if (g.th - g.rho < A.refine[lvl]) {
            int k = atomicAdd(n2s + warp, 4);
            if (k + 4 <= kPrepList) {
                for (int q = 0; q < 4; ++q) l2[k + q] = ((2 * cy + (q >> 1)) << 16) ^ ((2 * cx + (q & 1)) & 0xFFFF);
                continue;
            }
        }
        prep_leaf(A, P, lvl, wrap_cell(A, lvl, cx), g, hc, acc, false);
    }
    __syncwarp();
    const int n2 = min(n2s[warp], kPrepList);
    // 4-pixel cells; those crossing the core or truncation radius are listed
    // (in l3, free now) and their pixel-level estimate done below
    if (lane == 0) n3s[warp] = 0;
    __syncwarp();
    for (int i = lane; i < n2; i += 32) {
        const int lvl = 0;
        const int cy = l2[i] >> 16, cx = (int)(short)(l2[i] & 0xFFFF);
        CellGeom g;
        if (!cell_geom(A, P, lvl, cx, cy, g)) continue;
        if (prep_leaf(A, P, lvl, wrap_cell(A, lvl, cx), g, hc, acc, true)) {
            const int k = atomicAdd(n3s + warp, 1);
            if (k < kPrepList) {
                l3[k] = l2[i];
            } else {
                const size_t ci = cell_index(A, lvl, wrap_cell(A, lvl, cx), g);
                prep_estimate(A, lvl, ci, A.s[lvl][ci], pixel_mean_profile(A, P, g), hc, acc);
            }
        }
    }
    __syncwarp();
    // pixel-level estimate of the listed cells: half-warp per cell, one lane per pixel
    const int ns = min(n3s[warp], kPrepList);
    for (int base = 0; base < 16 * ns; base += 32) {
        const int i = base + lane, cell = i >> 4, pix = i & 15;
        float p = 0.f;
        CellGeom g;
        int cx = 0;
        bool ok = false;
        if (cell < ns) {
            const int cy = l3[cell] >> 16;
            cx = (int)(short)(l3[cell] & 0xFFFF);
            ok = cell_geom(A, P, 0, cx, cy, g);
            if (ok && (pix & 3) < g.nu && (pix >> 2) < g.nv) {
                float r_;
                const float th = ang_dist(A, P, (float)(g.u0 + (pix & 3)), (float)(g.v0 + (pix >> 2)), &r_);
                if (th > A.core) p = tail_profile(A, th * th);
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (ok && pix == 0) {
            const int cxw = wrap_cell(A, 0, cx);
            const size_t ci = cell_index(A, 0, cxw, g);
            prep_estimate(A, 0, ci, A.s[0][ci], p / (float)(g.nu * g.nv), hc, acc);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.eub += __shfl_xor_sync(0xffffffffu, acc.eub, o);
        acc.ahi += __shfl_xor_sync(0xffffffffu, acc.ahi, o);
        acc.alo += __shfl_xor_sync(0xffffffffu, acc.alo, o);
        acc.aest += __shfl_xor_sync(0xffffffffu, acc.aest, o);
    }
    __syncwarp();
    float *row = A.prior + (size_t)beam * (A.n_coarse + 4);
    float mass = 0.f;
    for (int c = lane; c < A.n_coarse; c += 32) {
        const float v = hc[c];
        row[c] = v;
        mass += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mass += __shfl_xor_sync(0xffffffffu, mass, o);
    if (lane == 0) {
        // the estimate lies in [alo, ahi]; its error is at most the larger distance
        const float aest = fminf(fmaxf(acc.aest, acc.alo), acc.ahi);
        row[A.n_coarse] = aest;
        row[A.n_coarse + 1] = fmaxf(acc.eub * 1.001f, mass);
        row[A.n_coarse + 2] = 1.001f * fmaxf(acc.ahi - aest, aest - acc.alo);
        row[A.n_coarse + 3] = mass;
    }
    if (!A.inputs) return;
    // network input: level l is a (64 >> l)^2 patch of the (4 << l)-pixel
    // cells around the axis; channel 0 = mass-weighted mean range as a
    // fraction of the waveform window (-1: no return), channel 1 = log2 of the
    // cell's mass x the profile at the core edge relative to the prior's mass,
    // scaled to about [0, 1]
    __half2 *out = reinterpret_cast<__half2 *>(A.inputs) + (size_t)beam * kNetInCells;
    const float rel = tail_profile(A, A.core * A.core) / (mass > 0.f ? mass : 1.f);
    int base = 0;
    for (int l = 0; l < kMipLevels; ++l) {
        const int S = 64 >> l, sidel = 4 << l;
        const int ccx = (int)floorf(bx / sidel) - S / 2, ccy = (int)floorf(by / sidel) - S / 2;
        for (int i = lane; i < S * S; i += 32) {
            const int cy = ccy + i / S, cx = ccx + i % S;
            float c0 = -1.f, c1 = 0.f;
            const bool in = cy >= 0 && cy < A.ncy[l] && (A.panorama || (cx >= 0 && cx < A.ncx[l]));
            if (in) {
                const float4 q = A.s[l][(size_t)cy * A.ncx[l] + wrap_cell(A, l, cx)];
                if (q.x > 0.f) {
                    c0 = fminf(2.f, fmaxf(-1.f, fmaf(q.y / q.x, A.x_scale, A.x_off) * A.inv_nb));
                    c1 = fminf(1.5f, fmaxf(0.f, lg2f(q.x * rel + 1e-12f) * (1.f / 40.f) + 1.f));
                }
            }
            out[base + i] = __floats2half2_rn(c0, c1);
        }
        base += S * S;
    }
}

cudaError_t launch_tail_prep(const PrepArgs &a, cudaStream_t s)
{
    const size_t smem = (size_t)kPrepWarps * (a.n_coarse * 4 + 2 * kPrepList * 4);
    const int smem_max = kPrepWarps * (1024 * 4 + 2 * kPrepList * 4);  // n_coarse <= 1024
    cudaError_t e = cudaFuncSetAttribute(tail_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return e;
    const int grid = (a.n_beams + kPrepWarps - 1) / kPrepWarps;
    tail_prep_kernel<<<grid, kPrepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ordered compaction of the re-run flags (one CTA; beams keep their order, so
// that neighbouring beams share a CTA of the re-run pass)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) compact_kernel(const uint8_t *flags, int n, int *out)
{
    __shared__ int wsum[32];
    __shared__ int base_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int i = c0 + tid;
        const int f = (i < n && flags[i]) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int v = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            wsum[lane] = v;  // inclusive
        }
        __syncthreads();
        const int base = base_s;
        const int off = base + (warp > 0 ? wsum[warp - 1] : 0) + pre;
        if (f) out[1 + off] = i;
        __syncthreads();
        if (tid == 0) base_s = base + wsum[31];
        __syncthreads();
    }
    if (tid == 0) out[0] = base_s;
}

cudaError_t launch_compact(const uint8_t *flags, int n, int *out, cudaStream_t s)
{
    compact_kernel<<<1, 1024, 0, s>>>(flags, n, out);
    return cudaGetLastError();
}

}  // namespace gbl
