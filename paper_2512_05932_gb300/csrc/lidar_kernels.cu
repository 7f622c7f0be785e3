// sm_103a kernels of the beam model (Alg. 1 beam iteration with the EPW
// post-processing of Sec. II-C).
//
//   setup_kernel      one launch, two roles:
//                     - per pixel: rho_hat * d omega, the time-of-flight
//                       interval from the plane extrapolation of Sec. II-D
//                       (pixelRangeInterval of Alg. 1), ambient * d omega, and
//                       the pixel's deposit plan -> one 32-byte record: the
//                       weights of the hat functions it touches (up to four
//                       consecutive bins for a narrow interval; two partial
//                       bins at each end and a constant run between them for a
//                       wide one) with their histogram positions or bin indices;
//                     - per beam (FP64): pose-rotated axis, its pixel-grid
//                       coordinates, the local frame's roll and the candidate
//                       pixel box.
//   footprint_wave_kernel  one CTA per group of G consecutive beams:
//                     - profile weight (Eq. centered kernel) for every
//                       (beam, pixel) pair of the group's box, times the
//                       record's hat weights added straight into the beam's
//                       histogram in shared memory (no difference arrays or
//                       prefix sums: those cancel in FP32 after strong echoes);
//                     - pulse convolution varpi * xi_b + ambient (Sec. II-C)
//                       over the histogram's support only;
//                     - echo intervals, EPW, peak and intensity.
#include <cuda_bf16.h>
#include <climits>
#include <math_constants.h>
#include <stdint.h>

#include "lidar_internal.h"

namespace gbl {

// --------------------------------------------------------------------------
// setup: per-pixel records
// --------------------------------------------------------------------------

__device__ __forceinline__ float hatf(float x) { return fmaxf(0.f, 1.f - fabsf(x)); }

// Position of padded bin index x in the footprint kernel's histogram buffer:
// one unused slot after every 32, so that lanes 8 bins apart hit distinct banks.
__host__ __device__ __forceinline__ int skew_pos(int x) { return x + (x >> 5); }

// Integral of hat(x - k) over [X0, X1] (bin-centre units; the mean times
// X1 - X0): the interval is cut at the kinks k-1, k, k+1; on each piece the
// hat is linear, so the piece's contribution is its length times the hat at
// its midpoint. The caller divides by X1 - X0 once for all bins (a point
// interval, X1 = X0, gives the hat at X0 and no division).
__device__ float int_hat(float X0, float X1, float k)
{
    if (!(X1 - X0 > 0.f)) return hatf(X0 - k);
    float lo = X0, acc = 0.f;
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
        float cut = k + (float)c;
        if (cut > lo && cut < X1) {
            acc += (cut - lo) * hatf(0.5f * (lo + cut) - k);
            lo = cut;
        }
    }
    acc += (X1 - lo) * hatf(0.5f * (lo + X1) - k);
    return acc;
}

// Returns the largest deposit weight the pixel's record holds (0 without one).
__device__ float setup_pixel(const SetupArgs &A, int idx)
{
    int v = idx / A.U;
    int u = idx - v * A.U;
    float az = A.az0 + ((float)u + 0.5f) * A.daz;
    float el = A.el0 + ((float)v + 0.5f) * A.del;
    float sa, ca, se, ce;
    sincosf(az, &sa, &ca);
    sincosf(el, &se, &ce);
    // exact solid angle of the cell: daz (sin(el + del/2) - sin(el - del/2))
    float domega = 2.f * A.daz * ce * A.sv;
    // all seven planes are loaded up front, so that their latencies overlap
    // (a sky pixel reads five values it does not use)
    float L = A.amb[idx];
    float a = isfinite(L) ? L * domega : 0.f;
    float rr = A.range[idx];
    const float nx = A.nx[idx], ny = A.ny[idx], nz = A.nz[idx];
    const float rho = A.rho[idx], retro = A.retro[idx];
    uint32_t kab = kNoDeposit, kq = kNoDeposit;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, cr = 0.f;
    if (isfinite(rr) && rr > 0.f) {
        float dn = ce * (ca * nx + sa * ny) + se * nz;
        float beta = rho * (1.f / CUDART_PI_F) + retro;
        // rho_hat d omega = beta |cos theta_i| / R^2 * d omega
        float w = beta * fabsf(dn) / (rr * rr) * domega;
        // range interval: plane through the hit point, extrapolated to the four
        // corner rays (r_c = r * (d.n) / (d_c.n)), normal facing the sensor.
        // Positions are kept in bin coordinates relative to an integer base, so
        // that a 2048-bin window keeps ~1e-7 bins of precision instead of the
        // ~1e-4 of an absolute FP32 coordinate:
        //   - the centre X = r x_scale + x_off as base + fraction, from an
        //     exact two-product (x_scale = xs_hi + xs_lo, x_off = xo_int + xo_fr);
        //   - each corner as X_c - X = r x_scale (mu_p - mu_c) / mu_c, with
        //     mu_p - mu_c = sgn n.(d_c - d) and d_c - d formed from small terms
        //     (1 - cos, sin of half a pixel), not as a difference of cosines.
        float sgn = dn > 0.f ? -1.f : 1.f;
        float mup = fmaxf(-sgn * dn, kMuMin);
        const float p = rr * A.xs_hi;
        const float pe = fmaf(rr, A.xs_hi, -p);
        const float pf = floorf(p);
        const float xc = (p - pf) + (pe + fmaf(rr, A.xs_lo, A.xo_fr));
        const float base = pf + A.xo_int;
        const float K = rr * A.xs_hi;
        float dlo, dhi;  // interval ends relative to X (bins)
        float mu_lo = INFINITY, mu_hi = 0.f, df_lo = 0.f, df_hi = 0.f;
        // n.(d_c - d) = ce Ph + dce Qh + nz dse: Ph, Qh depend on the corner's
        // azimuth side ci, dce = cos(el_c) - cos(el), dse = sin(el_c) - sin(el)
        // on its elevation side cj
        const float mu0 = -sgn * dn;
        const float nh = fmaf(nx, ca, ny * sa);
#pragma unroll
        for (int ci = -1; ci <= 1; ci += 2) {
            const float dca = fmaf(-ca, A.vh, -(float)ci * sa * A.sh);  // cos(az_c) - cos(az)
            const float dsa = fmaf(-sa, A.vh, (float)ci * ca * A.sh);   // sin(az_c) - sin(az)
            const float Ph = fmaf(nx, dca, ny * dsa);
            const float Qh = nh + Ph;
#pragma unroll
            for (int cj = -1; cj <= 1; cj += 2) {
                const float dce = fmaf(-ce, A.vv, -(float)cj * se * A.sv);
                const float dse = fmaf(-se, A.vv, (float)cj * ce * A.sv);
                const float ndd = fmaf(ce, Ph, fmaf(dce, Qh, nz * dse));
                const float mu_raw = fmaf(-sgn, ndd, mu0);
                const float mu = fmaxf(mu_raw, kMuMin);
                // mu_p - mu_c, in the exact form unless a clamp is active
                const float diff = (mu_raw >= kMuMin && mu0 >= kMuMin) ? sgn * ndd : mup - mu;
                // X_c - X = K (mu_p / mu_c - 1) decreases with mu_c: the
                // extremes come from the extreme denominators (two divisions)
                if (mu > mu_hi) { mu_hi = mu; df_hi = diff; }
                if (mu < mu_lo) { mu_lo = mu; df_lo = diff; }
            }
        }
        dlo = fminf(0.f, K * df_hi / mu_hi);
        dhi = fmaxf(0.f, K * df_lo / mu_lo);
        const float x0 = xc + dlo, x1 = xc + dhi;
        const float fl = floorf(x0);
        const float f = base + fl;           // first bin touched (integer)
        const float l0 = x0 - fl, l1 = x1 - fl;  // interval in bins relative to f
        const float nb = (float)A.n_bins;
        // the hat functions of bins 0..n-1 cover (-1, n): anything else is dropped
        if (w > 0.f && f + l1 > -1.f && f + l0 < nb) {
            // w times the mean of a hat over [l0, l1] = (w / (l1 - l0)) times its integral
            const float ww = l1 - l0 > 0.f ? w / (l1 - l0) : w;
            if (l1 <= 3.f) {
                // narrow: at most 4 bins f..f+3 touched; the record holds their
                // positions in the footprint kernel's skewed histogram buffer
                if (f >= -3.f) {
                    h0 = ww * int_hat(l0, l1, 0.f);
                    h1 = ww * int_hat(l0, l1, 1.f);
                    h2 = ww * int_hat(l0, l1, 2.f);
                    h3 = ww * int_hat(l0, l1, 3.f);
                    if (A.bin_records) {
                        // tensor-core deposit: the bin index itself
                        kab = (uint32_t)((int)f + kBinBias) | (0xFFFFu << 16);
                        kq = 0u;
                    } else {
                        int x = (int)f + A.pad;
                        kab = (uint32_t)skew_pos(x) | ((uint32_t)skew_pos(x + 1) << 16);
                        kq = (uint32_t)skew_pos(x + 2) | ((uint32_t)skew_pos(x + 3) << 16);
                    }
                }
            } else {
                // wide (l1 - l0 > 2): partial bins f, f+1 and g, g+1, every bin
                // in between fully covered with weight w / (l1 - l0)
                const float gl = floorf(l1);
                float g = f + gl;
                float ff = f;
                h0 = ww * int_hat(l0, l1, 0.f);
                h1 = ww * int_hat(l0, l1, 1.f);
                h2 = ww * int_hat(l0, l1, gl);
                h3 = ww * int_hat(l0, l1, gl + 1.f);
                cr = ww;
                // bins far outside the window: zero weight, parked next to it
                // (the run between them keeps its extent)
                if (ff < -4.f) { ff = -4.f; h0 = 0.f; h1 = 0.f; }
                if (g > nb + 2.f) { g = nb + 2.f; h2 = 0.f; h3 = 0.f; }
                kab = (uint32_t)((int)ff + kBinBias) | ((uint32_t)((int)g + kBinBias) << 16);
            }
        }
    }
    float4 r0 = make_float4(__uint_as_float(kab), a, h0, h1);
    float4 r1 = make_float4(__uint_as_float(kq), h2, h3, cr);
    A.rec[2 * (size_t)idx] = r0;
    A.rec[2 * (size_t)idx + 1] = r1;
    return fmaxf(fmaxf(fmaxf(h0, h1), fmaxf(h2, h3)), cr);
}

// Adds a thread's largest record weight to the frame's maximum (FP32 bits
// of a non-negative value order as unsigned integers): one atomic per warp.
__device__ __forceinline__ void wmax_reduce(unsigned *wmax, float m)
{
    const unsigned mask = __activemask();
    const unsigned v = __reduce_max_sync(mask, __float_as_uint(fmaxf(m, 0.f)));
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && v) atomicMax(wmax, v);
}

// --------------------------------------------------------------------------
// setup: per-beam parameters (FP64)
// --------------------------------------------------------------------------

// Not inlined: its FP64 work needs more registers than the per-pixel path, and
// inlined it would set the register count (and so the occupancy) of the whole
// setup kernel; as a call it spills inside itself instead.
__device__ __noinline__ void setup_beam(const SetupArgs &A, int b)
{
    const int src = A.beam_ids ? A.beam_ids[b] : b;
    double d[3] = {A.dirs[3 * src], A.dirs[3 * src + 1], A.dirs[3 * src + 2]};
    double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= nd; d[1] /= nd; d[2] /= nd;
    double e1[3] = {-d[1], d[0], 0.0};
    double ne = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    if (ne < 1e-12) { e1[0] = 0.0; e1[1] = 1.0; ne = 1.0; }
    e1[0] /= ne; e1[1] /= ne;
    double a[3], E1[3];
    for (int r = 0; r < 3; ++r) {
        a[r] = A.R[3 * r] * d[0] + A.R[3 * r + 1] * d[1] + A.R[3 * r + 2] * d[2];
        E1[r] = A.R[3 * r] * e1[0] + A.R[3 * r + 1] * e1[1] + A.R[3 * r + 2] * e1[2];
    }
    double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= na; a[1] /= na; a[2] /= na;
    double el_b = asin(fmin(1.0, fmax(-1.0, a[2])));
    double az_b = atan2(a[1], a[0]);
    const double two_pi = 2.0 * CUDART_PI;
    if (A.panorama) {
        while (az_b < A.az0d) az_b += two_pi;
        while (az_b >= A.az0d + two_pi) az_b -= two_pi;
    } else {
        // the representative within pi of the G-buffer's centre: its azimuth
        // range may cross the +-pi seam of atan2
        const double azc = A.az0d + 0.5 * (double)A.U * A.dazd;
        while (az_b < azc - CUDART_PI) az_b += two_pi;
        while (az_b >= azc + CUDART_PI) az_b -= two_pi;
    }
    double sab, cab, seb, ceb;
    sincos(az_b, &sab, &cab);
    sincos(el_b, &seb, &ceb);
    // east/north frame of the axis in the G-buffer frame
    double g1[3] = {-sab, cab, 0.0};
    double g2[3] = {-seb * cab, -seb * sab, ceb};
    double cg = E1[0] * g1[0] + E1[1] * g1[1] + E1[2] * g1[2];
    double sg = E1[0] * g2[0] + E1[1] * g2[1] + E1[2] * g2[2];
    double ng = sqrt(cg * cg + sg * sg);
    if (ng > 0) { cg /= ng; sg /= ng; } else { cg = 1.0; sg = 0.0; }
    double ua = (az_b - A.az0d) / A.dazd - 0.5;
    double va = (el_b - A.el0d) / A.deld - 0.5;
    BeamParam P;
    P.ci = (int)floor(ua);
    P.cf = (float)(ua - floor(ua));
    P.ri = (int)floor(va);
    P.rf = (float)(va - floor(va));
    P.sin_elb = (float)seb;
    P.cos_elb = (float)ceb;
    P.cg = (float)cg;
    P.sg = (float)sg;
    const int core = A.core_only ? (int)A.core_only[src] : 0;
    double th = core ? A.core_rad : A.support_rad;
    long r0 = (long)ceil((el_b - th - A.el0d) / A.deld - 0.5) - 1;
    long r1 = (long)floor((el_b + th - A.el0d) / A.deld - 0.5) + 1;
    // A table or separable profile is zero outside the rectangle |u| <= hu,
    // |v| <= hv, where every direction d has |d.E1| <= hu and |d.E2| <= hv
    // (d.E1 = sin(theta) cos(phi) <= u): with d = cos(theta) a + (d.E1) E1 +
    // (d.E2) E2 and theta <= th, its height d_z and its east component
    // d.g1 = cos(el) sin(az - az_b) are bounded by the same sums, which gives
    // a box of about half the circle's when the rectangle is a square. FP32
    // suffices: its errors (~1e-7 rad) are far below the one-pixel margin the
    // box keeps on each side.
    double dl_rect = -1.0;
    if (!core && A.sup_u > 0.0) {
        const float ax = (float)a[0], ay = (float)a[1], az = (float)a[2];
        const float e1x = (float)E1[0], e1y = (float)E1[1], e1z = (float)E1[2];
        const float e2x = ay * e1z - az * e1y, e2y = az * e1x - ax * e1z, e2z = ax * e1y - ay * e1x;
        const float su = (float)A.sup_u, sv = (float)A.sup_v;
        const float zc = az * (float)A.cos_sup;
        const float zs = su * fabsf(e1z) + sv * fabsf(e2z);
        const float el_lo = asinf(fmaxf(-1.f, fminf(az, zc) - zs));
        const float el_hi = asinf(fminf(1.f, fmaxf(az, zc) + zs));
        const long q0 = (long)ceil(((double)el_lo - A.el0d) / A.deld - 0.5) - 1;
        const long q1 = (long)floor(((double)el_hi - A.el0d) / A.deld - 0.5) + 1;
        if (q0 > r0) r0 = q0;
        if (q1 < r1) r1 = q1;
        const float g1x = (float)g1[0], g1y = (float)g1[1];
        const float S = su * fabsf(e1x * g1x + e1y * g1y) + sv * fabsf(e2x * g1x + e2y * g1y);
        const float cmin = fminf(cosf(el_lo), cosf(el_hi));
        if (cmin > 0.f && S < cmin) dl_rect = (double)asinf(S / cmin);
    }
    if (r0 < 0) r0 = 0;
    if (r1 > A.V - 1) r1 = A.V - 1;
    long c0, c1;
    bool full = fabs(el_b) + th >= 0.5 * CUDART_PI - 1e-9;
    if (!full) {
        double dl = asin(fmin(1.0, sin(th) / ceb));
        if (dl_rect >= 0.0 && dl_rect < dl) dl = dl_rect;
        c0 = (long)ceil((az_b - dl - A.az0d) / A.dazd - 0.5) - 1;
        c1 = (long)floor((az_b + dl - A.az0d) / A.dazd - 0.5) + 1;
        if (A.panorama && c1 - c0 + 1 >= A.U) full = true;
    }
    if (full) {
        if (A.panorama) { c0 = P.ci - A.U / 2; c1 = c0 + A.U - 1; }
        else { c0 = 0; c1 = A.U - 1; }
    }
    if (!A.panorama) {
        if (c0 < 0) c0 = 0;
        if (c1 > A.U - 1) c1 = A.U - 1;
    }
    P.row0 = (int)r0; P.row1 = (int)r1;
    P.col0 = (int)c0; P.col1 = (int)c1;
    P.valid = (r0 <= r1 && c0 <= c1) ? 1 : 0;
    P.pad0 = core; P.pad1 = 0.f; P.pad2 = 0.f;
    A.beams[b] = P;
}

// Blocks [0, gridDim.x - pix_blocks) set up the beams, the rest the pixels: the
// beams' FP64 blocks start first and run beside the pixel blocks instead of
// trailing them. Six blocks per SM (40 registers) for the memory-latency-bound
// pixel path.
__global__ void __launch_bounds__(256, 6) setup_kernel(SetupArgs A)
{
    const int beam_blocks = (int)gridDim.x - A.pix_blocks;
    if ((int)blockIdx.x < beam_blocks) {
        int b = blockIdx.x * blockDim.x + threadIdx.x;
        if (b < A.n_beams) setup_beam(A, b);
    } else {
        const int n = (int)A.pix_end;
        float m = 0.f;
        for (int idx = (int)A.pix_begin + ((int)blockIdx.x - beam_blocks) * blockDim.x + threadIdx.x; idx < n;
             idx += A.pix_blocks * blockDim.x)
            m = fmaxf(m, setup_pixel(A, idx));
        if (A.wmax) wmax_reduce(A.wmax, m);
    }
}

// Batched setup: frame f owns pixel blocks [pix_blk[f], pix_blk[f+1]) and beam
// blocks [beam_blk[f], beam_blk[f+1]) (pixel blocks first). Block 0 also resets
// the work counter of the batched footprint kernel that follows on the stream.
__global__ void __launch_bounds__(256, 6) setup_batch_kernel(const SetupArgs *frames, const int *pix_blk,
                                                          const int *beam_blk, int n_frames, int *counter)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    const int b = blockIdx.x;
    const int total_pix_blk = pix_blk[n_frames];
    if (b < total_pix_blk) {
        int lo = 0, hi = n_frames - 1;  // last f with pix_blk[f] <= b
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (pix_blk[mid] <= b) lo = mid; else hi = mid - 1;
        }
        const SetupArgs &A = frames[lo];
        int idx = (b - pix_blk[lo]) * blockDim.x + threadIdx.x;
        const float m = idx < A.U * A.V ? setup_pixel(A, idx) : 0.f;
        if (A.wmax) wmax_reduce(A.wmax, m);
    } else {
        const int bb = b - total_pix_blk;
        int lo = 0, hi = n_frames - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (beam_blk[mid] <= bb) lo = mid; else hi = mid - 1;
        }
        const SetupArgs &A = frames[lo];
        int beam = (bb - beam_blk[lo]) * blockDim.x + threadIdx.x;
        if (beam < A.n_beams) setup_beam(A, beam);
    }
}

cudaError_t launch_setup_batch(const SetupArgs *frames, const int *pix_blk, const int *beam_blk, int n_frames,
                               int total_blocks, int *counter, cudaStream_t s)
{
    setup_batch_kernel<<<total_blocks, 256, 0, s>>>(frames, pix_blk, beam_blk, n_frames, counter);
    return cudaGetLastError();
}

cudaError_t launch_setup(const SetupArgs &a, cudaStream_t s)
{
    int beam_blocks = (a.n_beams + 255) / 256;
    setup_kernel<<<a.pix_blocks + beam_blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// footprint + waveform + echoes
// --------------------------------------------------------------------------

constexpr int kSeg = 64;     // columns per work unit (one row)
constexpr int kSegLean = 256; // columns per work unit of the lean phase 1 (longer units: fewer per-row set-ups)
constexpr int kBlk = 256;    // waveform bins per convolution work item (8 per lane)

// Per-beam histogram buffer: bins [-pad, n_bins + pad) at positions
// x = bin + pad, stored at x + (x >> 5) so that lanes reading bins 8 apart hit
// distinct banks. pad >= M + 16 and is a multiple of 32.
constexpr int kTC = 257;     // columns per offset-table stripe (odd: conflict-free float2 rows)
constexpr int kRT = 256;     // rows of the per-(beam, row) elevation table; taller boxes compute on the fly

struct Layout {
    int pad;       // zero padding on each side, in bins
    int HB;        // floats per beam buffer (odd)
    int taps_off;  // tap m lives at index taps_off + m
    int taps_len;
    size_t off_taps, off_amb, off_nrm, off_tmass, off_supp, off_tsupp, off_tab, off_rtab, off_ctab, off_ctr, off_bp, total;
};


__host__ __device__ inline Layout make_layout(int G, int n_bins, int M)
{
    Layout L;
    L.pad = 32 * ((M + 16 + 31) / 32);
    int span = n_bins + 2 * L.pad;
    L.HB = skew_pos(span) + 1;
    if ((L.HB & 1) == 0) L.HB += 1;
    L.taps_off = M + 8;
    L.taps_len = 2 * M + 17;
    size_t off = (size_t)G * L.HB * 4;
    L.off_taps = off; off += (size_t)(skew_pos(L.taps_len) + 1) * 4;  // stored at skew_pos(index)
    L.off_amb = off; off += (size_t)G * 4;
    L.off_nrm = off; off += (size_t)G * 4;
    L.off_tmass = off; off += (size_t)G * 4;
    L.off_supp = off; off += (size_t)G * 8;
    L.off_tsupp = off; off += (size_t)G * 8;
    off = (off + 15) & ~(size_t)15;
    L.off_tab = off; off += (size_t)G * kTC * sizeof(float2);
    L.off_rtab = off; off += (size_t)G * kRT * sizeof(float2);
    L.off_ctab = off; off += (size_t)kRT * sizeof(float);
    L.off_ctr = off; off += 16;
    off = (off + 15) & ~(size_t)15;
    L.off_bp = off; off += (size_t)G * sizeof(BeamParam);
    L.total = off;
    return L;
}

// Profile weight of a local offset (x, y) = (sin theta) * (unit offset
// direction), i.e. the components of the pixel direction along the beam's
// local axes; s2 = x^2 + y^2 = sin^2 theta. Split in two stages so that the
// table load of several samples can be in flight together:
// profile_fetch issues the load (table) or evaluates the weight (radial),
// profile_finish interpolates.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct ProfFetch {
    float4 q;      // table: the 4 corner values; separable: H pair, V pair; radial: q.x = weight
    float fx, fy;
    bool ok;
};

// Echo-only form: the waveform-pool slot of this CTA (written by
// footprint_wave_kernel when FootprintArgs::slot_pool is set, read by the
// pulse convolution and the echo scan).
__shared__ int s_wave_slot;

template <int KIND>
__device__ __forceinline__ ProfFetch profile_fetch(const FootprintArgs &A, float x, float y, bool act,
                                                   float t2max = -1.f)
{
    ProfFetch r;
    float s2 = fmaf(x, x, y * y);
    if (KIND == LIDAR_PROFILE_RADIAL) {
        // theta^2 = asin(s)^2 = s^2 (1 + s^2/3 + 8 s^4/45 + ...)
        float t2 = s2 * fmaf(s2, fmaf(s2, 8.f / 45.f, 1.f / 3.f), 1.f);
        r.ok = act && t2 <= (t2max >= 0.f ? t2max : A.trunc2) && t2 > A.inner2;
        // Gaussian: 2^(t2 kg) with the hardware base-2 exponential (relative
        // error ~2^-22); tail: (theta/theta_c)^-p = rr^(-p/2), with the common
        // p = 3 as rr^-1.5 = rsqrt(rr)^3
        float g = ex2_approx(t2 * A.kg);
        float rr = t2 * A.tc2_inv;
        float tail;
        if (rr <= 1.f) tail = 1.f;
        else if (A.tail_hp == -1.5f) { float q = rsqrtf(rr); tail = q * q * q; }
        else tail = ex2_approx(A.tail_hp * __log2f(rr));
        r.q.x = fmaf(A.tail_amp, tail, g) * A.invZ;
        r.fx = r.fy = 0.f;
    } else {
        // azimuthal-equidistant coordinates: (x, y) * theta / sin theta,
        // theta / sin theta = asin(s)/s = 1 + s^2/6 + 3 s^4/40 + ...
        // The table coordinate is offset * tk + (tiu + tcu) with tiu an
        // integer: the cell index and the fraction come from the small,
        // centre-relative part, so that the steep core of a profile keeps
        // ~1e-7 cells of interpolation precision (an absolute coordinate near
        // 200 would keep only ~1e-5).
        float f = fmaf(s2, fmaf(s2, 3.f / 40.f, 1.f / 6.f), 1.f) * A.tk;
        float cu = fmaf(x, f, A.tcu);
        float cv = fmaf(y, f, A.tcv);
        float icu = floorf(cu), icv = floorf(cv);
        r.fx = cu - icu;
        r.fy = cv - icv;
        if (KIND == LIDAR_PROFILE_SEPARABLE) {
            int i = (int)(icu + A.tiu), j = (int)(icv + A.tiv);
            r.ok = act && (unsigned)i < (unsigned)A.qw && (unsigned)j < (unsigned)A.qh;
            if (!r.ok) {
                r.q = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float2 h = __ldg(A.hpairs + i), v = __ldg(A.vpairs + j);
                r.q = make_float4(h.x, h.y, v.x, v.y);
            }
        } else {
            // the cell's corner nodes (i..i+1, j..j+1) in one gather: it takes
            // the 2 x 2 texels around (i + 1, j + 1) - 1/2 and returns them in
            // the order (i, j+1), (i+1, j+1), (i+1, j), (i, j); texels outside
            // the grid read 0 (border), as the zero-extended profile is there
            const float4 g = tex2Dgather<float4>(A.nodes, icu + A.tiu1, icv + A.tiv1, 0);
            r.q = make_float4(g.w, g.z, g.x, g.y);
            r.ok = act;
        }
    }
    return r;
}

// Adds an accumulated wide deposit (end bins packed in key as for records):
// partial bins f, f+1 and g, g+1, and the run value on f+2 .. g-1 (clipped to
// the window; bins just outside it fall in the buffer's zeroed padding).
__device__ __forceinline__ void wide_flush(float *hj, uint32_t key, float a0, float a1, float a2, float a3, float c,
                                           int pad, int nb)
{
    int xf = (int)(key & 0xFFFFu) - kBinBias + pad;
    int xg = (int)(key >> 16) - kBinBias + pad;
    atomicAdd(hj + skew_pos(xf), a0);
    atomicAdd(hj + skew_pos(xf + 1), a1);
    atomicAdd(hj + skew_pos(xg), a2);
    atomicAdd(hj + skew_pos(xg + 1), a3);
    int xs = max(xf + 2, pad), xe = min(xg - 1, pad + nb - 1);
    for (int x3 = xs; x3 <= xe; ++x3) atomicAdd(hj + skew_pos(x3), c);
}

template <int KIND>
__device__ __forceinline__ float profile_finish(const FootprintArgs &A, const ProfFetch &r)
{
    if (!r.ok) return 0.f;
    if (KIND == LIDAR_PROFILE_RADIAL) return r.q.x;
    if (KIND == LIDAR_PROFILE_SEPARABLE) return fmaf(r.fx, r.q.y - r.q.x, r.q.x) * fmaf(r.fy, r.q.w - r.q.z, r.q.z);
    float top = fmaf(r.fx, r.q.y - r.q.x, r.q.x);
    float bot = fmaf(r.fx, r.q.w - r.q.z, r.q.z);
    return fmaf(r.fy, bot - top, top);
}


// --------------------------------------------------------------------------
// tensor-core form of the deposit (BF16 mma.sync, FP32 accumulation)
// --------------------------------------------------------------------------
//
// For a 16-pixel tile of one row, the deposits of all G (<= 8) beams of the
// group are the product C[bin][beam] += A[bin][pixel] * B[pixel][beam], with
// A the pixels' hat weights (w * D_k) on a block of 16 bins and B the profile
// weights. In the m16n8k16 fragment layout, lane (g, t) = (lane / 4, lane % 4)
// supplies B for beam g at tile pixels 2t, 2t+1, 2t+8, 2t+9 -- the samples it
// evaluates -- and A for the same pixels at bins g and g+8 of the block. Two
// accumulator slots stay in registers while tiles keep hitting the same bin
// blocks and are added to the histograms only when a slot is recycled.
// Each factor is split into BF16 hi + lo parts; hi*hi + hi*lo + lo*hi gives
// products accurate to ~2^-16 (tc_split), or hi*hi alone (plain BF16).

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<uint32_t *>(&h);
}

// x = hi + lo with hi, lo in BF16 (pairs packed low element first)
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    hi = *reinterpret_cast<uint32_t *>(&h);
    float r0 = x0 - __bfloat162float(h.x);
    float r1 = x1 - __bfloat162float(h.y);
    lo = pack_bf16(r0, r1);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One pixel's deposit in bin-index form (bin_records): weight at bin k.
struct PixDep {
    int f, g;       // first bin; for wide pixels the bin of the last partial pair, else -1
    float h0, h1, h2, h3, c;
};

__device__ __forceinline__ float dep_weight(const PixDep &d, int k)
{
    int e = k - d.f;
    if (d.g < 0) {  // narrow: bins f..f+3
        float v = 0.f;
        v = e == 0 ? d.h0 : v;
        v = e == 1 ? d.h1 : v;
        v = e == 2 ? d.h2 : v;
        v = e == 3 ? d.h3 : v;
        return v;
    }
    float v = (k >= d.f + 2 && k <= d.g - 1) ? d.c : 0.f;
    v = e == 0 ? d.h0 : v;
    v = e == 1 ? d.h1 : v;
    v = k == d.g ? d.h2 : v;
    v = k == d.g + 1 ? d.h3 : v;
    return v;
}

template <int G>
__device__ __forceinline__ void tc_flush(float *hbuf, int HB, int pad, const float (&c)[4], int blk, int g, int t)
{
    const int k0 = 16 * blk + g + pad;
    const int bA = 2 * t, bB = 2 * t + 1;
    if (bA < G) {
        if (c[0] != 0.f) atomicAdd(hbuf + bA * HB + skew_pos(k0), c[0]);
        if (c[2] != 0.f) atomicAdd(hbuf + bA * HB + skew_pos(k0 + 8), c[2]);
    }
    if (bB < G) {
        if (c[1] != 0.f) atomicAdd(hbuf + bB * HB + skew_pos(k0), c[1]);
        if (c[3] != 0.f) atomicAdd(hbuf + bB * HB + skew_pos(k0 + 8), c[3]);
    }
}

template <int KIND, int G>
__device__ __forceinline__ float phase1_tc(const FootprintArgs &A, const Layout &Ly, float *hbuf, float2 *tab,
                                           const BeamParam *bp, int gcount, int R0, int R1, int C0, int C1)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nb = A.n_bins, pad = Ly.pad;
    const BeamParam P = bp[g < G ? g : 0];
    const bool gok = g < G && g < gcount && P.valid;
    const float2 *tj = tab + (g < G ? g : 0) * kTC;
    const int blk_lo = -1, blk_hi = (nb + 3) / 16;  // blocks reachable by window deposits
    float amb_acc = 0.f;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    int slot_blk[2] = {INT_MIN, INT_MIN};
    int slot_next = 0;
    for (int cs = C0; cs <= C1; cs += kTC) {
        const int ce = min(C1, cs + kTC - 1);
        const int ncs = ce - cs + 1;
        __syncthreads();  // previous stripe's table no longer read
        for (int i = tid; i < G * ncs; i += blockDim.x) {
            int jj = i / ncs, cc = i - jj * ncs;
            const BeamParam &Q = bp[jj];
            float dAz = ((float)(cs + cc - Q.ci) - Q.cf) * A.daz;
            float sD, vers;
            if (fabsf(dAz) <= 0.1f) {
                float z2 = dAz * dAz;
                sD = dAz * fmaf(-z2 * (1.f / 6.f), fmaf(-z2, 1.f / 20.f, 1.f), 1.f);
                vers = 0.5f * z2 * fmaf(-z2 * (1.f / 12.f), fmaf(-z2, 1.f / 30.f, 1.f), 1.f);
            } else {
                float cD;
                sincosf(dAz, &sD, &cD);
                vers = 1.f - cD;
            }
            tab[jj * kTC + cc] = make_float2(sD, vers);
        }
        __syncthreads();
        if (R0 > R1) continue;
        const int nseg = (ncs + kSeg - 1) / kSeg;
        const int segw = (ncs + nseg - 1) / nseg;
        const int nunits = (R1 - R0 + 1) * nseg;
        for (int unit = warp; unit < nunits; unit += nwarps) {
            const int row = R0 + unit / nseg;
            const int seg = unit - (unit / nseg) * nseg;
            const bool act_row = gok && row >= P.row0 && row <= P.row1;
            const int c_lo = cs + seg * segw, c_hi = min(ce, c_lo + segw - 1);
            int my_lo = max(c_lo, P.col0), my_hi = min(c_hi, P.col1);
            if (!act_row) { my_lo = 1; my_hi = 0; }
            float el = A.el0 + ((float)row + 0.5f) * A.del;
            float cosEl = cosf(el);
            float dEl = ((float)(row - P.ri) - P.rf) * A.del;
            float sdEl = sinf(dEl), cdEl = cosf(dEl);
            float Kv = P.sin_elb * cosEl;
            float Kc = P.cos_elb * cosEl;
            const float ax = P.cg * cosEl, bx = P.sg * Kv, cx = P.sg * sdEl;
            const float ay = -P.sg * cosEl, by = P.cg * Kv, cy = P.cg * sdEl;
            const float4 *recrow = A.rec + 2 * (size_t)row * A.U;
            for (int ct = c_lo; ct <= c_hi; ct += 16) {  // warp-uniform
                PixDep dp[4];
                float Pw[4];
                int bmin = INT_MAX, bmax = INT_MIN;
                bool any_amb = false;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = ct + 2 * t + (u & 1) + 8 * (u >> 1);
                    const bool inrow = c <= c_hi;  // pixel of this unit (for every beam)
                    int cw = c;
                    if (A.panorama) {
                        // the group's columns lie within about one period of [0, U)
                        if (cw < 0) cw += A.U;
                        else if (cw >= A.U) cw -= A.U;
                        if ((unsigned)cw >= (unsigned)A.U) { cw = c % A.U; if (cw < 0) cw += A.U; }
                    }
                    cw = inrow ? cw : 0;
                    float4 r0 = __ldg(recrow + 2 * cw);
                    float4 r1 = __ldg(recrow + 2 * cw + 1);
                    uint32_t kab = __float_as_uint(r0.x);
                    const bool dep = inrow && kab != kNoDeposit;
                    dp[u].f = (int)(kab & 0xFFFFu) - kBinBias;
                    dp[u].g = ((kab >> 16) == 0xFFFFu) ? -1 : (int)(kab >> 16) - kBinBias;
                    dp[u].h0 = dep ? r0.z : 0.f;
                    dp[u].h1 = dep ? r0.w : 0.f;
                    dp[u].h2 = dep ? r1.y : 0.f;
                    dp[u].h3 = dep ? r1.z : 0.f;
                    dp[u].c = dep ? r1.w : 0.f;
                    if (dep) {
                        int last = dp[u].g < 0 ? dp[u].f + 3 : dp[u].g + 1;
                        bmin = min(bmin, max(blk_lo, dp[u].f >> 4));
                        bmax = max(bmax, min(blk_hi, last >> 4));
                    }
                    const float a = inrow ? r0.y : 0.f;
                    any_amb |= a != 0.f;
                    // profile weight of beam g at this pixel
                    const bool act = c >= my_lo && c <= my_hi && (dep || a != 0.f);
                    float2 tt = tj[act ? c - cs : 0];
                    const bool front = act && fmaf(-Kc, tt.y, cdEl) > 0.f;
                    float x = fmaf(ax, tt.x, fmaf(bx, tt.y, cx));
                    float y = fmaf(ay, tt.x, fmaf(by, tt.y, cy));
                    Pw[u] = profile_finish<KIND>(A, profile_fetch<KIND>(A, x, y, front));
                    amb_acc = fmaf(Pw[u], a, amb_acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
                    bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
                }
                if (bmin > bmax) continue;  // no deposit in this tile
                uint32_t bh0, bh1, bl0, bl1;
                split_bf16(Pw[0], Pw[1], bh0, bl0);
                split_bf16(Pw[2], Pw[3], bh1, bl1);
                for (int blk = bmin; blk <= bmax; ++blk) {  // warp-uniform
                    const int k_a = 16 * blk + g, k_b = k_a + 8;
                    float w[8];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        w[u] = dep_weight(dp[u], k_a);
                        w[4 + u] = dep_weight(dp[u], k_b);
                    }
                    bool touch = false;
#pragma unroll
                    for (int i = 0; i < 8; ++i) touch |= w[i] != 0.f;
                    if (!__any_sync(0xffffffffu, touch)) continue;
                    int sl = slot_blk[0] == blk ? 0 : (slot_blk[1] == blk ? 1 : -1);
                    if (sl < 0) {
                        sl = slot_next;
                        slot_next ^= 1;
                        if (slot_blk[sl] != INT_MIN) tc_flush<G>(hbuf, Ly.HB, pad, acc[sl], slot_blk[sl], g, t);
                        slot_blk[sl] = blk;
#pragma unroll
                        for (int i = 0; i < 4; ++i) acc[sl][i] = 0.f;
                    }
                    // A: rows = bins (g, g+8), columns = tile pixels (2t, 2t+1 | 2t+8, 2t+9)
                    uint32_t ah0, ah1, ah2, ah3, al0, al1, al2, al3;
                    split_bf16(w[0], w[1], ah0, al0);  // bin g,   pixels 2t, 2t+1
                    split_bf16(w[4], w[5], ah1, al1);  // bin g+8, pixels 2t, 2t+1
                    split_bf16(w[2], w[3], ah2, al2);  // bin g,   pixels 2t+8, 2t+9
                    split_bf16(w[6], w[7], ah3, al3);  // bin g+8, pixels 2t+8, 2t+9
                    if (sl == 0) {
                        mma_bf16(acc[0], ah0, ah1, ah2, ah3, bh0, bh1);
                        if (A.tc_split) {
                            mma_bf16(acc[0], ah0, ah1, ah2, ah3, bl0, bl1);
                            mma_bf16(acc[0], al0, al1, al2, al3, bh0, bh1);
                        }
                    } else {
                        mma_bf16(acc[1], ah0, ah1, ah2, ah3, bh0, bh1);
                        if (A.tc_split) {
                            mma_bf16(acc[1], ah0, ah1, ah2, ah3, bl0, bl1);
                            mma_bf16(acc[1], al0, al1, al2, al3, bh0, bh1);
                        }
                    }
                }
                (void)any_amb;
            }
        }
    }
    if (slot_blk[0] != INT_MIN) tc_flush<G>(hbuf, Ly.HB, pad, acc[0], slot_blk[0], g, t);
    if (slot_blk[1] != INT_MIN) tc_flush<G>(hbuf, Ly.HB, pad, acc[1], slot_blk[1], g, t);
    return amb_acc;
}

// Adds an accumulated deposit to a beam's histogram: narrow (kq holds the
// positions of bins f+2, f+3) or wide (kq == kNoDeposit, end bins in kab).
__device__ __forceinline__ void dep_flush(float *hj, uint32_t kab, uint32_t kq, float a0, float a1, float a2, float a3,
                                          float c, int pad, int nb)
{
    if (kq != kNoDeposit) {
        atomicAdd(hj + (kab & 0xFFFFu), a0);
        if (a1 != 0.f) atomicAdd(hj + (kab >> 16), a1);
        if (a2 != 0.f) atomicAdd(hj + (kq & 0xFFFFu), a2);
        if (a3 != 0.f) atomicAdd(hj + (kq >> 16), a3);
    } else {
        wide_flush(hj, kab, a0, a1, a2, a3, c, pad, nb);
    }
}

// Phase 1 with shared-memory atomics: the profile-weighted deposits of the
// group's beams over their union pixel box (Alg. 1 kernel loop). The box is
// walked in stripes of kTC columns; for each stripe tab[j][c] holds sin(dAz)
// and 1 - cos(dAz) of column c relative to beam j. A work unit is one row x
// kSeg columns, taken by one warp: lane (j, q) handles beam j on columns
// q, q + CQ, q + 2 CQ, ..., so that a warp's profile lookups stay within one
// row of the table and the lanes on one pixel share its record load.
// CHECKED: the box may wrap around a 2 pi panorama or reach beyond 45 degrees
// from a beam's axis (then every sample is tested for the front hemisphere);
// otherwise neither test is needed. Returns this lane's ambient sum.
// Samples (columns) per lane and loop step of the atomic deposit: their
// record loads and profile fetches are issued together.
constexpr int kSamples = 2;

template <int KIND, int G, bool CHECKED>
__device__ __forceinline__ float phase1_atomic(const FootprintArgs &A, const Layout &Ly, float *hbuf, float2 *tab,
                                               const float2 *rtab, const float *ctab, int *uctr, const BeamParam *bp,
                                               int gcount, int R0, int R1, int C0, int C1, bool use_rtab)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nb = A.n_bins, pad = Ly.pad;
    constexpr int CQ = kWarp / G;  // columns handled side by side per beam
    const int j = lane % G;
    const int q = lane / G;
    const BeamParam P = bp[j];
    const float t2max = P.pad0 ? A.core2 : A.trunc2;
    const bool jok = (j < gcount) && P.valid;
    float *hj = hbuf + j * Ly.HB;
    // Deposits of this lane's successive pixels (all of its beam) that land on
    // the same bins -- the same 4 bins for a narrow interval, the same end
    // bins for a wide one, as a surface at near-constant range gives -- are
    // summed in registers (a0..a3 at the record's 4 bin weights, c at its run
    // value, which is 0 in narrow records) and written with one set of
    // atomics when the key (k0, k1) changes or at the end; this keeps lanes of
    // one beam from hitting the same addresses at the same time.
    uint32_t k0 = kNoDeposit, k1 = kNoDeposit;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, ac = 0.f;
    float amb_acc = 0.f;
    for (int cs = C0; cs <= C1; cs += kTC) {
        const int ce = min(C1, cs + kTC - 1);
        const int ncs = ce - cs + 1;
        __syncthreads();  // previous stripe's table no longer read
        for (int i = tid; i < G * ncs; i += blockDim.x) {
            int jj = i / ncs, cc = i - jj * ncs;
            const BeamParam &Q = bp[jj];
            float dAz = ((float)(cs + cc - Q.ci) - Q.cf) * A.daz;
            float sD, vers;
            if (fabsf(dAz) <= 0.1f) {
                // Taylor series (relative accuracy ~1e-12 for |dAz| <= 0.1)
                float z2 = dAz * dAz;
                sD = dAz * fmaf(-z2 * (1.f / 6.f), fmaf(-z2, 1.f / 20.f, 1.f), 1.f);
                vers = 0.5f * z2 * fmaf(-z2 * (1.f / 12.f), fmaf(-z2, 1.f / 30.f, 1.f), 1.f);
            } else {
                float cD;
                sincosf(dAz, &sD, &cD);
                vers = 1.f - cD;
            }
            tab[jj * kTC + cc] = make_float2(sD, vers);
        }
        if (tid == 0) *uctr = nwarps;
        __syncthreads();
        if (R0 > R1) continue;
        // this lane's table, indexed by absolute column
        const float2 *tjc = tab + j * kTC - cs;
        // columns split into nseg segments of (nearly) equal width <= kSeg
        const int nseg = (ncs + kSeg - 1) / kSeg;
        const int segw = (ncs + nseg - 1) / nseg;
        const int nunits = (R1 - R0 + 1) * nseg;
        // units are handed out to warps from a counter (costs differ: sky
        // units are cheap), the first nwarps directly
        for (int unit = warp; unit < nunits;) {
            const int row = R0 + unit / nseg;
            const int seg = unit - (unit / nseg) * nseg;
            const int c_lo = cs + seg * segw, c_hi = min(ce, c_lo + segw - 1);
            int my_lo = max(c_lo, P.col0), my_hi = min(c_hi, P.col1);
            if (!(jok && row >= P.row0 && row <= P.row1)) { my_lo = 1; my_hi = 0; }
            // active columns: (unsigned)(c - my_lo) <= my_span (none if my_hi < my_lo)
            const unsigned my_span = my_hi >= my_lo ? (unsigned)(my_hi - my_lo) : 0u;
            if (my_hi < my_lo) my_lo = INT_MIN / 2;
            float cosEl, sdEl, cdEl;
            if (use_rtab) {
                const float2 rt = rtab[j * kRT + (row - R0)];
                sdEl = rt.x; cdEl = rt.y; cosEl = ctab[row - R0];
            } else {
                cosEl = cosf(A.el0 + ((float)row + 0.5f) * A.del);
                float dEl = ((float)(row - P.ri) - P.rf) * A.del;
                sincosf(dEl, &sdEl, &cdEl);
            }
            const float Kv = P.sin_elb * cosEl;
            // x = cg xg + sg yg, y = cg yg - sg xg with xg = cosEl sD and
            // yg = sdEl + Kv vers: per-row coefficients of (sD, vers, 1)
            const float ax = P.cg * cosEl, bx = P.sg * Kv, cx = P.sg * sdEl;
            const float ay = -P.sg * cosEl, by = P.cg * Kv, cy = P.cg * sdEl;
            const float Kc = P.cos_elb * cosEl;
            const float4 *recrow = A.rec + 2 * (size_t)row * A.U;
            // kSamples columns per step: all their loads are issued before use.
            // With CQ >= 8 column phases, lane q takes a contiguous run of Lq
            // columns (its successive deposits then share their bins more
            // often, which saves flushes); with fewer phases the columns are
            // interleaved (q, q + CQ, ...), which keeps a warp's table lookups
            // and record loads within a narrower stretch of the row.
            constexpr bool kContig = CQ >= 8;
            const int Lq = kContig ? (c_hi - c_lo + CQ) / CQ : 0;
            const int nsteps = kContig ? (Lq + kSamples - 1) / kSamples
                                       : (c_hi - c_lo + kSamples * CQ) / (kSamples * CQ);
            for (int st = 0; st < nsteps; ++st) {  // warp-uniform trip count
                const int cb = kContig ? c_lo + q * Lq + st * kSamples : c_lo + q + st * kSamples * CQ;
                constexpr int du = kContig ? 1 : CQ;  // column step between a lane's samples
                float4 r0[kSamples], r1s[kSamples];
                bool act[kSamples];
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    const int c = cb + u * du;
                    act[u] = (unsigned)c - (unsigned)my_lo <= my_span && (!kContig || st * kSamples + u < Lq);
                    int cw = c;
                    if (CHECKED && A.panorama) {
                        // the group's columns lie within about one period of [0, U)
                        if (cw < 0) cw += A.U;
                        else if (cw >= A.U) cw -= A.U;
                        if ((unsigned)cw >= (unsigned)A.U) { cw = c % A.U; if (cw < 0) cw += A.U; }
                    }
                    // both halves of the record (one 32-byte sector), issued together
                    r0[u] = act[u] ? __ldg(recrow + 2 * cw) : make_float4(__uint_as_float(kNoDeposit), 0.f, 0.f, 0.f);
                    r1s[u] = act[u] ? __ldg(recrow + 2 * cw + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                    // a pixel with neither a return nor ambient light adds nothing
                    act[u] = act[u] && !(__float_as_uint(r0[u].x) == kNoDeposit && r0[u].y == 0.f);
                }
                bool any = false;
#pragma unroll
                for (int u = 0; u < kSamples; ++u) any |= act[u];
                if (!__any_sync(0xffffffffu, any)) continue;
                ProfFetch pf[kSamples];
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    const int c = cb + u * du;
                    const float2 t = tjc[act[u] ? c : cs];
                    bool ok = act[u];
                    // front hemisphere only: d.a = cos(dEl) - cos el_b cos el (1 - cos dAz)
                    if (CHECKED) ok = ok && fmaf(-Kc, t.y, cdEl) > 0.f;
                    const float x = fmaf(ax, t.x, fmaf(bx, t.y, cx));
                    const float y = fmaf(ay, t.x, fmaf(by, t.y, cy));
                    pf[u] = profile_fetch<KIND>(A, x, y, ok, t2max);
                }
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    // Pw = 0 for an inactive sample or outside the support:
                    // the ambient term adds nothing then
                    const float Pw = profile_finish<KIND>(A, pf[u]);
                    amb_acc = fmaf(Pw, r0[u].y, amb_acc);
                    const uint32_t kab = __float_as_uint(r0[u].x);
                    const bool dep = Pw > 0.f && kab != kNoDeposit;
                    const float4 r1 = r1s[u];
                    const uint32_t kq = __float_as_uint(r1.x);
                    if (dep && (kab != k0 || kq != k1)) {
                        if (k0 != kNoDeposit) dep_flush(hj, k0, k1, a0, a1, a2, a3, ac, pad, nb);
                        k0 = kab; k1 = kq;
                        a0 = 0.f; a1 = 0.f; a2 = 0.f; a3 = 0.f; ac = 0.f;
                    }
                    const float pw = dep ? Pw : 0.f;
                    a0 = fmaf(pw, r0[u].z, a0);
                    a1 = fmaf(pw, r0[u].w, a1);
                    a2 = fmaf(pw, r1.y, a2);
                    a3 = fmaf(pw, r1.z, a3);
                    ac = fmaf(pw, r1.w, ac);
                }
            }
            int nu = 0;
            if (lane == 0) nu = atomicAdd(uctr, 1);
            unit = __shfl_sync(0xffffffffu, nu, 0);
        }
    }
    if (k0 != kNoDeposit) dep_flush(hj, k0, k1, a0, a1, a2, a3, ac, pad, nb);
    return amb_acc;
}

// The box a lean phase 1 walks for each beam of a group: the group's union
// box (all beams share the origin (C0, R0)), or, for beams too far apart for
// their boxes to overlap much, each beam's own box widened to the common
// size Wb x Hb and shifted inside the G-buffer where it reaches an edge.
struct LeanBox {
    int pb;        // 1: per-beam boxes, 0: the union box
    int R0, C0;    // origin of the union box
    int Hb, Wb;    // rows and columns walked for every beam (Wb a multiple of the warp step)
};

__device__ __forceinline__ int2 lean_origin(const BeamParam &Q, const LeanBox &B, int U, int V)
{
    if (!B.pb) return make_int2(B.C0, B.R0);
    if (!Q.valid) return make_int2(0, 0);
    return make_int2(min(Q.col0, U - B.Wb), min(Q.row0, V - B.Hb));
}

// Phase 1, lean form of the atomic deposit, for groups whose boxes need
// neither the panorama wrap nor the front-hemisphere test. Every beam's box
// (the group's union box, or the beam's own box for a group of beams too far
// apart to share much of it) is widened to whole warp steps inside the
// G-buffer: a column outside a beam's own box lies outside its profile's
// support, where the profile weight is exactly 0, so no sample needs a bounds
// or activity test. A lane whose beam slot is empty evaluates its profile far
// outside any support (weight 0).
// Lane (j, q) takes beam j on columns q, q + CQ, ... of each step of CQ *
// kSamples columns (or, with 4 or fewer beams per CTA, a contiguous run of
// columns); its loads use fixed offsets from two pointers advanced once per
// step (the offset table is stored [column][beam], so that a warp reads
// consecutive entries). A record's first word alone identifies its
// deposit (the bin positions of a narrow record differ by 1 or 2, the end bins
// of a wide one by at least 3), so one compare decides whether a deposit joins
// the lane's accumulated one. Accumulating a lane's successive deposits that
// share their bins also keeps the FP32 sums of a bin that thousands of samples
// reach (a plane facing the sensor) short.
template <int KIND, int G, bool PB>
__device__ __forceinline__ float phase1_lean(const FootprintArgs &A, const Layout &Ly, float *hbuf, float2 *tab,
                                             float2 *rtab, float *ctab, int *uctr, const BeamParam *bp,
                                             int gcount, const LeanBox &B)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int nb = A.n_bins, pad = Ly.pad;
    constexpr int CQ = kWarp / G;
    constexpr int kStep = CQ * kSamples;                // columns per warp step
    constexpr int kStripe = (kTC - 1) / kStep * kStep;  // columns per offset-table stripe
    // With 8 or more column phases (4 or fewer beams per CTA) a lane walks a
    // contiguous run of columns: its successive deposits then share their bins
    // far more often (a surface at slowly varying range), which saves flushes;
    // with fewer phases the columns are interleaved (q, q + CQ, ...), which
    // keeps a warp's record loads within one or two cache lines.
    constexpr bool kContig = CQ >= 8;
    constexpr int kDu = kContig ? 1 : CQ;                // columns between a lane's samples of a step
    constexpr int kAdv = kContig ? kSamples : kStep;     // columns a lane advances per step
    const int j = lane % G;
    const int q = lane / G;
    const BeamParam P = bp[j];
    const float t2max = P.pad0 ? A.core2 : A.trunc2;
    const bool jok = (j < gcount) && P.valid;
    // this lane's box origin (the same in every lane for the union box)
    const int2 org = PB ? lean_origin(P, B, A.U, A.V) : make_int2(B.C0, B.R0);
    float *hj = hbuf + j * Ly.HB;
    uint32_t k0 = kNoDeposit, k1 = kNoDeposit;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, ac = 0.f;
    float amb_acc = 0.f;
    // per (beam, row of its box): sin of the elevation offset, and cos(el) of
    // the row (per row in ctab for the union box, beside the sine otherwise)
    const bool use_rtab = B.Hb <= kRT;
    if (use_rtab) {
        for (int i = tid; i < G * B.Hb; i += blockDim.x) {
            const int rr = i / G, jj = i - rr * G;
            const BeamParam &Q = bp[jj];
            const int row = (PB ? lean_origin(Q, B, A.U, A.V).y : B.R0) + rr;
            const float dEl = ((float)(row - Q.ri) - Q.rf) * A.del;
            if (PB) {
                rtab[jj * kRT + rr] = make_float2(sinf(dEl), cosf(A.el0 + ((float)row + 0.5f) * A.del));
            } else {
                rtab[jj * kRT + rr].x = sinf(dEl);
                if (jj == 0) ctab[rr] = cosf(A.el0 + ((float)row + 0.5f) * A.del);
            }
        }
    }
    for (int cs = 0; cs < B.Wb; cs += kStripe) {
        const int ncs = min(B.Wb - cs, kStripe);  // a multiple of kStep
        __syncthreads();  // previous stripe's table no longer read (and the row table is written)
        for (int i = tid; i < G * ncs; i += blockDim.x) {
            const int cc = i / G, jj = i - cc * G;
            const BeamParam &Q = bp[jj];
            const int col = (PB ? lean_origin(Q, B, A.U, A.V).x : B.C0) + cs + cc;
            float dAz = ((float)(col - Q.ci) - Q.cf) * A.daz;
            float sD, vers;
            if (fabsf(dAz) <= 0.1f) {
                float z2 = dAz * dAz;
                sD = dAz * fmaf(-z2 * (1.f / 6.f), fmaf(-z2, 1.f / 20.f, 1.f), 1.f);
                vers = 0.5f * z2 * fmaf(-z2 * (1.f / 12.f), fmaf(-z2, 1.f / 30.f, 1.f), 1.f);
            } else {
                float cD;
                sincosf(dAz, &sD, &cD);
                vers = 1.f - cD;
            }
            tab[i] = make_float2(sD, vers);
        }
        if (tid == 0) *uctr = nwarps;
        __syncthreads();
        // segments of whole steps, at most kSegLean (rounded up to a step) wide
        const int nseg = (ncs + kSegLean - 1) / kSegLean;
        const int segw = ((ncs + nseg - 1) / nseg + kStep - 1) / kStep * kStep;
        const int nunits = B.Hb * nseg;
        for (int unit = warp; unit < nunits;) {
            const int rr = unit / nseg;
            const int seg = unit - rr * nseg;
            const int c_lo = seg * segw;  // relative to the stripe
            const int nsteps = max(0, min(ncs - c_lo, segw)) / kStep;
            const int row = org.y + rr;
            float cosEl, sdEl;
            if (use_rtab) {
                const float2 rt = rtab[j * kRT + rr];
                sdEl = rt.x;
                cosEl = PB ? rt.y : ctab[rr];
            } else {
                cosEl = cosf(A.el0 + ((float)row + 0.5f) * A.del);
                sdEl = sinf(((float)(row - P.ri) - P.rf) * A.del);
            }
            const float Kv = P.sin_elb * cosEl;
            float ax = P.cg * cosEl, bx = P.sg * Kv, cx = P.sg * sdEl;
            float ay = -P.sg * cosEl, by = P.cg * Kv, cy = P.cg * sdEl;
            if (!jok) {
                // (x, y) = (3, 0): far outside every profile's support
                ax = 0.f; bx = 0.f; cx = 3.f; ay = 0.f; by = 0.f; cy = 0.f;
            }
            // lane (j, q) starts at column q (interleaved: q + CQ u) or at q Lq
            // (contiguous: Lq columns per lane, Lq = nsteps kSamples)
            const int q0 = kContig ? q * nsteps * kSamples : q;
            const float4 *rp = A.rec + 2 * ((size_t)row * A.U + (size_t)(org.x + cs + c_lo + q0));
            const float2 *tp = tab + (c_lo + q0) * G + j;
            for (int st = 0; st < nsteps; ++st) {
                float4 r0[kSamples], r1s[kSamples];
                float2 t[kSamples];
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    r0[u] = __ldg(rp + 2 * kDu * u);
                    r1s[u] = __ldg(rp + 2 * kDu * u + 1);
                    t[u] = tp[G * kDu * u];
                }
                rp += 2 * kAdv;
                tp += G * kAdv;
                // a record with neither a deposit nor ambient light adds nothing
                uint32_t live = 0u;
#pragma unroll
                for (int u = 0; u < kSamples; ++u)
                    live |= (__float_as_uint(r0[u].x) + 1u) | __float_as_uint(r0[u].y);
                if (!__any_sync(0xffffffffu, live != 0u)) continue;
                ProfFetch pf[kSamples];
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    const float x = fmaf(ax, t[u].x, fmaf(bx, t[u].y, cx));
                    const float y = fmaf(ay, t[u].x, fmaf(by, t[u].y, cy));
                    pf[u] = profile_fetch<KIND>(A, x, y, true, t2max);
                }
#pragma unroll
                for (int u = 0; u < kSamples; ++u) {
                    // records without a deposit carry zero weights, and a zero
                    // profile weight adds zeros: only the key switch is tested
                    const float Pw = profile_finish<KIND>(A, pf[u]);
                    amb_acc = fmaf(Pw, r0[u].y, amb_acc);
                    const uint32_t kab = __float_as_uint(r0[u].x);
                    if (Pw > 0.f && kab != k0 && kab != kNoDeposit) {
                        if (k0 != kNoDeposit) dep_flush(hj, k0, k1, a0, a1, a2, a3, ac, pad, nb);
                        k0 = kab; k1 = __float_as_uint(r1s[u].x);
                        a0 = 0.f; a1 = 0.f; a2 = 0.f; a3 = 0.f; ac = 0.f;
                    }
                    a0 = fmaf(Pw, r0[u].z, a0);
                    a1 = fmaf(Pw, r0[u].w, a1);
                    a2 = fmaf(Pw, r1s[u].y, a2);
                    a3 = fmaf(Pw, r1s[u].z, a3);
                    ac = fmaf(Pw, r1s[u].w, ac);
                }
            }
            int nu = 0;
            if (lane == 0) nu = atomicAdd(uctr, 1);
            unit = __shfl_sync(0xffffffffu, nu, 0);
        }
    }
    if (k0 != kNoDeposit) dep_flush(hj, k0, k1, a0, a1, a2, a3, ac, pad, nb);
    return amb_acc;
}

// Phases 2-4 of a group whose histograms are in hbuf (G slots; slot jj for
// beam slot b0 + jj, jj < gcount): window edges and support, pulse convolution +
// ambient with the waveform written out, echo extraction. Every thread of the
// CTA must call it (it contains block barriers). The echo-only form keeps the
// waveforms in rows slot_row0 + jj of the CTA's pool slot of slot_rows rows.
__device__ __forceinline__ void footprint_finish(const FootprintArgs &A, const Layout &Ly, float *hbuf,
                                              const float *taps, float *amb_s, int *supp, int *tsupp,
                                              float *nrm2_s, float *tmass_s, const BeamParam *bp, int b0,
                                              int gcount, int G, int slot_row0, int slot_rows)
{
    const int nb = A.n_bins, M = A.M;
    const int pad = Ly.pad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    (void)tid;
    // ---- phase 2: drop contributions outside the window, support ----------
    for (int jj = warp; jj < G; jj += nwarps) {
        float *hj = hbuf + jj * Ly.HB;
        if (lane < 4) {
            hj[skew_pos(pad - 4 + lane)] = 0.f;
            hj[skew_pos(pad + nb + lane)] = 0.f;
        }
        __syncwarp();
        int tlo = 1 << 30, thi = -1;
        if (jj < gcount && (A.tail_in || A.coarse_out)) {
            const int cf = nb / A.n_coarse;
            const size_t row = (size_t)(b0 + jj) * A.tail_stride;
            if (A.tail_in && bp[jj].pad0) {
                // added tail of a core-only beam: its coarse support and ambient sum
                // (the coarse histogram itself enters in the convolution phase)
                float tm = 0.f;
                for (int c = lane; c < A.n_coarse; c += 32) {
                    const float v = A.tail_in[row + c];
                    if (v != 0.f) { tlo = min(tlo, c); thi = max(thi, c); }
                    tm += v;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    tlo = min(tlo, __shfl_xor_sync(0xffffffffu, tlo, o));
                    thi = max(thi, __shfl_xor_sync(0xffffffffu, thi, o));
                    tm += __shfl_xor_sync(0xffffffffu, tm, o);
                }
                if (lane == 0) { amb_s[jj] += A.tail_in[row + A.n_coarse]; tmass_s[jj] = tm; }
            }
            if (A.coarse_out) {
                float tot = 0.f;
                for (int cb = 0; cb < A.n_coarse; ++cb) {
                    float v = 0.f;
                    for (int k = cb * cf + lane; k < (cb + 1) * cf; k += 32) v += hj[skew_pos(k + pad)];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) A.coarse_out[row + cb] = v;
                    tot += v;
                }
                if (lane == 0) {
                    A.coarse_out[row + A.n_coarse] = amb_s[jj];
                    A.coarse_out[row + A.n_coarse + 1] = 0.f;
                    A.coarse_out[row + A.n_coarse + 2] = 0.f;
                    A.coarse_out[row + A.n_coarse + 3] = tot;
                }
            }
            __syncwarp();
        }
        int lo = 1 << 30, hi = -1;
        for (int k = lane; k < nb; k += 32) {
            if (hj[skew_pos(k + pad)] != 0.f) { lo = min(lo, k); hi = max(hi, k); }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) { supp[2 * jj] = lo; supp[2 * jj + 1] = hi; tsupp[2 * jj] = tlo; tsupp[2 * jj + 1] = thi; }
    }
    __syncthreads();

    // ---- phase 3: pulse convolution + ambient, waveform to HBM -------------
    // Lane L of an item owns bins o0 + 8L .. o0 + 8L + 7; the 8 inputs it needs
    // for tap m are a window that slides by one bin per tap, kept in registers.
    const int nblk = (nb + kBlk - 1) / kBlk;
    for (int it = warp; it < gcount * nblk; it += nwarps) {
        int jj = it / nblk;
        int o0 = (it - jj * nblk) * kBlk;
        const float *hj = hbuf + jj * Ly.HB;
        const int lo = supp[2 * jj], hi = supp[2 * jj + 1];
        const float ambv = amb_s[jj] * A.s_amb;
        float acc[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r] = ambv;
        const int kb = min(o0 + 8 * lane, nb - 8);  // lanes past the end compute a copy, not stored
        // taps that connect this lane's 8 outputs with the histogram's support
        // (the rest multiply zeros); lanes then read the same histogram bin
        // and taps 8 apart, which the skewed tap layout keeps in distinct banks
        int m_lo = max(-M, kb - hi), m_hi = min(M, kb + 7 - lo);
        if (hi >= 0 && m_lo <= m_hi) {
            m_lo = (m_lo >> 3) << 3;  // floor to a multiple of 8
            const float *hb = hj;
            float win[8];
#pragma unroll
            for (int r = 1; r < 8; ++r) win[r] = hb[skew_pos(kb + r - m_lo + pad)];
            for (int m0 = m_lo; m0 <= m_hi; m0 += 8) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int m = m0 + i;
                    win[(8 - i) & 7] = hb[skew_pos(kb - m + pad)];
                    const float t = taps[skew_pos(Ly.taps_off + m)];
#pragma unroll
                    for (int r = 0; r < 8; ++r) acc[r] = fmaf(t, win[(r - i) & 7], acc[r]);
                }
            }
        }
        const int tlo = tsupp[2 * jj], thi = tsupp[2 * jj + 1];
        if (thi >= 0) {
            // added coarse tail: mass T_c spread evenly over the cf fine bins of
            // coarse bin c, convolved with the pulse = sum_c T_c B(k - c cf),
            // B(x) = (1/cf) sum_{j<cf} p(x - j) (tail_box, index x + tb_off)
            const int cf = nb / A.n_coarse;
            const float *Tr = A.tail_in + (size_t)(b0 + jj) * A.tail_stride;
            // first coarse bin reaching output kb: ceil((kb - M - cf + 1) / cf) = floor((kb - M) / cf)
            const int c0 = max(tlo, (kb - M + cf * (M + 1)) / cf - (M + 1));
            const int c1 = min(thi, (kb + 7 + M) / cf);
            if ((cf & 3) == 0) {
                // kb, c * cf and tb_off are multiples of 4: two 16-byte loads of B per coarse bin
                for (int c = c0; c <= c1; ++c) {
                    const float t = __ldg(Tr + c);
                    const float4 *bx = reinterpret_cast<const float4 *>(A.tail_box + A.tb_off + kb - c * cf);
                    const float4 u = __ldg(bx), w = __ldg(bx + 1);
                    acc[0] = fmaf(t, u.x, acc[0]); acc[1] = fmaf(t, u.y, acc[1]);
                    acc[2] = fmaf(t, u.z, acc[2]); acc[3] = fmaf(t, u.w, acc[3]);
                    acc[4] = fmaf(t, w.x, acc[4]); acc[5] = fmaf(t, w.y, acc[5]);
                    acc[6] = fmaf(t, w.z, acc[6]); acc[7] = fmaf(t, w.w, acc[7]);
                }
            } else {
                for (int c = c0; c <= c1; ++c) {
                    const float t = __ldg(Tr + c);
                    const float *bx = A.tail_box + A.tb_off + kb - c * cf;
#pragma unroll
                    for (int r = 0; r < 8; ++r) acc[r] = fmaf(t, __ldg(bx + r), acc[r]);
                }
            }
        }
        if (o0 + 8 * lane < nb) {
            const size_t orow = A.out_ids ? (size_t)A.out_ids[b0 + jj] : (size_t)(b0 + jj);
            float *wrow = A.slot_pool ? A.slot_pool + ((size_t)s_wave_slot * slot_rows + slot_row0 + jj) * nb : A.wave + orow * nb;
            float4 *dst = reinterpret_cast<float4 *>(wrow + o0 + 8 * lane);
            dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        }
        if (A.tail_in && bp[jj].pad0) {
            // squared L2 norm of the waveform (acceptance test of the tail)
            float s2 = 0.f;
            if (o0 + 8 * lane < nb) {
#pragma unroll
                for (int r = 0; r < 8; ++r) s2 = fmaf(acc[r], acc[r], s2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            if (lane == 0) atomicAdd(nrm2_s + jj, s2);
        }
    }
    __syncthreads();

    // ---- phase 4: echoes ---------------------------------------------------
    // With the ambient level at or below T, bins farther than M from the
    // histogram's support hold the ambient level only and cannot be part of a
    // run, so the scan covers [lo - M - 1, hi + M + 1]. Loads run one chunk ahead.
    for (int jj = warp; jj < gcount; jj += nwarps) {
        const int beam = A.out_ids ? A.out_ids[b0 + jj] : b0 + jj;
        const float *xw = A.slot_pool ? A.slot_pool + ((size_t)s_wave_slot * slot_rows + slot_row0 + jj) * nb : A.wave + (size_t)beam * nb;
        lidar_echo_t *eo = A.echoes + (size_t)beam * A.max_echoes;
        const float T = A.T;
        const float ambv = amb_s[jj] * A.s_amb;
        const int lo = supp[2 * jj], hi = supp[2 * jj + 1];
        int kbeg, kend;
        if (ambv > T) { kbeg = 0; kend = nb - 1; }
        else if (hi < 0) { kbeg = 1; kend = 0; }
        else { kbeg = max(0, lo - M - 1); kend = min(nb - 1, hi + M + 1); }
        // Acceptance test of a core-only beam whose tail was predicted: the
        // exact tail and the prediction are both non-negative with mass at
        // most Eub, so the difference moves any bin by at most eps and bin
        // differences by at most 2 Eub times the pulse's differences. The beam
        // is re-run exactly unless neither can change a bin's side of T, the
        // peak bin, or move the waveform, a crossing or the peak vertex by more
        // than the budgets.
        const bool gated = A.tail_in != nullptr && bp[jj].pad0 != 0;
        float g_eub = 0.f, g_eps = 0.f;
        bool gfail = false;
        if (gated) {
            const float *trow = A.tail_in + (size_t)beam * A.tail_stride;
            g_eub = trow[A.n_coarse + 1];
            const float dAs = trow[A.n_coarse + 2] * A.s_amb;
            g_eps = 1.01f * fmaf(g_eub, A.g_pmax, dAs);
            const float l2err = 1.01f * (1.4142136f * g_eub * A.g_pl2 + dAs * sqrtf((float)nb));
            gfail = !(l2err <= A.g_l2 * sqrtf(nrm2_s[jj]));
            if (ambv <= T) gfail |= !(T - ambv > g_eps);  // bins outside the scan
            gfail |= !(isfinite(g_eub) && isfinite(g_eps));
        }
        // An added tail widens the scan to its own support, unless it is too
        // weak to matter there: away from the core's support the waveform is at
        // most ambv + (tail mass) max(p), and if that stays below T - eps
        // neither this waveform nor the exact one (within eps of it) can have a
        // bin at or above T there.
        if (tsupp[2 * jj + 1] >= 0 && !(ambv > T) &&
            !(gated && ambv + 1.01f * tmass_s[jj] * A.g_pmax < T - g_eps)) {
            const int cf = nb / A.n_coarse;
            const int tb = max(0, tsupp[2 * jj] * cf - M - 1), te = min(nb - 1, (tsupp[2 * jj + 1] + 1) * cf + M);
            if (kbeg > kend) { kbeg = tb; kend = te; }
            else { kbeg = min(kbeg, tb); kend = max(kend, te); }
        }
        int count = 0;
        bool open = false;
        int bs = 0, pk = 0;
        float pv = 0.f;
        // the strongest-echo form scans every run and keeps the best one (lane 0)
        const int cap = A.strongest ? INT_MAX : A.max_echoes;
        lidar_echo_t best{};
        const int cfirst = kbeg >> 5, clast = kend >> 5;
        float v = 0.f, prev_last = 0.f;
        if (kbeg <= kend) {
            v = xw[32 * cfirst + lane];
            prev_last = cfirst > 0 ? xw[32 * cfirst - 1] : 0.f;
        }
        for (int c = cfirst; c <= clast && kbeg <= kend && count < cap; ++c) {
            const int k = 32 * c + lane;
            const float v_next = (k + 32 < nb) ? xw[k + 32] : 0.f;
            float vn = __shfl_down_sync(0xffffffffu, v, 1);
            float vnn = __shfl_sync(0xffffffffu, v_next, 0);
            if (lane == 31) vn = vnn;
            float vp = __shfl_up_sync(0xffffffffu, v, 1);
            if (lane == 0) vp = prev_last;
            if (gated) gfail |= __any_sync(0xffffffffu, k >= kbeg && k <= kend && fabsf(v - T) <= g_eps);
            bool ab = v > T;
            bool st = ab && !(k > 0 && vp > T);
            bool en = ab && !(k + 1 < nb && vn > T);
            uint32_t Sm = __ballot_sync(0xffffffffu, st);
            uint32_t Em = __ballot_sync(0xffffffffu, en);
            int seg_lo = 0;
            uint32_t ev = Sm | Em;
            while (ev && count < cap) {
                int i = __ffs(ev) - 1;
                ev &= ev - 1;
                if ((Sm >> i) & 1u) { open = true; bs = 32 * c + i; pv = -1.f; pk = bs; seg_lo = i; }
                if ((Em >> i) & 1u) {
                    // argmax over [seg_lo, i] of this chunk, lowest bin on ties
                    float mv = (lane >= seg_lo && lane <= i) ? v : -1.f;
                    int mi = k;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        float ov = __shfl_xor_sync(0xffffffffu, mv, o);
                        int oi = __shfl_xor_sync(0xffffffffu, mi, o);
                        if (ov > mv || (ov == mv && oi < mi)) { mv = ov; mi = oi; }
                    }
                    if (mv > pv) { pv = mv; pk = mi; }
                    int be = 32 * c + i;
                    if (lane == 0) {
                        lidar_echo_t e;
                        uint32_t fl = 0;
                        float x0, x1;
                        float vbs = xw[bs], vbe = xw[be];
                        float eps = kNearRel * T;
                        if (bs > 0) {
                            float vm = xw[bs - 1];
                            x0 = (float)(bs - 1) + (T - vm) / (vbs - vm);
                            if (fabsf(vm - T) <= eps) fl |= LIDAR_ECHO_NEAR_THRESHOLD;
                        } else { x0 = 0.f; fl |= LIDAR_ECHO_CLIPPED_START; }
                        if (be < nb - 1) {
                            float vq = xw[be + 1];
                            x1 = (float)be + (vbe - T) / (vbe - vq);
                            if (fabsf(vq - T) <= eps) fl |= LIDAR_ECHO_NEAR_THRESHOLD;
                        } else { x1 = (float)(nb - 1); fl |= LIDAR_ECHO_CLIPPED_END; }
                        if (fabsf(vbs - T) <= eps || fabsf(vbe - T) <= eps) fl |= LIDAR_ECHO_NEAR_THRESHOLD;
                        float dl = 0.f;
                        if (pk > 0 && pk < nb - 1) {
                            float va = xw[pk - 1], vb = xw[pk], vc = xw[pk + 1];
                            if (va > 0.f && vb > 0.f && vc > 0.f) {
                                float la = logf(va), lb = logf(vb), lc = logf(vc);
                                float den = la - 2.f * lb + lc;
                                if (den < 0.f) dl = 0.5f * (la - lc) / den;
                                if (gated) {
                                    // first-order change of the log-parabola vertex, plus
                                    // the second-order term of each log
                                    const float D = 2.02f * g_eub;
                                    const float q = g_eps / fminf(va, fminf(vb, vc));
                                    const float dnum = D * A.g_d2 / va + g_eps * fabsf(1.f / va - 1.f / vc) + 2.f * q * q;
                                    const float dden = D * A.g_dd / vb +
                                                       g_eps * (fabsf(1.f / va - 1.f / vb) + fabsf(1.f / vc - 1.f / vb)) +
                                                       4.f * q * q;
                                    const float ad = fabsf(den);
                                    if (!(ad > 2.f * dden)) gfail = true;
                                    else {
                                        float ddl = 0.5f * (dnum * ad + fabsf(la - lc) * dden) / (ad * (ad - dden));
                                        if (!(ddl * A.rB <= A.g_dr)) gfail = true;
                                    }
                                    // the bins next to the peak must stay below it
                                    if (pk - 1 >= bs && !(vb - va > D * A.g_d1)) gfail = true;
                                    if (pk + 1 <= be && !(vb - vc > D * A.g_d1)) gfail = true;
                                }
                            } else {
                                float den = va - 2.f * vb + vc;
                                if (den < 0.f) dl = 0.5f * (va - vc) / den;
                                if (gated) gfail = true;
                            }
                            dl = fminf(0.5f, fmaxf(-0.5f, dl));
                        }
                        float r0m = fmaf(x0, A.rB, A.rA), r1m = fmaf(x1, A.rB, A.rA);
                        float epw = r1m - r0m;
                        float E2 = epw * epw;
                        if (gated) {
                            // crossings: x = k + (T - a) / (b - a) moves by at most
                            // (|b - T| + |T - a|) eps / (b - a)^2 to first order
                            float dx = 0.f;
                            if (bs > 0) {
                                float vm = xw[bs - 1], w = vbs - vm, q = g_eps / w;
                                dx += (fabsf(vbs - T) + fabsf(T - vm)) * g_eps / (w * w) + 4.f * q * q;
                            }
                            if (be < nb - 1) {
                                float vq = xw[be + 1], w = vbe - vq, q = g_eps / w;
                                dx += (fabsf(vbe - T) + fabsf(T - vq)) * g_eps / (w * w) + 4.f * q * q;
                            }
                            const float dE = dx * A.rB;
                            const float slope = fabsf(2.f * A.c1 * epw + 4.f * A.c2 * epw * E2);
                            if (!(dE <= A.g_dr && slope * dE <= 3e-4f && g_eps <= 3e-4f * pv)) gfail = true;
                        }
                        e.range_m = fmaf((float)pk + dl, A.rB, A.rA);
                        e.epw_m = epw;
                        e.intensity = expf(fmaf(A.c2 * E2, E2, fmaf(A.c1, E2, A.c0)));
                        e.peak = pv;
                        e.bin_peak = pk;
                        e.bin_start = bs;
                        e.bin_end = be;
                        e.flags = fl;
                        if (!A.strongest) eo[count] = e;
                        else if (count == 0 || e.intensity > best.intensity) best = e;
                    }
                    if (gated) {
                        // every other bin of the run must stay below the peak
                        float m2 = -1.f;
                        for (int qb = bs + lane; qb <= be; qb += 32)
                            if (qb < pk - 1 || qb > pk + 1) m2 = fmaxf(m2, xw[qb]);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                        if (m2 >= 0.f && !(pv - m2 > 2.02f * g_eub * A.g_pmax)) gfail = true;
                    }
                    ++count;
                    open = false;
                    seg_lo = i + 1;
                }
            }
            if (open) {
                float mv = (lane >= seg_lo) ? v : -1.f;
                int mi = k;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    float ov = __shfl_xor_sync(0xffffffffu, mv, o);
                    int oi = __shfl_xor_sync(0xffffffffu, mi, o);
                    if (ov > mv || (ov == mv && oi < mi)) { mv = ov; mi = oi; }
                }
                if (mv > pv) { pv = mv; pk = mi; }
            }
            prev_last = __shfl_sync(0xffffffffu, v, 31);
            v = v_next;
        }
        if (lane == 0) {
            if (A.strongest) {
                eo[0] = best;  // zero when there is no echo
                count = count > 0 ? 1 : 0;
                for (int e = 1; e < A.max_echoes; ++e) eo[e] = lidar_echo_t{};
            } else {
                for (int e = count; e < A.max_echoes; ++e) eo[e] = lidar_echo_t{};
            }
            A.counts[beam] = count;
        }
        if (gated && __any_sync(0xffffffffu, gfail) && lane == 0) A.fb_flags[beam] = 1;
    }
}

// One group of G consecutive beams of one frame (the whole per-CTA pipeline).
// Every thread of the CTA must call it (it contains block barriers).
template <int KIND, int G, bool TC>
__device__ __forceinline__ void footprint_group(const FootprintArgs &A, const int group, unsigned char *smem_raw)
{
    const int nb = A.n_bins, M = A.M;
    const Layout Ly = make_layout(G, nb, M);
    float *hbuf = reinterpret_cast<float *>(smem_raw);
    float *taps = reinterpret_cast<float *>(smem_raw + Ly.off_taps);
    float *amb_s = reinterpret_cast<float *>(smem_raw + Ly.off_amb);
    int *supp = reinterpret_cast<int *>(smem_raw + Ly.off_supp);
    int *tsupp = reinterpret_cast<int *>(smem_raw + Ly.off_tsupp);  // coarse support of an added tail
    float *nrm2_s = reinterpret_cast<float *>(smem_raw + Ly.off_nrm);
    float *tmass_s = reinterpret_cast<float *>(smem_raw + Ly.off_tmass);  // mass of an added tail
    float2 *tab = reinterpret_cast<float2 *>(smem_raw + Ly.off_tab);
    float2 *rtab = reinterpret_cast<float2 *>(smem_raw + Ly.off_rtab);
    float *ctab = reinterpret_cast<float *>(smem_raw + Ly.off_ctab);
    int *uctr = reinterpret_cast<int *>(smem_raw + Ly.off_ctr);
    BeamParam *bp = reinterpret_cast<BeamParam *>(smem_raw + Ly.off_bp);

    const int tid = threadIdx.x, lane = tid & 31;
    const int b0 = group * G;
    const int gcount = min(G, A.n_beams - b0);

    // ---- phase 0: clear, load parameters, union box ----------------------
    for (int i = tid; i < G * Ly.HB; i += blockDim.x) hbuf[i] = 0.f;
    for (int i = tid; i < Ly.taps_len; i += blockDim.x) {
        int m = i - Ly.taps_off;
        taps[skew_pos(i)] = (m >= -M && m <= M) ? A.taps_pad[A.tp_off + m] : 0.f;
    }
    if (tid < G) {
        amb_s[tid] = 0.f;
        nrm2_s[tid] = 0.f;
        BeamParam P;
        if (tid < gcount) P = A.beams[b0 + tid];
        else { P = BeamParam{}; P.valid = 0; }
        bp[tid] = P;
    }
    __syncthreads();
    if (tid < G && A.panorama) {
        // keep all boxes of the group in the unwrapped period of the first valid beam
        int ref = -1;
        for (int j = 0; j < gcount; ++j) if (bp[j].valid) { ref = bp[j].ci; break; }
        BeamParam &P = bp[tid];
        if (P.valid && ref >= 0) {
            int sh = 0;
            while (P.ci + sh - ref > A.U / 2) sh -= A.U;
            while (P.ci + sh - ref < -A.U / 2) sh += A.U;
            P.ci += sh; P.col0 += sh; P.col1 += sh;
        }
    }
    __syncthreads();
    // Box extents and the tests below, one beam per lane (G <= 16), reduced
    // across the warp: every warp computes them, no barrier needed.
    const unsigned full = 0xffffffffu;
    const BeamParam &Ql = bp[min(lane, G - 1)];
    const bool vl = lane < gcount && Ql.valid;
    const int R0 = __reduce_min_sync(full, vl ? Ql.row0 : (1 << 30));
    const int R1 = __reduce_max_sync(full, vl ? Ql.row1 : -(1 << 30));
    const int C0 = __reduce_min_sync(full, vl ? Ql.col0 : (1 << 30));
    const int C1 = __reduce_max_sync(full, vl ? Ql.col1 : -(1 << 30));
    // Boxes that wrap around a panorama or reach beyond 45 degrees from a
    // beam's axis need the per-sample wrap and front-hemisphere tests
    // (within 45 degrees in both offsets, d.a >= cos 45 - (1 - cos 45) > 0)
    bool checked = A.panorama != 0;
    {
        const float da = fmaxf(fabsf((float)(Ql.col0 - Ql.ci) - Ql.cf), fabsf((float)(Ql.col1 - Ql.ci) - Ql.cf)) * A.daz;
        const float de = fmaxf(fabsf((float)(Ql.row0 - Ql.ri) - Ql.rf), fabsf((float)(Ql.row1 - Ql.ri) - Ql.rf)) * A.del;
        checked = checked || __any_sync(full, vl && !(da <= 0.78f && de <= 0.78f));
    }
    // Lean form (atomic deposit): the union box, or each beam's own box when
    // that walks at most 4/5 of the union's samples (the union lets lanes on
    // one pixel share its record load), widened to whole warp steps inside
    // the G-buffer; every beam must stay within 45 degrees of every pixel of
    // the box it walks.
    LeanBox LB{};
    bool lean = false;
    if (!TC && G >= 4 && !checked && R0 <= R1) {
        constexpr int kStepL = (kWarp / G) * kSamples;
        const int Wu = (C1 - C0 + kStepL) / kStepL * kStepL;
        const int Hm = __reduce_max_sync(full, vl ? Ql.row1 - Ql.row0 + 1 : 0);
        const int Wm = (__reduce_max_sync(full, vl ? Ql.col1 - Ql.col0 + 1 : 0) + kStepL - 1) / kStepL * kStepL;
        const bool pb = (long)Hm * Wm * 5 < (long)(R1 - R0 + 1) * Wu * 4 && Wm <= A.U && Hm <= A.V;
        if (pb) LB = LeanBox{1, 0, 0, Hm, Wm};
        else LB = LeanBox{0, R0, min(C0, A.U - Wu), R1 - R0 + 1, Wu};
        const int2 o = lean_origin(Ql, LB, A.U, A.V);
        const float da = fmaxf(fabsf((float)(o.x - Ql.ci) - Ql.cf), fabsf((float)(o.x + LB.Wb - 1 - Ql.ci) - Ql.cf)) * A.daz;
        const float de = fmaxf(fabsf((float)(o.y - Ql.ri) - Ql.rf), fabsf((float)(o.y + LB.Hb - 1 - Ql.ri) - Ql.rf)) * A.del;
        lean = LB.Wb <= A.U && __all_sync(full, !vl || (da <= 0.78f && de <= 0.78f));
    }
    // per-(beam, row) sin and cos of the elevation offset and per-row cos(el)
    // (the lean form fills its own table)
    const bool use_rtab = R0 <= R1 && R1 - R0 + 1 <= kRT;
    if (use_rtab && !lean) {
        const int nr = R1 - R0 + 1;
        for (int i = tid; i < G * nr; i += blockDim.x) {
            int jj = i / nr, rr = i - jj * nr;
            const BeamParam &Q = bp[jj];
            float dEl = ((float)(R0 + rr - Q.ri) - Q.rf) * A.del;
            float sv, cv;
            sincosf(dEl, &sv, &cv);
            rtab[jj * kRT + rr] = make_float2(sv, cv);
            if (jj == 0) ctab[rr] = cosf(A.el0 + ((float)(R0 + rr) + 0.5f) * A.del);
        }
    }

    // ---- phase 1: profile-weighted deposits into the range bins -----------
    float amb_acc = 0.f;
    if constexpr (TC) {
        amb_acc = phase1_tc<KIND, G>(A, Ly, hbuf, tab, bp, gcount, R0, R1, C0, C1);
    } else {
        if (lean && LB.pb)
            amb_acc = phase1_lean<KIND, G, true>(A, Ly, hbuf, tab, rtab, ctab, uctr, bp, gcount, LB);
        else if (lean)
            amb_acc = phase1_lean<KIND, G, false>(A, Ly, hbuf, tab, rtab, ctab, uctr, bp, gcount, LB);
        else if (checked)
            amb_acc = phase1_atomic<KIND, G, true>(A, Ly, hbuf, tab, rtab, ctab, uctr, bp, gcount, R0, R1, C0, C1,
                                                   use_rtab);
        else
            amb_acc = phase1_atomic<KIND, G, false>(A, Ly, hbuf, tab, rtab, ctab, uctr, bp, gcount, R0, R1, C0, C1,
                                                    use_rtab);
    }
    if constexpr (TC) {
        // ambient sum per beam: lane (g, t) holds beam g; sum the 4 lanes t
        amb_acc += __shfl_xor_sync(0xffffffffu, amb_acc, 1);
        amb_acc += __shfl_xor_sync(0xffffffffu, amb_acc, 2);
        if ((lane & 3) == 0 && (lane >> 2) < G && amb_acc != 0.f) atomicAdd(amb_s + (lane >> 2), amb_acc);
    } else {
        // ambient sum per beam: lanes j, j+G, j+2G, ... of each warp
#pragma unroll
        for (int o = G; o < kWarp; o <<= 1) amb_acc += __shfl_xor_sync(0xffffffffu, amb_acc, o);
        if (lane < G && amb_acc != 0.f) atomicAdd(amb_s + lane, amb_acc);
    }
    __syncthreads();

    footprint_finish(A, Ly, hbuf, taps, amb_s, supp, tsupp, nrm2_s, tmass_s, bp, b0, gcount, G, 0, G);
}

// Claims a free slot of the echo-only waveform pool. The pool has
// slots_per_sm slots for each SM id below slot_sms; a CTA first tries the
// slots of its own SM, of which at most slots_per_sm - 1 are held by the
// other CTAs resident there, then (another kernel sharing the pool, an SM id
// beyond slot_sms) scans the whole pool. Bounded: -1 after 1024 passes.
__device__ int claim_slot(int *busy, int n, int slot_sms, int per_sm)
{
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    if ((int)smid < slot_sms) {
        for (int k = 0; k < per_sm; ++k) {
            const int s = (int)smid * per_sm + k;
            if (atomicCAS(busy + s, 0, 1) == 0) {
                __threadfence();
                return s;
            }
        }
    }
    const int start = (int)(blockIdx.x % (unsigned)n);
    for (int pass = 0; pass < 1024; ++pass) {
        for (int i = 0; i < n; ++i) {
            const int s = (start + i) % n;
            if (atomicCAS(busy + s, 0, 1) == 0) {
                __threadfence();
                return s;
            }
        }
        __nanosleep(1000);
    }
    return -1;
}

template <int KIND, int G, bool TC>
__global__ void __launch_bounds__(512, TC ? 1 : 2) footprint_wave_kernel(FootprintArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Echo-only: the group's waveforms go to a pooled slot (G rows) instead of
    // the caller's memory, one of its own SM's slots in the common case.
    if (A.slot_pool) {
        if (threadIdx.x == 0) s_wave_slot = claim_slot(A.slot_busy, A.n_slots, A.slot_sms, A.slots_per_sm);
        __syncthreads();
        if (s_wave_slot < 0) {
            if (threadIdx.x == 0) atomicExch(A.err, 1);
            return;
        }
    }
    footprint_group<KIND, G, TC>(A, blockIdx.x, smem_raw);
    if (A.slot_pool) {
        __syncthreads();  // every read of the slot (echo scan) is done
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(A.slot_busy + s_wave_slot, 0);
        }
    }
}

// Batched form: a persistent grid whose CTAs take (frame, group) items, in the
// order of `items`, from a counter that the batch setup kernel resets.
template <int KIND, int G, bool TC>
__global__ void __launch_bounds__(512, TC ? 1 : 2) footprint_batch_kernel(FootprintArgs base, const FrameDesc *frames,
                                                              const int2 *items, int n_items, int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (it >= n_items) break;
        const int2 fg = items[it];
        const FrameDesc F = frames[fg.x];
        FootprintArgs A = base;
        A.U = F.U; A.V = F.V; A.panorama = F.panorama;
        A.az0 = F.az0; A.el0 = F.el0; A.daz = F.daz; A.del = F.del;
        A.rec = F.rec; A.beams = F.beams; A.n_beams = F.n_beams;
        A.wave = F.wave; A.echoes = F.echoes; A.counts = F.counts;
        footprint_group<KIND, G, TC>(A, fg.y, smem_raw);
        __syncthreads();  // shared memory is reused by the next item
    }
}

#include "lidar_deposit_umma.cuh"

size_t umma_smem_bytes(int n_bins, int M) { return umd::um_layout(n_bins, M).total; }

#define GBL_UMMA_EACH(X) X(0, true) X(0, false) X(1, true) X(1, false) X(2, true) X(2, false)

cudaError_t prepare_umma(int kind, bool bf16, size_t smem)
{
#define GBL_CASE(K, B)                                                                                      \
    if (kind == K && bf16 == B) {                                                                           \
        cudaError_t e = cudaFuncSetAttribute(footprint_umma_kernel<K, B>,                                   \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
        if (e != cudaSuccess) return e;                                                                     \
        return cudaFuncSetAttribute(footprint_umma_batch_kernel<K, B>,                                      \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                \
    }
    GBL_UMMA_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_umma(int kind, bool bf16, size_t smem, const FootprintArgs &a, cudaStream_t s)
{
    if (a.n_bins > kUmmaMaxBins || smem < umma_smem_bytes(a.n_bins, a.M)) return cudaErrorInvalidValue;
    const int groups = (a.n_beams + kUmmaBeams - 1) / kUmmaBeams;
    if (groups == 0) return cudaSuccess;
#define GBL_CASE(K, B)                                                                    \
    if (kind == K && bf16 == B) {                                                         \
        footprint_umma_kernel<K, B><<<groups, umd::kUThreads, smem, s>>>(a);              \
        return cudaGetLastError();                                                        \
    }
    GBL_UMMA_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_umma_batch(int kind, bool bf16, int grid, size_t smem, const FootprintArgs &base,
                              const FrameDesc *frames, const int2 *items, int n_items, int *counter, cudaStream_t s)
{
    if (base.n_bins > kUmmaMaxBins || smem < umma_smem_bytes(base.n_bins, base.M)) return cudaErrorInvalidValue;
#define GBL_CASE(K, B)                                                                                      \
    if (kind == K && bf16 == B) {                                                                           \
        footprint_umma_batch_kernel<K, B><<<grid, umd::kUThreads, smem, s>>>(base, frames, items, n_items,  \
                                                                             counter);                      \
        return cudaGetLastError();                                                                          \
    }
    GBL_UMMA_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

size_t footprint_smem_bytes(int G, const FootprintArgs &a)
{
    return make_layout(G, a.n_bins, a.M).total;
}

int footprint_pad(int M) { return make_layout(1, 32, M).pad; }

// Instantiated configurations: profile kind (radial, table, separable) x
// beams per CTA x deposit form. Shared-memory atomics: G in {1, 2, 4, 8, 16}
// (1: scattered beams, e.g. the exact re-run of the tail split); tensor
// cores: G in {4, 8}.
#define GBL_FOR_EACH(X)                                                                                \
    X(0, 1, false) X(0, 2, false) X(0, 4, false) X(0, 8, false) X(0, 16, false) X(1, 1, false)        \
    X(1, 2, false) X(1, 4, false) X(1, 8, false) X(1, 16, false) X(0, 4, true) X(0, 8, true)          \
    X(1, 4, true) X(1, 8, true) X(2, 1, false) X(2, 2, false) X(2, 4, false) X(2, 8, false)           \
    X(2, 16, false) X(2, 4, true) X(2, 8, true)

cudaError_t prepare_footprint(int kind, int G, bool tc, size_t smem)
{
#define GBL_CASE(K, GG, T)                                                                                    \
    if (kind == K && G == GG && tc == T)                                                                      \
        return cudaFuncSetAttribute(footprint_wave_kernel<K, GG, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)smem);
    GBL_FOR_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t footprint_occupancy(int kind, int G, bool tc, int threads, size_t smem, int *blocks_per_sm)
{
#define GBL_CASE(K, GG, T)                                                                                       \
    if (kind == K && G == GG && tc == T)                                                                         \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, footprint_wave_kernel<K, GG, T>, threads, \
                                                             smem);
    GBL_FOR_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

// The shared-memory layout a kernel instantiation uses: a launch with less
// dynamic shared memory is refused.
bool smem_covers_layout(int G, size_t smem, const FootprintArgs &a)
{
    return smem >= make_layout(G, a.n_bins, a.M).total;
}

cudaError_t launch_footprint(int kind, int G, bool tc, int threads, size_t smem, const FootprintArgs &a,
                             cudaStream_t s)
{
    if (!smem_covers_layout(G, smem, a)) return cudaErrorInvalidValue;
    int groups = (a.n_beams + G - 1) / G;
#define GBL_CASE(K, GG, T)                                               \
    if (kind == K && G == GG && tc == T) {                               \
        footprint_wave_kernel<K, GG, T><<<groups, threads, smem, s>>>(a); \
        return cudaGetLastError();                                       \
    }
    GBL_FOR_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t prepare_footprint_batch(int kind, int G, bool tc, size_t smem)
{
#define GBL_CASE(K, GG, T)                                                                          \
    if (kind == K && G == GG && tc == T)                                                            \
        return cudaFuncSetAttribute(footprint_batch_kernel<K, GG, T>,                               \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    GBL_FOR_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_footprint_batch(int kind, int G, bool tc, int threads, int grid, size_t smem,
                                   const FootprintArgs &base, const FrameDesc *frames, const int2 *items,
                                   int n_items, int *counter, cudaStream_t s)
{
    if (!smem_covers_layout(G, smem, base)) return cudaErrorInvalidValue;
#define GBL_CASE(K, GG, T)                                                                                     \
    if (kind == K && G == GG && tc == T) {                                                                     \
        footprint_batch_kernel<K, GG, T><<<grid, threads, smem, s>>>(base, frames, items, n_items, counter); \
        return cudaGetLastError();                                                                             \
    }
    GBL_FOR_EACH(GBL_CASE)
#undef GBL_CASE
    return cudaErrorInvalidValue;
}

}  // namespace gbl
