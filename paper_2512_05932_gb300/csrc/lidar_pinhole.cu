// Reprojection of a pinhole G-buffer onto the spherical grid of the beam model
// (include/lidar.h, lidar_reproject_pinhole). Sec. II-C names reprojection of
// the rendered images as one way to use pinhole renderings; Sec. II-D gives
// the normal-based extrapolation of a pixel's range to another direction,
// r_corr = (p . n) / (v . n) r, which avoids interpolating ranges between
// pixels (that would create ghost points between objects).
//
// One thread per target pixel, 32 x 8 pixels per CTA. The projection and the
// choice of the source cell are FP64, so that the cell a direction falls in is
// decided as an FP64 reference decides it; the FP64 sines and cosines are
// taken once per tile column and row (shared memory); the range correction
// forms p - v and v.n in FP64 and the rest in FP32 (its result is an FP32
// range). A streaming kernel: 7 x 4 bytes written
// per target pixel and at most 7 x 4 bytes gathered from the source.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "lidar.h"
#include "lidar_host.h"

namespace {

struct ReprojArgs {
    // source (pinhole)
    int W, H;
    double fx, fy, cx, cy;
    double R[9];  // camera -> sensor, row-major
    int depth_is_z;
    const float *s_range, *s_nx, *s_ny, *s_nz, *s_rho, *s_retro, *s_amb;
    // target (spherical grid)
    int U, V;
    double az0, el0, daz, del;
    float *d_range, *d_nx, *d_ny, *d_nz, *d_rho, *d_retro, *d_amb;
};

constexpr int kRW = 32, kRH = 8;  // target tile per CTA (one thread per pixel)

__global__ void __launch_bounds__(kRW * kRH) reproject_kernel(ReprojArgs A)
{
    // Per tile: for each column the FP64 azimuth terms and for each row the
    // elevation terms of c = R^T v, v = (cos el cos az, cos el sin az, sin el):
    // c_k = cos(el) (cos(az) R[0][k] + sin(az) R[1][k]) + sin(el) R[2][k].
    __shared__ double colA[kRW][3];
    __shared__ double rowB[kRH][4];  // cos el, sin(el) R[2][k]
    const int tx = threadIdx.x % kRW, ty = threadIdx.x / kRW;
    const int u0 = blockIdx.x * kRW, v0 = blockIdx.y * kRH;
    if (threadIdx.x < kRW) {
        double sa, ca;
        sincos(A.az0 + (u0 + threadIdx.x + 0.5) * A.daz, &sa, &ca);
        for (int k = 0; k < 3; ++k) colA[threadIdx.x][k] = ca * A.R[k] + sa * A.R[3 + k];
    } else if (threadIdx.x < kRW + kRH) {
        const int r = threadIdx.x - kRW;
        double se, ce;
        sincos(A.el0 + (v0 + r + 0.5) * A.del, &se, &ce);
        rowB[r][0] = ce;
        for (int k = 0; k < 3; ++k) rowB[r][1 + k] = se * A.R[6 + k];
    }
    __syncthreads();
    const int u = u0 + tx, v = v0 + ty;
    if (u >= A.U || v >= A.V) return;
    const long idx = (long)v * A.U + u;
    const double ce = rowB[ty][0];
    const double c0 = ce * colA[tx][0] + rowB[ty][1];
    const double c1 = ce * colA[tx][1] + rowB[ty][2];
    const double c2 = ce * colA[tx][2] + rowB[ty][3];
    float o_range = INFINITY, o_nx = 0.f, o_ny = 0.f, o_nz = 0.f, o_rho = 0.f, o_retro = 0.f, o_amb = 0.f;
    if (c2 > 0.0) {
        // the source cell: FP64, as an FP64 reference decides it
        const double inv = 1.0 / c2;
        const double fi = floor(A.cx + A.fx * (c0 * inv)), fj = floor(A.cy + A.fy * (c1 * inv));
        if (fi >= 0.0 && fi < (double)A.W && fj >= 0.0 && fj < (double)A.H) {
            const int i = (int)fi, j = (int)fj;
            const long s = (long)j * A.W + i;
            const float nx = A.s_nx[s], ny = A.s_ny[s], nz = A.s_nz[s];
            o_nx = nx; o_ny = ny; o_nz = nz;
            o_rho = A.s_rho[s]; o_retro = A.s_retro[s]; o_amb = A.s_amb[s];
            const float r = A.s_range[s];
            if (isfinite(r) && r > 0.f) {
                // r_corr = (p.n)/(v.n) r = r (1 + ((p - v).n) / (v.n)): the
                // correction term is small, so it is exact enough in FP32 once
                // p - v (pixel-sized) is formed in FP64 in the camera frame,
                // where v = c and p = (X, Y, 1) / |(X, Y, 1)|
                const double X = (i + 0.5 - A.cx) / A.fx, Y = (j + 0.5 - A.cy) / A.fy;
                const double ip = rsqrt(fma(X, X, fma(Y, Y, 1.0)));
                const float e0 = (float)(X * ip - c0), e1 = (float)(Y * ip - c1), e2 = (float)(ip - c2);
                // normal in the camera frame, R^T n, and v.n in FP64: v.n may be
                // small (grazing incidence), where FP32 would lose its digits
                const double m0 = A.R[0] * nx + A.R[3] * ny + A.R[6] * nz;
                const double m1 = A.R[1] * nx + A.R[4] * ny + A.R[7] * nz;
                const double m2 = A.R[2] * nx + A.R[5] * ny + A.R[8] * nz;
                const float vn = (float)(c0 * m0 + c1 * m1 + c2 * m2);
                const float dn = e0 * (float)m0 + e1 * (float)m1 + e2 * (float)m2;
                const float pn = vn + dn;
                const float rp = A.depth_is_z ? r / (float)ip : r;
                float rc = rp;
                if (fabsf(vn) >= 1e-3f && vn * pn > 0.f) rc = fmaf(rp, dn / vn, rp);
                o_range = rc;
            } else {
                o_range = r;  // no hit (kept as given)
            }
        }
    }
    A.d_range[idx] = o_range;
    A.d_nx[idx] = o_nx;
    A.d_ny[idx] = o_ny;
    A.d_nz[idx] = o_nz;
    A.d_rho[idx] = o_rho;
    A.d_retro[idx] = o_retro;
    A.d_amb[idx] = o_amb;
}

}  // namespace

extern "C" lidar_status_t lidar_reproject_pinhole(const lidar_pinhole_t *src, const lidar_gbuffer_t *dst, void *stream)
{
    using gblh::fail;
    if (!src || !dst) return fail(nullptr, LIDAR_EINVAL, "reproject: src or dst is NULL");
    if (src->W < 1 || src->H < 1 || (long long)src->W * src->H > (1LL << 30))
        return fail(nullptr, LIDAR_EINVAL, "reproject: pinhole size must be 1..2^30 pixels");
    if (!(std::isfinite(src->fx) && src->fx > 0 && std::isfinite(src->fy) && src->fy > 0 && std::isfinite(src->cx) &&
          std::isfinite(src->cy)))
        return fail(nullptr, LIDAR_EINVAL, "reproject: fx, fy must be > 0 and cx, cy finite");
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            // columns of R orthonormal: (R^T R)_ij = delta_ij
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += src->R[3 * k + i] * src->R[3 * k + j];
            if (!(std::fabs(s - (i == j ? 1.0 : 0.0)) <= 1e-3))
                return fail(nullptr, LIDAR_EINVAL, "reproject: R must be orthonormal");
        }
    if (!src->range || !src->nx || !src->ny || !src->nz || !src->rho_d || !src->retro || !src->ambient)
        return fail(nullptr, LIDAR_EINVAL, "reproject: a pinhole plane pointer is NULL");
    if (dst->U < 1 || dst->V < 1 || (long long)dst->U * dst->V > (1LL << 30))
        return fail(nullptr, LIDAR_EINVAL, "reproject: target grid size must be 1..2^30 pixels");
    if (!(std::isfinite(dst->daz) && dst->daz > 0 && std::isfinite(dst->del) && dst->del > 0 &&
          std::isfinite(dst->az0) && std::isfinite(dst->el0)))
        return fail(nullptr, LIDAR_EINVAL, "reproject: target daz, del must be > 0 and az0, el0 finite");
    if (!dst->range || !dst->nx || !dst->ny || !dst->nz || !dst->rho_d || !dst->retro || !dst->ambient)
        return fail(nullptr, LIDAR_EINVAL, "reproject: a target plane pointer is NULL");
    ReprojArgs a{};
    a.W = src->W; a.H = src->H;
    a.fx = src->fx; a.fy = src->fy; a.cx = src->cx; a.cy = src->cy;
    for (int i = 0; i < 9; ++i) a.R[i] = src->R[i];
    a.depth_is_z = src->depth_is_z ? 1 : 0;
    a.s_range = src->range; a.s_nx = src->nx; a.s_ny = src->ny; a.s_nz = src->nz;
    a.s_rho = src->rho_d; a.s_retro = src->retro; a.s_amb = src->ambient;
    a.U = dst->U; a.V = dst->V;
    a.az0 = dst->az0; a.el0 = dst->el0; a.daz = dst->daz; a.del = dst->del;
    // the target planes are written: the struct's pointers are const only for lidar_simulate
    a.d_range = const_cast<float *>(dst->range); a.d_nx = const_cast<float *>(dst->nx);
    a.d_ny = const_cast<float *>(dst->ny); a.d_nz = const_cast<float *>(dst->nz);
    a.d_rho = const_cast<float *>(dst->rho_d); a.d_retro = const_cast<float *>(dst->retro);
    a.d_amb = const_cast<float *>(dst->ambient);
    const dim3 grid((dst->U + kRW - 1) / kRW, (dst->V + kRH - 1) / kRH);
    reproject_kernel<<<grid, kRW * kRH, 0, (cudaStream_t)stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gblh::cuda_fail(nullptr, e, "reprojection kernel launch");
    return LIDAR_OK;
}
