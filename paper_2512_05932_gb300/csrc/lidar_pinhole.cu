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
// taken once per tile column and row (shared memory). The range correction
// needs v.n in FP64 (it may be small) and p - v, which is formed in FP32 from
// exact pixel-sized offsets (see below). A streaming kernel: 7 x 4 bytes
// written per target pixel and at most 7 x 4 bytes gathered from the source.
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
    float inv_fx, inv_fy;
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
    // elevation terms of v = (cos el cos az, cos el sin az, sin el) and of
    // c = R^T v: c_k = cos(el) (cos(az) R[0][k] + sin(az) R[1][k]) + sin(el) R[2][k].
    __shared__ double colA[kRW][5];  // cos(az) R[0][k] + sin(az) R[1][k], cos az, sin az
    __shared__ double rowB[kRH][5];  // cos el, sin(el) R[2][k], sin el
    const int tx = threadIdx.x % kRW, ty = threadIdx.x / kRW;
    const int u0 = blockIdx.x * kRW, v0 = blockIdx.y * kRH;
    if (threadIdx.x < kRW) {
        double sa, ca;
        sincos(A.az0 + (u0 + threadIdx.x + 0.5) * A.daz, &sa, &ca);
        for (int k = 0; k < 3; ++k) colA[threadIdx.x][k] = ca * A.R[k] + sa * A.R[3 + k];
        colA[threadIdx.x][3] = ca;
        colA[threadIdx.x][4] = sa;
    } else if (threadIdx.x < kRW + kRH) {
        const int r = threadIdx.x - kRW;
        double se, ce;
        sincos(A.el0 + (v0 + r + 0.5) * A.del, &se, &ce);
        rowB[r][0] = ce;
        for (int k = 0; k < 3; ++k) rowB[r][1 + k] = se * A.R[6 + k];
        rowB[r][4] = se;
    }
    __syncthreads();
    const int u = u0 + tx, v = v0 + ty;
    if (u >= A.U || v >= A.V) return;
    const long idx = (long)v * A.U + u;
    const double ce = rowB[ty][0];
    const double c0 = fma(ce, colA[tx][0], rowB[ty][1]);
    const double c1 = fma(ce, colA[tx][1], rowB[ty][2]);
    const double c2 = fma(ce, colA[tx][2], rowB[ty][3]);
    float o_range = INFINITY, o_nx = 0.f, o_ny = 0.f, o_nz = 0.f, o_rho = 0.f, o_retro = 0.f, o_amb = 0.f;
    if (c2 > 0.0) {
        // image-plane point (xv, yv) = (c0, c1) / c2 and the source cell: FP64,
        // floor and conversion in one step (saturating far outside the image)
        const double inv = 1.0 / c2;
        const double xv = c0 * inv, yv = c1 * inv;
        const double px = fma(A.fx, xv, A.cx), py = fma(A.fy, yv, A.cy);
        const int i = __double2int_rd(px), j = __double2int_rd(py);
        if (i >= 0 && i < A.W && j >= 0 && j < A.H) {
            const long s = (long)j * A.W + i;
            const float nx = A.s_nx[s], ny = A.s_ny[s], nz = A.s_nz[s];
            o_nx = nx; o_ny = ny; o_nz = nz;
            o_rho = A.s_rho[s]; o_retro = A.s_retro[s]; o_amb = A.s_amb[s];
            const float r = A.s_range[s];
            if (isfinite(r) && r > 0.f) {
                // r_corr = (p.n)/(v.n) r = r (1 + ((p - v).n) / (v.n)).
                // v.n in FP64 (world frame): it may be small (grazing incidence).
                const float vn = (float)fma(ce, fma(colA[tx][3], (double)nx, colA[tx][4] * (double)ny),
                                            rowB[ty][4] * (double)nz);
                // p - v in the camera frame, v = c = c2 (xv, yv, 1) and
                // p = ip (xv + dX, yv + dY, 1), ip = 1 / |(xv + dX, yv + dY, 1)|,
                // with the offsets of the pixel centre dX = (i + 1/2 - px) / fx,
                // dY likewise (exact in FP64, pixel-sized):
                //   p - v = (ip - c2) (xv, yv, 1) + ip (dX, dY, 0),
                //   ip - c2 = -dq (c2 ip)^2 / (c2 + ip), dq = dX (2 xv + dX) + dY (2 yv + dY).
                // Every term is small and free of cancellation, so FP32 keeps
                // p - v to a relative 1e-7.
                const float dX = -(float)(px - (i + 0.5)) * A.inv_fx;
                const float dY = -(float)(py - (j + 0.5)) * A.inv_fy;
                const float xf = (float)xv, yf = (float)yv, c2f = (float)c2;
                const float X = xf + dX, Y = yf + dY;
                const float ip = rsqrtf(fmaf(X, X, fmaf(Y, Y, 1.f)));
                const float dq = fmaf(dX, fmaf(2.f, xf, dX), dY * fmaf(2.f, yf, dY));
                const float cp = c2f * ip;
                const float dip = -dq * (cp * cp) / (c2f + ip);
                const float e0 = fmaf(dip, xf, ip * dX), e1 = fmaf(dip, yf, ip * dY), e2 = dip;
                // normal in the camera frame, R^T n (FP32: it multiplies p - v)
                const float m0 = fmaf((float)A.R[0], nx, fmaf((float)A.R[3], ny, (float)A.R[6] * nz));
                const float m1 = fmaf((float)A.R[1], nx, fmaf((float)A.R[4], ny, (float)A.R[7] * nz));
                const float m2 = fmaf((float)A.R[2], nx, fmaf((float)A.R[5], ny, (float)A.R[8] * nz));
                const float dn = fmaf(e0, m0, fmaf(e1, m1, e2 * m2));
                const float pn = vn + dn;
                const float rp = A.depth_is_z ? r / ip : r;  // z depth -> distance along p
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
    a.inv_fx = (float)(1.0 / src->fx); a.inv_fy = (float)(1.0 / src->fy);
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
