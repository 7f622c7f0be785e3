// Reprojection of a pinhole G-buffer onto the spherical grid of the beam model
// (include/lidar.h, lidar_reproject_pinhole). Sec. II-C names reprojection of
// the rendered images as one way to use pinhole renderings; Sec. II-D gives
// the normal-based extrapolation of a pixel's range to another direction,
// r_corr = (p . n) / (v . n) r, which avoids interpolating ranges between
// pixels (that would create ghost points between objects).
//
// One thread per target pixel, grid-stride. The geometry (direction,
// projection, cell choice, correction) is FP64 so that the cell a direction
// falls in is decided as an FP64 reference decides it; the planes are read
// and written as FP32. A streaming kernel: 7 x 4 bytes written per target
// pixel and at most 7 x 4 bytes gathered from the source.
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

__global__ void __launch_bounds__(256) reproject_kernel(ReprojArgs A)
{
    const long n = (long)A.U * A.V;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        const int v = (int)(idx / A.U), u = (int)(idx - (long)v * A.U);
        double sa, ca, se, ce;
        sincos(A.az0 + (u + 0.5) * A.daz, &sa, &ca);
        sincos(A.el0 + (v + 0.5) * A.del, &se, &ce);
        const double d[3] = {ce * ca, ce * sa, se};  // target direction, sensor frame
        // camera frame: c = R^T d
        const double c0 = A.R[0] * d[0] + A.R[3] * d[1] + A.R[6] * d[2];
        const double c1 = A.R[1] * d[0] + A.R[4] * d[1] + A.R[7] * d[2];
        const double c2 = A.R[2] * d[0] + A.R[5] * d[1] + A.R[8] * d[2];
        float o_range = INFINITY, o_nx = 0.f, o_ny = 0.f, o_nz = 0.f, o_rho = 0.f, o_retro = 0.f, o_amb = 0.f;
        if (c2 > 0.0) {
            const double px = A.cx + A.fx * (c0 / c2), py = A.cy + A.fy * (c1 / c2);
            const double fi = floor(px), fj = floor(py);
            if (fi >= 0.0 && fi < (double)A.W && fj >= 0.0 && fj < (double)A.H) {
                const long s = (long)fj * A.W + (long)fi;
                const double nx = A.s_nx[s], ny = A.s_ny[s], nz = A.s_nz[s];
                o_nx = (float)nx; o_ny = (float)ny; o_nz = (float)nz;
                o_rho = A.s_rho[s]; o_retro = A.s_retro[s]; o_amb = A.s_amb[s];
                const double r = A.s_range[s];
                if (isfinite(r) && r > 0.0) {
                    // source pixel-centre direction p (sensor frame)
                    const double X = (fi + 0.5 - A.cx) / A.fx, Y = (fj + 0.5 - A.cy) / A.fy;
                    const double inv = 1.0 / sqrt(X * X + Y * Y + 1.0);
                    const double p0 = (A.R[0] * X + A.R[1] * Y + A.R[2]) * inv;
                    const double p1 = (A.R[3] * X + A.R[4] * Y + A.R[5]) * inv;
                    const double p2 = (A.R[6] * X + A.R[7] * Y + A.R[8]) * inv;
                    const double rp = A.depth_is_z ? r / inv : r;  // distance along p
                    const double pn = p0 * nx + p1 * ny + p2 * nz;
                    const double vn = d[0] * nx + d[1] * ny + d[2] * nz;
                    double rc = rp;
                    if (fabs(vn) >= 1e-3 && vn * pn > 0.0) rc = pn / vn * rp;
                    o_range = (float)rc;
                } else {
                    o_range = (float)r;  // no hit (kept as given)
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
    const long n = (long)dst->U * dst->V;
    const int grid = (int)std::min<long>((n + 255) / 256, 152L * 16);
    reproject_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gblh::cuda_fail(nullptr, e, "reprojection kernel launch");
    return LIDAR_OK;
}
