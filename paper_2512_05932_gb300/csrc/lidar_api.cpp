// Host side of the C ABI declared in include/lidar.h: argument validation,
// create-time FP64 work (profile normalisation, pulse taps, EPW calibration
// fit), device memory and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <string>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lidar_host.h"
#include "lidar_internal.h"

namespace gblh {

thread_local char g_create_err[512] = "no error";


lidar_status_t fail(lidar_t *l, lidar_status_t st, const char *fmt, ...)
{
    char *buf = l ? l->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

lidar_status_t cuda_fail(lidar_t *l, cudaError_t e, const char *what)
{
    return fail(l, e == cudaErrorMemoryAllocation ? LIDAR_ENOMEM : LIDAR_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// ---------------------------------------------------------------------------
// FP64 profile normalisation: Z = integral of the raw profile over the sphere
// ---------------------------------------------------------------------------

double radial_raw(const lidar_profile_t *p, double th_deg)
{
    if (th_deg > p->trunc_deg) return 0.0;
    double g = std::exp(-0.5 * th_deg * th_deg / (p->sigma_deg * p->sigma_deg));
    double t = th_deg > p->tail_core_deg ? std::pow(th_deg / p->tail_core_deg, -p->tail_pow) : 1.0;
    return g + p->tail_amp * t;
}

// 2 pi int_0^trunc P(theta) sin(theta) dtheta with 8-point Gauss-Legendre on
// 4096 panels per smooth piece (pieces split at the tail core).
double radial_norm(const lidar_profile_t *p)
{
    static const double x8[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double w8[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    double cuts[3] = {0.0, std::min(p->tail_core_deg, p->trunc_deg), p->trunc_deg};
    double acc = 0.0;
    for (int s = 0; s < 2; ++s) {
        double a = cuts[s], b = cuts[s + 1];
        if (!(b > a)) continue;
        const int panels = 4096;
        double h = (b - a) / panels;
        for (int k = 0; k < panels; ++k) {
            double mid = a + (k + 0.5) * h, half = 0.5 * h;
            for (int q = 0; q < 4; ++q)
                for (int sg = -1; sg <= 1; sg += 2) {
                    double th = mid + sg * x8[q] * half;
                    acc += w8[q] * half * radial_raw(p, th) * std::sin(th * kDeg);
                }
        }
    }
    return 2.0 * kPi * acc * kDeg;
}

// Integral of the zero-extended bilinear table times the azimuthal-equidistant
// area element sin(theta)/theta: 3x3 Gauss-Legendre per cell (exact for the
// bilinear part, the area element is smooth).
double table_norm(const lidar_profile_t *p, const std::vector<double> &padded, int pw, int ph)
{
    static const double xg[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};
    static const double wg[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    double pr = p->pitch_deg * kDeg;
    double acc = 0.0;
    for (int j = 0; j + 1 < ph; ++j)
        for (int i = 0; i + 1 < pw; ++i) {
            double t00 = padded[(size_t)j * pw + i], t10 = padded[(size_t)j * pw + i + 1];
            double t01 = padded[(size_t)(j + 1) * pw + i], t11 = padded[(size_t)(j + 1) * pw + i + 1];
            if (t00 == 0 && t10 == 0 && t01 == 0 && t11 == 0) continue;
            for (int qy = 0; qy < 3; ++qy)
                for (int qx = 0; qx < 3; ++qx) {
                    double fx = 0.5 * (1 + xg[qx]), fy = 0.5 * (1 + xg[qy]);
                    double val = (1 - fy) * ((1 - fx) * t00 + fx * t10) + fy * ((1 - fx) * t01 + fx * t11);
                    // padded index i <-> table column i - 1
                    double u = (i + fx - 1 - 0.5 * (p->table_w - 1)) * pr;
                    double v = (j + fy - 1 - 0.5 * (p->table_h - 1)) * pr;
                    double th = std::sqrt(u * u + v * v);
                    double jac = th > 0 ? std::sin(th) / th : 1.0;
                    acc += 0.25 * wg[qx] * wg[qy] * val * jac;
                }
        }
    return acc * pr * pr;
}

// ---------------------------------------------------------------------------
// Pulse taps and the EPW calibration fit (FP64)
// ---------------------------------------------------------------------------

std::vector<double> pulse_taps(const lidar_pulse_t *pu, int *Mout)
{
    double sigma = pu->fwhm_s / (2.0 * std::sqrt(2.0 * std::log(2.0))) / pu->dt_s;
    int M = (int)std::ceil(pu->trunc_sigmas * sigma);
    std::vector<double> t(2 * M + 1);
    double s = 0.0;
    for (int m = -M; m <= M; ++m) s += (t[m + M] = std::exp(-0.5 * (m / sigma) * (m / sigma)));
    for (double &x : t) x /= s;
    *Mout = M;
    return t;
}

// EPW (m) of the single echo of a point target of energy `amp` at bin-centre
// coordinate X (no ambient): the waveform is amp * (hat split of X onto the
// two nearest bins) convolved with the pulse; the echo's edges are the linear
// interpolations of the threshold crossings. Returns < 0 if there is not
// exactly one run above T.
double point_target_epw(const std::vector<double> &taps, int M, int n, double X, double amp, double T, double dt)
{
    int k0 = (int)std::floor(X);
    double f = X - k0;
    std::vector<double> xi(n, 0.0);
    for (int m = -M; m <= M; ++m) {
        int a = k0 + m, b = k0 + 1 + m;
        if (a >= 0 && a < n) xi[a] += amp * (1 - f) * taps[m + M];
        if (b >= 0 && b < n) xi[b] += amp * f * taps[m + M];
    }
    int first = -1, last = -1, runs = 0;
    for (int k = 0; k < n; ++k) {
        bool ab = xi[k] > T;
        if (ab && (k == 0 || !(xi[k - 1] > T))) { ++runs; if (first < 0) first = k; }
        if (ab) last = k;
    }
    if (runs != 1 || first <= 0 || last >= n - 1) return -1.0;
    double x0 = (first - 1) + (T - xi[first - 1]) / (xi[first] - xi[first - 1]);
    double x1 = last + (xi[last] - T) / (xi[last] - xi[last + 1]);
    return (x1 - x0) * dt * kC * 0.5;
}

bool fit_epw(const lidar_pulse_t *pu, double T, double coef[3])
{
    int M = 0;
    std::vector<double> taps = pulse_taps(pu, &M);
    int n = 4 * M + 64;
    // normal equations of ln a = c0 + c1 E^2 + c2 E^4
    double A[3][4] = {{0}};
    int used = 0;
    for (int ia = 0; ia < 64; ++ia) {
        double e = std::log10(50.0) + ia * (6.0 - std::log10(50.0)) / 63.0;
        double amp = T * std::pow(10.0, e);
        for (int ph = 0; ph < 4; ++ph) {
            double E = point_target_epw(taps, M, n, n / 2 + 0.25 * ph, amp, T, pu->dt_s);
            if (E < 0) continue;
            double phi[3] = {1.0, E * E, E * E * E * E};
            double y = std::log(amp);
            for (int r = 0; r < 3; ++r) {
                for (int q = 0; q < 3; ++q) A[r][q] += phi[r] * phi[q];
                A[r][3] += phi[r] * y;
            }
            ++used;
        }
    }
    if (used < 8) return false;
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r) if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        for (int q = 0; q < 4; ++q) std::swap(A[c][q], A[piv][q]);
        if (A[c][c] == 0.0) return false;
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            double f = A[r][c] / A[c][c];
            for (int q = c; q < 4; ++q) A[r][q] -= f * A[c][q];
        }
    }
    for (int r = 0; r < 3; ++r) coef[r] = A[r][3] / A[r][r];
    return std::isfinite(coef[0]) && std::isfinite(coef[1]) && std::isfinite(coef[2]);
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------

lidar_status_t check_create(const lidar_profile_t *p, const lidar_pattern_t *pat, const lidar_pulse_t *pu,
                            const lidar_calib_t *ca)
{
    if (!p || !pat || !pu || !ca) return fail(nullptr, LIDAR_EINVAL, "null parameter struct");
    if (p->kind == LIDAR_PROFILE_RADIAL) {
        if (!finite_pos(p->sigma_deg)) return fail(nullptr, LIDAR_EINVAL, "profile.sigma_deg must be > 0");
        if (!(std::isfinite(p->tail_amp) && p->tail_amp >= 0))
            return fail(nullptr, LIDAR_EINVAL, "profile.tail_amp must be >= 0");
        if (!finite_pos(p->tail_core_deg)) return fail(nullptr, LIDAR_EINVAL, "profile.tail_core_deg must be > 0");
        if (!(std::isfinite(p->tail_pow) && p->tail_pow >= 0))
            return fail(nullptr, LIDAR_EINVAL, "profile.tail_pow must be >= 0");
        if (!finite_pos(p->trunc_deg) || p->trunc_deg > kMaxSupportDeg)
            return fail(nullptr, LIDAR_EINVAL, "profile.trunc_deg must be in (0, 10]");
    } else if (p->kind == LIDAR_PROFILE_TABLE || p->kind == LIDAR_PROFILE_SEPARABLE) {
        if (p->table_w < 2 || p->table_h < 2 || p->table_w > 4096 || p->table_h > 4096)
            return fail(nullptr, LIDAR_EINVAL, "profile table size must be 2..4096 per side");
        if (!p->table) return fail(nullptr, LIDAR_EINVAL, "profile.table is NULL");
        if (!finite_pos(p->pitch_deg)) return fail(nullptr, LIDAR_EINVAL, "profile.pitch_deg must be > 0");
        double hu = (0.5 * (p->table_w - 1) + 1) * p->pitch_deg, hv = (0.5 * (p->table_h - 1) + 1) * p->pitch_deg;
        if (std::sqrt(hu * hu + hv * hv) > kMaxSupportDeg)
            return fail(nullptr, LIDAR_EINVAL, "profile table support exceeds 10 degrees");
        const long nv = p->kind == LIDAR_PROFILE_SEPARABLE ? (long)p->table_w + p->table_h
                                                           : (long)p->table_w * p->table_h;
        for (long i = 0; i < nv; ++i)
            if (!(std::isfinite(p->table[i]) && p->table[i] >= 0.f))
                return fail(nullptr, LIDAR_EINVAL, "profile.table[%ld] is negative or not finite", i);
    } else {
        return fail(nullptr, LIDAR_EINVAL, "profile.kind %d unknown", p->kind);
    }
    if (pat->n_beams < 1) return fail(nullptr, LIDAR_EINVAL, "pattern.n_beams must be >= 1");
    if (!pat->dirs) return fail(nullptr, LIDAR_EINVAL, "pattern.dirs is NULL");
    for (long b = 0; b < pat->n_beams; ++b) {
        const float *d = pat->dirs + 3 * b;
        double n = (double)d[0] * d[0] + (double)d[1] * d[1] + (double)d[2] * d[2];
        if (!(std::isfinite(n) && n > 1e-20))
            return fail(nullptr, LIDAR_EINVAL, "pattern.dirs[%ld] is zero or not finite", b);
    }
    if (pu->n_bins < 32 || pu->n_bins > gbl::kMaxBins || pu->n_bins % 32 != 0)
        return fail(nullptr, LIDAR_EINVAL, "pulse.n_bins must be a multiple of 32 in [32, %d]", gbl::kMaxBins);
    if (!finite_pos(pu->dt_s)) return fail(nullptr, LIDAR_EINVAL, "pulse.dt_s must be > 0");
    if (!std::isfinite(pu->t0_s)) return fail(nullptr, LIDAR_EINVAL, "pulse.t0_s must be finite");
    if (!finite_pos(pu->fwhm_s)) return fail(nullptr, LIDAR_EINVAL, "pulse.fwhm_s must be > 0");
    if (!finite_pos(pu->trunc_sigmas) || pu->trunc_sigmas > 12)
        return fail(nullptr, LIDAR_EINVAL, "pulse.trunc_sigmas must be in (0, 12]");
    double sigma = pu->fwhm_s / (2.0 * std::sqrt(2.0 * std::log(2.0))) / pu->dt_s;
    if (std::ceil(pu->trunc_sigmas * sigma) > 2048)
        return fail(nullptr, LIDAR_EINVAL, "pulse support exceeds 2048 bins");
    if (!finite_pos(ca->threshold)) return fail(nullptr, LIDAR_EINVAL, "calib.threshold must be > 0");
    if (!(std::isfinite(ca->ambient_scale) && ca->ambient_scale >= 0))
        return fail(nullptr, LIDAR_EINVAL, "calib.ambient_scale must be >= 0");
    if (ca->max_echoes < 1 || ca->max_echoes > 3) return fail(nullptr, LIDAR_EINVAL, "calib.max_echoes must be 1..3");
    if (!ca->fit_epw)
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(ca->epw_coef[i])) return fail(nullptr, LIDAR_EINVAL, "calib.epw_coef not finite");
    return LIDAR_OK;
}

lidar_status_t check_gbuffer(lidar_t *l, const lidar_gbuffer_t *g)
{
    if (!g) return fail(l, LIDAR_EINVAL, "gbuffer is NULL");
    if (g->U < 1 || g->V < 1) return fail(l, LIDAR_EINVAL, "gbuffer U, V must be >= 1");
    if ((long long)g->U * g->V > (1LL << 30)) return fail(l, LIDAR_EINVAL, "gbuffer has more than 2^30 pixels");
    if (!finite_pos(g->daz) || !finite_pos(g->del) || !std::isfinite(g->az0) || !std::isfinite(g->el0))
        return fail(l, LIDAR_EINVAL, "gbuffer angles must be finite with daz, del > 0");
    if (g->U * g->daz > 2 * kPi * (1 + 1e-9)) return fail(l, LIDAR_EINVAL, "gbuffer azimuth span exceeds 2 pi");
    if (g->el0 < -0.5 * kPi - 1e-9 || g->el0 + g->V * g->del > 0.5 * kPi + 1e-9)
        return fail(l, LIDAR_EINVAL, "gbuffer elevation span leaves [-pi/2, pi/2]");
    if (!g->range || !g->nx || !g->ny || !g->nz || !g->rho_d || !g->retro || !g->ambient)
        return fail(l, LIDAR_EINVAL, "gbuffer plane pointer is NULL");
    return LIDAR_OK;
}

lidar_status_t check_pose(lidar_t *l, const lidar_pose_t *p, double R[9])
{
    static const double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (!p) { std::memcpy(R, I, sizeof I); return LIDAR_OK; }
    for (int i = 0; i < 9; ++i) {
        R[i] = p->R[i];
        if (!std::isfinite(R[i])) return fail(l, LIDAR_EINVAL, "pose.R not finite");
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[3 * k + a] * R[3 * k + b];
            if (std::fabs(s - (a == b)) > 1e-3) return fail(l, LIDAR_EINVAL, "pose.R is not orthonormal");
        }
    double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) + R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (det < 0) return fail(l, LIDAR_EINVAL, "pose.R is a reflection");
    return LIDAR_OK;
}

lidar_status_t ensure_scratch(lidar_t *l, size_t pixels)
{
    if (pixels <= l->rec_cap) return LIDAR_OK;
    if (l->d_rec) cudaFree(l->d_rec);
    l->d_rec = nullptr;
    l->rec_cap = 0;
    cudaError_t e = cudaMalloc(&l->d_rec, pixels * 2 * sizeof(float4));
    if (e != cudaSuccess) return cuda_fail(l, e, "cudaMalloc(per-pixel records)");
    l->rec_cap = pixels;
    return LIDAR_OK;
}

void free_events(lidar_t *l)
{
    for (cudaEvent_t e : l->ev) cudaEventDestroy(e);
    l->ev.clear();
    l->ev_used = 0;
}

// Returns the next event of the profiling pool (creating it if needed), or
// nullptr when profiling is off.
cudaEvent_t next_event(lidar_t *l)
{
    if (!l->prof) return nullptr;
    if (l->ev_used == l->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        l->ev.push_back(e);
    }
    return l->ev[l->ev_used++];
}

void free_batch(lidar_t *l)
{
    if (l->gexec) cudaGraphExecDestroy(l->gexec);
    l->gexec = nullptr;
    l->gkey.clear();
    cudaFree(l->d_brec);
    cudaFree(l->d_bbeams);
    cudaFree(l->d_blob);
    cudaFreeHost(l->h_blob);
    cudaFree(l->d_counter);
    if (l->cap_stream) cudaStreamDestroy(l->cap_stream);
    if (l->blob_free) cudaEventDestroy(l->blob_free);
    l->d_brec = nullptr; l->d_bbeams = nullptr; l->d_blob = nullptr; l->h_blob = nullptr; l->d_counter = nullptr;
    l->cap_stream = nullptr; l->blob_free = nullptr;
    l->brec_cap = l->bbeams_cap = l->blob_cap = 0;
}

void free_all(lidar_t *l)
{
    free_batch(l);
    free_events(l);
    cudaFree(l->d_wmax);
    cudaFree(l->d_perm);
    cudaFree(l->d_dirs);
    if (l->node_tex) cudaDestroyTextureObject(l->node_tex);
    if (l->d_nodes) cudaFreeArray(l->d_nodes);
    cudaFree(l->d_pairs);
    cudaFree(l->d_taps);
    cudaFree(l->d_beams);
    cudaFree(l->d_rec);
    cudaFree(l->d_planes);
    cudaFree(l->d_wave);
    cudaFree(l->d_echo);
    cudaFree(l->d_counts);
    cudaFree(l->d_rec2);
    cudaFree(l->d_beams2);
    cudaFree(l->d_planes2);
    cudaFree(l->d_wave2);
    cudaFree(l->d_echo2);
    cudaFree(l->d_counts2);
    cudaFree(l->d_slot_pool);
    cudaFree(l->d_slot_busy);
    cudaFree(l->d_err);
    if (l->copy_stream) cudaStreamDestroy(l->copy_stream);
    for (cudaStream_t &st : l->aux_stream)
        if (st) cudaStreamDestroy(st);
    if (l->setup_stream) cudaStreamDestroy(l->setup_stream);
    for (cudaStream_t &st : l->d2h_stream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t &ev : l->chunk_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t &ev : l->setup_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t &ev : l->band_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t &ev : l->join_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &set : l->done_ev)
        for (cudaEvent_t &ev : set)
            if (ev) cudaEventDestroy(ev);
    if (l->start_ev) cudaEventDestroy(l->start_ev);
    tail_free(l);
}

bool is_panorama(const lidar_gbuffer_t *g) { return std::fabs(g->U * g->daz - 2 * kPi) <= 1e-6; }

// Setup-kernel arguments of one frame (geometry, planes, pose, scratch).
gbl::SetupArgs setup_args(const lidar_t *l, const lidar_t *sensor, const lidar_gbuffer_t *g, const double R[9],
                          float4 *rec, gbl::BeamParam *beams)
{
    gbl::SetupArgs sa{};
    size_t pixels = (size_t)g->U * g->V;
    sa.U = g->U; sa.V = g->V;
    sa.az0 = (float)g->az0; sa.el0 = (float)g->el0; sa.daz = (float)g->daz; sa.del = (float)g->del;
    sa.ch = (float)std::cos(0.5 * g->daz); sa.sh = (float)std::sin(0.5 * g->daz);
    sa.cv = (float)std::cos(0.5 * g->del); sa.sv = (float)std::sin(0.5 * g->del);
    sa.range = g->range; sa.nx = g->nx; sa.ny = g->ny; sa.nz = g->nz;
    sa.rho = g->rho_d; sa.retro = g->retro; sa.amb = g->ambient;
    sa.rec = rec;
    sa.x_scale = (float)(2.0 / (kC * l->dt));
    sa.x_off = (float)(-l->t0 / l->dt - 0.5);
    {
        const double xs = 2.0 / (kC * l->dt), xo = -l->t0 / l->dt - 0.5;
        sa.xs_hi = (float)xs;
        sa.xs_lo = (float)(xs - (double)sa.xs_hi);
        sa.xo_int = (float)std::floor(xo);
        sa.xo_fr = (float)(xo - std::floor(xo));
        sa.vh = (float)(2.0 * std::sin(0.25 * g->daz) * std::sin(0.25 * g->daz));
        sa.vv = (float)(2.0 * std::sin(0.25 * g->del) * std::sin(0.25 * g->del));
    }
    sa.n_bins = l->n_bins;
    sa.pad = gbl::footprint_pad(l->M);
    long pb = (long)((pixels + 255) / 256);
    sa.pix_blocks = (int)std::min<long>(pb, 152L * 64);
    sa.pix_begin = 0;
    sa.pix_end = (long)pixels;
    sa.n_beams = sensor->n_beams;
    sa.dirs = sensor->d_dirs;
    for (int i = 0; i < 9; ++i) sa.R[i] = R[i];
    sa.az0d = g->az0; sa.el0d = g->el0; sa.dazd = g->daz; sa.deld = g->del;
    sa.panorama = is_panorama(g) ? 1 : 0;
    sa.support_rad = l->support_rad;
    sa.sup_u = l->sup_u;
    sa.sup_v = l->sup_v;
    sa.cos_sup = std::cos(l->support_rad);
    sa.beams = beams;
    sa.bin_records = l->deposit != 0 ? 1 : 0;
    return sa;
}

// Footprint-kernel arguments that depend on the sensor model only.
gbl::FootprintArgs model_args(const lidar_t *l)
{
    gbl::FootprintArgs fa{};
    fa.kg = l->kg; fa.trunc2 = l->trunc2; fa.tail_amp = l->tail_amp; fa.tc2_inv = l->tc2_inv; fa.tail_hp = l->tail_hp;
    fa.invZ = (float)(1.0 / l->Z);
    fa.nodes = l->node_tex; fa.qw = l->qw; fa.qh = l->qh;
    fa.hpairs = l->d_pairs;
    fa.vpairs = l->d_pairs ? l->d_pairs + l->qw : nullptr;
    fa.tk = l->tk;
    fa.tiu = std::floor(l->tcu); fa.tiv = std::floor(l->tcv);
    fa.tcu = l->tcu - fa.tiu; fa.tcv = l->tcv - fa.tiv;
    fa.tiu1 = fa.tiu + 1.f; fa.tiv1 = fa.tiv + 1.f;
    fa.n_bins = l->n_bins; fa.nch = l->n_bins / 32; fa.M = l->M; fa.R = l->R;
    fa.taps_pad = l->d_taps; fa.tp_len = l->tp_len; fa.tp_off = l->tp_off;
    fa.T = (float)l->T; fa.s_amb = (float)l->s_amb; fa.max_echoes = l->max_echoes;
    fa.strongest = l->echo_mode == LIDAR_ECHOES_STRONGEST ? 1 : 0;
    fa.c0 = (float)l->coef[0]; fa.c1 = (float)l->coef[1]; fa.c2 = (float)l->coef[2];
    fa.rA = (float)(0.5 * kC * (l->t0 + 0.5 * l->dt));
    fa.rB = (float)(0.5 * kC * l->dt);
    fa.tc_split = l->deposit == 1 ? 1 : 0;
    fa.umma_pmax = (float)l->pmax;
    fa.umma_wmax = nullptr;
    fa.inner2 = -1.f;  // no annulus: the whole profile
    return fa;
}

// SM ids covered by per-SM slots of the echo-only pool (ids of enabled SMs
// need not be contiguous; a CTA on a higher id takes any free slot).
constexpr int kSlotSms = 256;

// Waveform pool of the echo-only path: a slot of G rows for every CTA of the
// footprint kernel that an SM can hold at once, for SM ids 0..kSlotSms-1
// (grown with cudaMalloc).
lidar_status_t ensure_slots(lidar_t *l, int G, bool tc)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = gbl::footprint_occupancy(l->kind, G, tc, l->threads, tc ? l->smem_tc : l->smem, &per_sm)) != cudaSuccess)
        return cuda_fail(l, e, "footprint occupancy");
    (void)sms;
    per_sm = std::max(1, per_sm);
    const int n = kSlotSms * per_sm;
    const size_t need = (size_t)n * G * l->n_bins;
    if (n == l->n_slots && per_sm == l->slots_per_sm && need == l->slot_floats) return LIDAR_OK;
    cudaFree(l->d_slot_pool);
    cudaFree(l->d_slot_busy);
    l->d_slot_pool = nullptr;
    l->d_slot_busy = nullptr;
    l->n_slots = 0;
    l->slot_floats = 0;
    if ((e = cudaMalloc(&l->d_slot_pool, need * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&l->d_slot_busy, (size_t)n * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(l->d_slot_busy, 0, (size_t)n * sizeof(int))) != cudaSuccess ||
        (!l->d_err && (e = cudaMalloc(&l->d_err, sizeof(int))) != cudaSuccess) ||
        (e = cudaMemset(l->d_err, 0, sizeof(int))) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
        return cuda_fail(l, e, "cudaMalloc(echo-only waveform pool)");
    l->n_slots = n;
    l->slots_per_sm = per_sm;
    l->slot_floats = need;
    return LIDAR_OK;
}

// Footprint-kernel arguments of one frame (outputs not set).
gbl::FootprintArgs frame_args(const lidar_t *l, const lidar_gbuffer_t *g, const gbl::SetupArgs &sa)
{
    gbl::FootprintArgs fa = model_args(l);
    fa.U = g->U; fa.V = g->V; fa.panorama = sa.panorama;
    fa.az0 = sa.az0; fa.el0 = sa.el0; fa.daz = sa.daz; fa.del = sa.del;
    fa.rec = l->d_rec;
    fa.beams = l->d_beams;
    fa.n_beams = l->n_beams;
    return fa;
}

// Order of the beams for the tcgen05 deposit's groups of 16: beams in bands
// of height s of the pattern's (azimuth * cos(elevation), elevation) plane,
// each band by azimuth, s the side of the square that holds 16 beams at the
// pattern's mean density. Consecutive slots are then near each other in both
// directions (a grid gives groups of about 4 x 4 beams; a line scan whose rows
// are farther apart than s keeps its rows), which keeps a group's union pixel
// box close to one beam's.
std::vector<int32_t> group_order(const lidar_t *l)
{
    const int n = l->n_beams;
    std::vector<double> x(n), y(n);
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int b = 0; b < n; ++b) {
        const double dx = l->h_dirs[3 * b], dy = l->h_dirs[3 * b + 1], dz = l->h_dirs[3 * b + 2];
        const double el = std::asin(std::max(-1.0, std::min(1.0, dz)));
        y[b] = el;
        x[b] = std::atan2(dy, dx) * std::cos(el);
        x0 = std::min(x0, x[b]); x1 = std::max(x1, x[b]);
        y0 = std::min(y0, y[b]); y1 = std::max(y1, y[b]);
    }
    std::vector<int32_t> order(n);
    for (int b = 0; b < n; ++b) order[b] = b;
    const double area = std::max(x1 - x0, 1e-9) * std::max(y1 - y0, 1e-9);
    const double side = 4.0 * std::sqrt(area / std::max(n, 1));
    std::vector<long> band(n);
    for (int b = 0; b < n; ++b) band[b] = (long)std::floor((y[b] - y0) / std::max(side, 1e-12));
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
        if (band[a] != band[c]) return band[a] < band[c];
        return x[a] < x[c];
    });
    return order;
}

// One frame with the tcgen05 deposit: the setup kernel (with the frame's
// largest record weight for FP16 operands) and the tensor-core footprint kernel.
lidar_status_t enqueue_umma(lidar_t *l, const lidar_gbuffer_t *g, const double R[9], float *wave,
                            lidar_echo_t *echoes, int32_t *counts, cudaStream_t s)
{
    const bool bf16 = l->deposit == LIDAR_DEPOSIT_TCGEN05_BF16;
    lidar_status_t st = ensure_scratch(l, (size_t)g->U * g->V);
    if (st != LIDAR_OK) return st;
    gbl::SetupArgs sa = setup_args(l, l, g, R, l->d_rec, l->d_beams);
    sa.beam_ids = l->d_perm;  // beam slots in group order
    cudaError_t e;
    if (!bf16) {
        sa.wmax = l->d_wmax;
        if ((e = cudaMemsetAsync(l->d_wmax, 0, sizeof(unsigned), s)) != cudaSuccess)
            return cuda_fail(l, e, "cudaMemsetAsync(weight maximum)");
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    if (l->prof) {
        size_t mark = l->ev_used;
        ev0 = next_event(l); ev1 = next_event(l); ev2 = next_event(l);
        if (!ev0 || !ev1 || !ev2) { l->ev_used = mark; ev0 = ev1 = ev2 = nullptr; }
    }
    if (ev0) cudaEventRecord(ev0, s);
    if ((e = gbl::launch_setup(sa, s)) != cudaSuccess) return cuda_fail(l, e, "setup kernel launch");
    if (ev1) cudaEventRecord(ev1, s);
    gbl::FootprintArgs fa = frame_args(l, g, sa);
    fa.wave = wave; fa.echoes = echoes; fa.counts = counts;
    fa.err = l->d_err;
    fa.out_ids = l->d_perm;  // slot b writes the outputs of pattern beam d_perm[b]
    fa.umma_wmax = bf16 ? nullptr : l->d_wmax;
    if ((e = gbl::launch_umma(l->kind, bf16, l->smem_um, fa, s)) != cudaSuccess)
        return cuda_fail(l, e, "tcgen05 footprint kernel launch");
    if (ev2) cudaEventRecord(ev2, s);
    return LIDAR_OK;
}

// Enqueues the setup and footprint kernels of one frame on `s`; wave == NULL
// selects the echo-only form (waveforms in the pooled slots).
lidar_status_t enqueue(lidar_t *l, const lidar_gbuffer_t *g, const double R[9], float *wave, lidar_echo_t *echoes,
                       int32_t *counts, cudaStream_t s)
{
    if (l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16) {
        if (!wave) return fail(l, LIDAR_EINVAL, "the tcgen05 deposit has no echo-only form");
        return enqueue_umma(l, g, R, wave, echoes, counts, s);
    }
    const bool tc = l->deposit != 0;
    if (!wave) {
        lidar_status_t st0 = ensure_slots(l, tc ? l->G_tc : l->G, tc);
        if (st0 != LIDAR_OK) return st0;
    }
    size_t pixels = (size_t)g->U * g->V;
    lidar_status_t st = ensure_scratch(l, pixels);
    if (st != LIDAR_OK) return st;
    gbl::SetupArgs sa = setup_args(l, l, g, R, l->d_rec, l->d_beams);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    if (l->prof) {
        size_t mark = l->ev_used;
        ev0 = next_event(l); ev1 = next_event(l); ev2 = next_event(l);
        if (!ev0 || !ev1 || !ev2) { l->ev_used = mark; ev0 = ev1 = ev2 = nullptr; }
    }
    if (ev0) cudaEventRecord(ev0, s);
    cudaError_t e = cudaSuccess;
    e = gbl::launch_setup(sa, s);
    if (e != cudaSuccess) return cuda_fail(l, e, "setup kernel launch");
    if (ev1) cudaEventRecord(ev1, s);

    gbl::FootprintArgs fa = frame_args(l, g, sa);
    fa.wave = wave; fa.echoes = echoes; fa.counts = counts;
    if (!wave) {
        fa.slot_pool = l->d_slot_pool;
        fa.slot_busy = l->d_slot_busy;
        fa.n_slots = l->n_slots;
        fa.slot_sms = kSlotSms;
        fa.slots_per_sm = l->slots_per_sm;
        fa.err = l->d_err;
    }
    const int G = tc ? l->G_tc : l->G;
    e = gbl::launch_footprint(l->kind, G, tc, l->threads, tc ? l->smem_tc : l->smem, fa, s);
    if (e != cudaSuccess) return cuda_fail(l, e, "footprint kernel launch");
    if (ev2) cudaEventRecord(ev2, s);
    return LIDAR_OK;
}

// ---------------------------------------------------------------------------
// batched execution
// ---------------------------------------------------------------------------

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
lidar_status_t grow(lidar_t *l, T **p, size_t *cap, size_t need, const char *what)
{
    if (need <= *cap) return LIDAR_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, need * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(l, e, what);
    *cap = need;
    return LIDAR_OK;
}

// Builds the descriptor blob of a batch (host copy) and returns its layout.
struct BlobLayout {
    size_t off_setup, off_pix, off_beam, off_frames, off_items, off_wmax, size;
    int n_items, total_blocks;
};

lidar_status_t batch_validate(lidar_t *l, const lidar_frame_t *fr, int n, std::vector<std::array<double, 9>> &Rs)
{
    if (!fr || n < 1) return fail(l, LIDAR_EINVAL, "batch needs at least one frame");
    Rs.resize(n);
    for (int f = 0; f < n; ++f) {
        const lidar_frame_t &F = fr[f];
        if (!F.sensor) return fail(l, LIDAR_EINVAL, "frame %d: sensor is NULL", f);
        if (F.sensor->model_hash != l->model_hash)
            return fail(l, LIDAR_EINVAL, "frame %d: sensor model differs from the executor's", f);
        lidar_status_t st = check_gbuffer(l, &F.gbuffer);
        if (st != LIDAR_OK) return fail(l, st, "frame %d: %s", f, std::string(l->err).c_str());
        if ((st = check_pose(l, &F.pose, Rs[f].data())) != LIDAR_OK) return fail(l, st, "frame %d: %s", f, std::string(l->err).c_str());
        if (!F.out_waveforms || !F.out_echoes.echoes || !F.out_echoes.counts)
            return fail(l, LIDAR_EINVAL, "frame %d: output pointer is NULL", f);
    }
    return LIDAR_OK;
}

lidar_status_t batch_run(lidar_t *l, const lidar_frame_t *fr, int n, cudaStream_t s, int G, int cps)
{
    std::vector<std::array<double, 9>> Rs;
    lidar_status_t st = batch_validate(l, fr, n, Rs);
    if (st != LIDAR_OK) return st;
    cudaError_t e;
    if (!l->cap_stream) {
        if ((e = cudaStreamCreateWithFlags(&l->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(l, e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&l->blob_free, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(l, e, "cudaEventCreate");
        if ((e = cudaMalloc(&l->d_counter, sizeof(int))) != cudaSuccess) return cuda_fail(l, e, "cudaMalloc(counter)");
    }
    // scratch for all frames
    size_t tot_pix = 0, tot_beams = 0;
    std::vector<size_t> pix_off(n), beam_off(n);
    for (int f = 0; f < n; ++f) {
        pix_off[f] = tot_pix;
        beam_off[f] = tot_beams;
        tot_pix += (size_t)fr[f].gbuffer.U * fr[f].gbuffer.V;
        tot_beams += (size_t)fr[f].sensor->n_beams;
    }
    if ((st = grow(l, &l->d_brec, &l->brec_cap, 2 * tot_pix, "cudaMalloc(batch records)")) != LIDAR_OK) return st;
    if ((st = grow(l, &l->d_bbeams, &l->bbeams_cap, tot_beams, "cudaMalloc(batch beams)")) != LIDAR_OK) return st;
    // items: (frame, group), frames with the widest footprints (pixels per beam) first
    std::vector<int> order(n);
    for (int f = 0; f < n; ++f) order[f] = f;
    auto cost = [&](int f) {
        const lidar_gbuffer_t &g = fr[f].gbuffer;
        return l->support_rad * l->support_rad / (g.daz * g.del);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    const bool um = l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16;
    if (um) G = gbl::kUmmaBeams;
    else if (l->deposit != 0 && G != 4 && G != 8) G = l->G_tc;
    std::vector<int2> items;
    for (int f : order) {
        int groups = (fr[f].sensor->n_beams + G - 1) / G;
        for (int g = 0; g < groups; ++g) items.push_back(make_int2(f, g));
    }
    BlobLayout B;
    B.off_setup = 0;
    B.off_pix = align16(B.off_setup + n * sizeof(gbl::SetupArgs));
    B.off_beam = align16(B.off_pix + (n + 1) * sizeof(int));
    B.off_frames = align16(B.off_beam + (n + 1) * sizeof(int));
    B.off_items = align16(B.off_frames + n * sizeof(gbl::FrameDesc));
    B.off_wmax = align16(B.off_items + items.size() * sizeof(int2));
    B.size = align16(B.off_wmax + n * sizeof(unsigned));
    B.n_items = (int)items.size();
    // the previous batch's graph may still be reading the pinned staging copy
    if (l->blob_pending) {
        if ((e = cudaEventSynchronize(l->blob_free)) != cudaSuccess) return cuda_fail(l, e, "cudaEventSynchronize");
        l->blob_pending = false;
    }
    if (B.size > l->blob_cap) {
        if (l->gexec) { cudaGraphExecDestroy(l->gexec); l->gexec = nullptr; l->gkey.clear(); }
        cudaFree(l->d_blob);
        cudaFreeHost(l->h_blob);
        l->d_blob = nullptr; l->h_blob = nullptr; l->blob_cap = 0;
        size_t cap = B.size * 2;
        if ((e = cudaMalloc(&l->d_blob, cap)) != cudaSuccess) return cuda_fail(l, e, "cudaMalloc(batch descriptors)");
        if ((e = cudaMallocHost(&l->h_blob, cap)) != cudaSuccess) return cuda_fail(l, e, "cudaMallocHost(batch descriptors)");
        l->blob_cap = cap;
    }
    unsigned char *hb = l->h_blob;
    gbl::SetupArgs *hs = reinterpret_cast<gbl::SetupArgs *>(hb + B.off_setup);
    int *hpix = reinterpret_cast<int *>(hb + B.off_pix);
    int *hbeam = reinterpret_cast<int *>(hb + B.off_beam);
    gbl::FrameDesc *hf = reinterpret_cast<gbl::FrameDesc *>(hb + B.off_frames);
    int pb = 0, bb = 0;
    for (int f = 0; f < n; ++f) {
        const lidar_frame_t &F = fr[f];
        float4 *rec = l->d_brec + 2 * pix_off[f];
        gbl::BeamParam *bp = l->d_bbeams + beam_off[f];
        hs[f] = setup_args(l, F.sensor, &F.gbuffer, Rs[f].data(), rec, bp);
        hpix[f] = pb;
        hbeam[f] = bb;
        pb += (int)(((size_t)F.gbuffer.U * F.gbuffer.V + 255) / 256);
        bb += (F.sensor->n_beams + 255) / 256;
        gbl::FrameDesc D{};
        D.U = F.gbuffer.U; D.V = F.gbuffer.V; D.panorama = hs[f].panorama; D.n_beams = F.sensor->n_beams;
        D.az0 = hs[f].az0; D.el0 = hs[f].el0; D.daz = hs[f].daz; D.del = hs[f].del;
        D.rec = rec; D.beams = bp;
        D.wave = F.out_waveforms; D.echoes = F.out_echoes.echoes; D.counts = F.out_echoes.counts;
        if (l->deposit == LIDAR_DEPOSIT_TCGEN05_FP16) {
            // the frame's largest record weight: zero in the uploaded blob, maximised by the setup kernel
            unsigned *wm = reinterpret_cast<unsigned *>(l->d_blob + B.off_wmax) + f;
            hs[f].wmax = wm;
            D.wmax = wm;
        }
        hf[f] = D;
    }
    std::memset(hb + B.off_wmax, 0, n * sizeof(unsigned));
    hpix[n] = pb;
    hbeam[n] = bb;
    B.total_blocks = pb + bb;
    std::memcpy(hb + B.off_items, items.data(), items.size() * sizeof(int2));

    // persistent grid size
    const bool tc = l->deposit != 0 && !um;
    if (tc && G != 4 && G != 8) G = l->G_tc;  // tensor-core form: 4 or 8 beams per CTA
    size_t smem = um ? l->smem_um : gbl::footprint_smem_bytes(G, model_args(l));
    if (!um && (e = gbl::prepare_footprint_batch(l->kind, G, tc, smem)) != cudaSuccess)
        return cuda_fail(l, e, "cudaFuncSetAttribute");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, l->device);
    int per_sm = um ? 1 : (cps > 0 ? cps : 2);  // tcgen05: one CTA per SM (its tensor memory)
    int grid = std::max(1, std::min(B.n_items, per_sm * sms));

    // graph keyed on everything the captured launches depend on
    std::vector<long long> key = {n, (long long)B.size, B.n_items, B.total_blocks, G, grid, (long long)smem, l->deposit,
                                  (long long)(uintptr_t)l->d_blob, (long long)(uintptr_t)l->h_blob};
    if (!l->gexec || key != l->gkey) {
        if (l->gexec) { cudaGraphExecDestroy(l->gexec); l->gexec = nullptr; }
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(l->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(l, e, "cudaStreamBeginCapture");
        cudaError_t e1 = cudaMemcpyAsync(l->d_blob, l->h_blob, B.size, cudaMemcpyHostToDevice, l->cap_stream);
        const unsigned char *db = l->d_blob;
        cudaError_t e2 = gbl::launch_setup_batch(reinterpret_cast<const gbl::SetupArgs *>(db + B.off_setup),
                                                 reinterpret_cast<const int *>(db + B.off_pix),
                                                 reinterpret_cast<const int *>(db + B.off_beam), n, B.total_blocks,
                                                 l->d_counter, l->cap_stream);
        gbl::FootprintArgs base = model_args(l);
        cudaError_t e3;
        if (um) {
            base.err = l->d_err;
            e3 = gbl::launch_umma_batch(l->kind, l->deposit == LIDAR_DEPOSIT_TCGEN05_BF16, grid, smem, base,
                                        reinterpret_cast<const gbl::FrameDesc *>(db + B.off_frames),
                                        reinterpret_cast<const int2 *>(db + B.off_items), B.n_items, l->d_counter,
                                        l->cap_stream);
        } else {
            e3 = gbl::launch_footprint_batch(l->kind, G, tc, l->threads, grid, smem, base,
                                             reinterpret_cast<const gbl::FrameDesc *>(db + B.off_frames),
                                             reinterpret_cast<const int2 *>(db + B.off_items), B.n_items,
                                             l->d_counter, l->cap_stream);
        }
        e = cudaStreamEndCapture(l->cap_stream, &graph);
        if (e1 != cudaSuccess) return cuda_fail(l, e1, "descriptor upload capture");
        if (e2 != cudaSuccess) return cuda_fail(l, e2, "batch setup launch capture");
        if (e3 != cudaSuccess) return cuda_fail(l, e3, "batch footprint launch capture");
        if (e != cudaSuccess) return cuda_fail(l, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&l->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { l->gexec = nullptr; return cuda_fail(l, e, "cudaGraphInstantiate"); }
        l->gkey = key;
    }
    if ((e = cudaGraphLaunch(l->gexec, s)) != cudaSuccess) return cuda_fail(l, e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(l->blob_free, s)) != cudaSuccess) return cuda_fail(l, e, "cudaEventRecord");
    l->blob_pending = true;
    return LIDAR_OK;
}

}  // namespace gblh

using namespace gblh;

extern "C" {

lidar_status_t lidar_create(const lidar_profile_t *p, const lidar_pattern_t *pat, const lidar_pulse_t *pu,
                            const lidar_calib_t *ca, lidar_t **out)
{
    if (!out) return fail(nullptr, LIDAR_EINVAL, "out is NULL");
    *out = nullptr;
    lidar_status_t st = check_create(p, pat, pu, ca);
    if (st != LIDAR_OK) return st;
    lidar_t *l = new (std::nothrow) lidar();
    if (!l) return fail(nullptr, LIDAR_ENOMEM, "host allocation failed");
    l->n_beams = pat->n_beams;
    l->kind = p->kind;
    l->separable = p->kind == LIDAR_PROFILE_SEPARABLE;
    l->n_bins = pu->n_bins;
    l->dt = pu->dt_s;
    l->t0 = pu->t0_s;
    l->T = ca->threshold;
    l->s_amb = ca->ambient_scale;
    l->max_echoes = ca->max_echoes;

    // profile normalisation and device form
    std::vector<float> nodes;  // table: zero-ringed nodes / Z
    int nodes_w = 0, nodes_h = 0;
    std::vector<float2> pairs;
    if (p->kind == LIDAR_PROFILE_RADIAL) {
        l->Z = radial_norm(p);
        double s = p->sigma_deg * kDeg, tc = p->tail_core_deg * kDeg, tr = p->trunc_deg * kDeg;
        l->kg = (float)(-1.0 / (2.0 * s * s * std::log(2.0)));
        l->trunc2 = (float)(tr * tr);
        l->tail_amp = (float)p->tail_amp;
        l->tc2_inv = (float)(1.0 / (tc * tc));
        l->tail_hp = (float)(-0.5 * p->tail_pow);
        l->support_rad = tr;
    } else {
        int pw = p->table_w + 2, ph = p->table_h + 2;
        std::vector<double> padded((size_t)pw * ph, 0.0);
        for (int j = 0; j < p->table_h; ++j)
            for (int i = 0; i < p->table_w; ++i)
                padded[(size_t)(j + 1) * pw + i + 1] =
                    l->separable ? (double)p->table[p->table_w + j] * p->table[i] : p->table[(size_t)j * p->table_w + i];
        l->Z = table_norm(p, padded, pw, ph);
        l->qw = p->table_w + 1;
        l->qh = p->table_h + 1;
        if (l->separable) {
            // zero-padded H (divided by Z) and V as pairs of consecutive nodes
            auto hz = [&](int i) { return (i < 1 || i > p->table_w) ? 0.0 : p->table[i - 1] / l->Z; };
            auto vz = [&](int j) { return (j < 1 || j > p->table_h) ? 0.0 : (double)p->table[p->table_w + j - 1]; };
            for (int i = 0; i < l->qw; ++i) pairs.push_back(make_float2((float)hz(i), (float)hz(i + 1)));
            for (int j = 0; j < l->qh; ++j) pairs.push_back(make_float2((float)vz(j), (float)vz(j + 1)));
        } else {
            // cell (i, j) of the lookup spans nodes (i..i+1, j..j+1) of the
            // zero-ringed grid, gathered by the footprint kernel from a texture
            nodes.resize((size_t)pw * ph);
            for (size_t k = 0; k < nodes.size(); ++k) nodes[k] = (float)(padded[k] / l->Z);
            nodes_w = pw;
            nodes_h = ph;
        }
        l->tk = (float)(1.0 / (p->pitch_deg * kDeg));
        l->tcu = (float)(0.5 * (p->table_w - 1) + 1.0);
        l->tcv = (float)(0.5 * (p->table_h - 1) + 1.0);
        double hu = (0.5 * (p->table_w - 1) + 1) * p->pitch_deg, hv = (0.5 * (p->table_h - 1) + 1) * p->pitch_deg;
        l->support_rad = std::sqrt(hu * hu + hv * hv) * kDeg;
        l->sup_u = hu * kDeg;
        l->sup_v = hv * kDeg;
    }
    if (!(std::isfinite(l->Z) && l->Z > 0)) {
        double Z = l->Z;
        delete l;
        return fail(nullptr, LIDAR_ENUMERIC, "profile integrates to %g", Z);
    }
    // the profile's maximum (after normalisation), for the FP16 deposit's scale
    if (p->kind == LIDAR_PROFILE_RADIAL) {
        l->pmax = (1.0 + std::max(0.0, p->tail_amp)) / l->Z;
    } else {
        double m = 0.0;
        const int n = l->separable ? p->table_w + p->table_h : p->table_w * p->table_h;
        if (l->separable) {
            double mh = 0.0, mv = 0.0;
            for (int i = 0; i < p->table_w; ++i) mh = std::max(mh, (double)p->table[i]);
            for (int j = 0; j < p->table_h; ++j) mv = std::max(mv, (double)p->table[p->table_w + j]);
            m = mh * mv;
        } else {
            for (int i = 0; i < n; ++i) m = std::max(m, (double)p->table[i]);
        }
        l->pmax = m / l->Z;
    }

    // pulse taps, zero-padded so that every tap index of the 32x32 blocks of
    // the convolution is in range
    int M = 0;
    std::vector<double> taps = pulse_taps(pu, &M);
    l->M = M;
    l->R = (M + 31) / 32;
    l->tp_off = 32 * l->R + 31;
    l->tp_len = 64 * l->R + 63;
    std::vector<float> tpad(l->tp_len, 0.f);
    for (int m = -M; m <= M; ++m) tpad[l->tp_off + m] = (float)taps[m + M];

    if (ca->fit_epw) {
        if (!fit_epw(pu, ca->threshold, l->coef)) {
            delete l;
            return fail(nullptr, LIDAR_ENUMERIC, "EPW calibration fit failed");
        }
    } else {
        for (int i = 0; i < 3; ++i) l->coef[i] = ca->epw_coef[i];
    }

    // fingerprint of the sensor model (profile, pulse, calibration): frames of a
    // batch must share the executor's model
    {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&h](const void *p, size_t n) {
            const unsigned char *c = static_cast<const unsigned char *>(p);
            for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
        };
        double md[12] = {l->Z, l->dt, l->t0, l->T, l->s_amb, l->coef[0], l->coef[1], l->coef[2],
                         (double)l->kg, (double)l->trunc2, (double)l->tail_amp, (double)l->tail_hp};
        int32_t mi[7] = {l->kind, l->n_bins, l->M, l->max_echoes, l->qw, l->qh, l->separable ? 1 : 0};
        mix(md, sizeof md);
        mix(mi, sizeof mi);
        if (p->kind == LIDAR_PROFILE_TABLE || p->kind == LIDAR_PROFILE_SEPARABLE) {
            mix(p->table, (p->kind == LIDAR_PROFILE_SEPARABLE ? (size_t)p->table_w + p->table_h
                                                              : (size_t)p->table_w * p->table_h) * sizeof(float));
            mix(&p->pitch_deg, sizeof p->pitch_deg);
        } else {
            double pr[5] = {p->sigma_deg, p->tail_amp, p->tail_core_deg, p->tail_pow, p->trunc_deg};
            mix(pr, sizeof pr);
        }
        l->model_hash = h;
    }

    // launch shape: largest beam group whose histograms fit in shared memory
    // while leaving at least two groups per SM of a 152-SM part
    cudaError_t e = cudaGetDevice(&l->device);
    if (e != cudaSuccess) { delete l; return cuda_fail(nullptr, e, "cudaGetDevice"); }
    // lidar_simulate_noalloc's fixed records: their address on this device
    // (this also places the array, so that the no-allocation call never does);
    // a failure is reported by that call, not here
    l->noalloc_err = gbl::noalloc_records(&l->noalloc_rec);
    if (l->noalloc_err != cudaSuccess) {
        l->noalloc_rec = nullptr;
        cudaGetLastError();  // not sticky: keep it out of later launch checks
    }
    int smem_optin = 0, sms = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, l->device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, l->device);
    gbl::FootprintArgs probe{};
    probe.n_bins = l->n_bins;
    probe.M = l->M;
    // prefer the largest group that still lets two CTAs share an SM, then
    // the largest group that fits at all
    int chosen = 0;
    for (int pass = 0; pass < 2 && !chosen; ++pass)
        for (int G : {8, 4, 2}) {
            size_t need = gbl::footprint_smem_bytes(G, probe);
            if ((long)need > smem_optin) continue;
            if (pass == 0 && 2 * need > 226 * 1024) continue;
            long groups = (l->n_beams + G - 1) / G;
            if (G > 2 && groups < 2L * sms) continue;
            chosen = G;
            break;
        }
    if (!chosen) {
        chosen = 2;
        if ((long)gbl::footprint_smem_bytes(2, probe) > smem_optin) {
            delete l;
            return fail(nullptr, LIDAR_EINVAL, "n_bins too large for shared memory");
        }
    }
    l->G = chosen;
    l->threads = 512;
    l->smem = gbl::footprint_smem_bytes(l->G, probe);
    e = gbl::prepare_footprint(l->kind, l->G, false, l->smem);
    if (e != cudaSuccess) { delete l; return cuda_fail(nullptr, e, "cudaFuncSetAttribute"); }
    // tensor-core form: 8 beams per CTA if two CTAs still share an SM, else 4
    l->G_tc = 8;
    if (2 * gbl::footprint_smem_bytes(8, probe) > 226 * 1024) l->G_tc = 4;
    l->smem_tc = gbl::footprint_smem_bytes(l->G_tc, probe);

    // device copies (and the host copy of the pattern)
    size_t nd = (size_t)pat->n_beams * 3 * sizeof(float);
    try {
        // unit vectors (the beams' set-up normalises them the same way)
        l->h_dirs.resize((size_t)pat->n_beams * 3);
        for (int b = 0; b < pat->n_beams; ++b) {
            const double x = pat->dirs[3 * b], y = pat->dirs[3 * b + 1], z = pat->dirs[3 * b + 2];
            const double n = std::sqrt(x * x + y * y + z * z);
            l->h_dirs[3 * b] = (float)(x / n); l->h_dirs[3 * b + 1] = (float)(y / n); l->h_dirs[3 * b + 2] = (float)(z / n);
        }
    } catch (...) {
        free_all(l);
        delete l;
        return fail(nullptr, LIDAR_ENOMEM, "host allocation failed");
    }
    if ((e = cudaMalloc(&l->d_dirs, nd)) != cudaSuccess ||
        (e = cudaMemcpy(l->d_dirs, pat->dirs, nd, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&l->d_taps, tpad.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(l->d_taps, tpad.data(), tpad.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&l->d_beams, (size_t)pat->n_beams * sizeof(gbl::BeamParam))) != cudaSuccess) {
        free_all(l);
        delete l;
        return cuda_fail(nullptr, e, "device allocation at create");
    }
    if (!nodes.empty()) {
        cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
        cudaResourceDesc rd{};
        cudaTextureDesc td{};
        td.addressMode[0] = cudaAddressModeBorder;  // zero outside the grid
        td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        if ((e = cudaMallocArray(&l->d_nodes, &ch, nodes_w, nodes_h)) != cudaSuccess ||
            (e = cudaMemcpy2DToArray(l->d_nodes, 0, 0, nodes.data(), nodes_w * sizeof(float), nodes_w * sizeof(float),
                                     nodes_h, cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_all(l);
            delete l;
            return cuda_fail(nullptr, e, "profile table upload");
        }
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = l->d_nodes;
        if ((e = cudaCreateTextureObject(&l->node_tex, &rd, &td, nullptr)) != cudaSuccess) {
            free_all(l);
            delete l;
            return cuda_fail(nullptr, e, "profile table texture");
        }
    }
    if (!pairs.empty()) {
        if ((e = cudaMalloc(&l->d_pairs, pairs.size() * sizeof(float2))) != cudaSuccess ||
            (e = cudaMemcpy(l->d_pairs, pairs.data(), pairs.size() * sizeof(float2), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
            free_all(l);
            delete l;
            return cuda_fail(nullptr, e, "separable profile upload");
        }
    }
    *out = l;
    return LIDAR_OK;
}

lidar_status_t lidar_simulate(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *wave,
                              lidar_echoes_t *echoes, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    lidar_status_t st = check_gbuffer(l, g);
    if (st != LIDAR_OK) return st;
    double R[9];
    if ((st = check_pose(l, pose, R)) != LIDAR_OK) return st;
    if (!wave || !echoes || !echoes->echoes || !echoes->counts)
        return fail(l, LIDAR_EINVAL, "output pointer is NULL");
    return enqueue(l, g, R, wave, echoes->echoes, echoes->counts, (cudaStream_t)stream);
}

lidar_status_t lidar_simulate_echoes(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose,
                                     lidar_echoes_t *echoes, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    lidar_status_t st = check_gbuffer(l, g);
    if (st != LIDAR_OK) return st;
    double R[9];
    if ((st = check_pose(l, pose, R)) != LIDAR_OK) return st;
    if (!echoes || !echoes->echoes || !echoes->counts) return fail(l, LIDAR_EINVAL, "output pointer is NULL");
    if (l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16)
        return fail(l, LIDAR_EINVAL, "the tcgen05 deposit has no echo-only form");
    return enqueue(l, g, R, nullptr, echoes->echoes, echoes->counts, (cudaStream_t)stream);
}

// Device address of page-locked host memory mapped into the device's address
// space (cudaHostAlloc, cudaHostRegister with mapping), or null for anything
// else (pageable or device memory).
static const float *mapped_host(const float *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // not known to CUDA: pageable memory
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<const float *>(a.devicePointer);
}

// lidar_simulate_host for large frames. The G-buffer goes up in kHostBands
// bands of rows on copy_stream; each band is set up on setup_stream (highest
// priority, so its CTAs are scheduled ahead of pending footprint CTAs) as soon
// as it lands; the beams run as kHostChunks footprint launches alternating
// between aux_stream[0] and [1] (one launch's CTAs fill the SMs the previous
// one is leaving), each launched once the rows its beams can reach are set up;
// each launch's waveforms go down on d2h_stream while later ones run (echoes
// and counts at the end), and the last two launches hold 6 % and 3 % of the
// beams so that little copying is left at the end. The host enqueues in that
// order (band, its set-up, the launches it completes), so the first launches
// are queued before the last bands' copies. Planes in page-locked,
// device-mapped host memory are not copied at all: the set-up kernel reads
// each band over the host link where it lies.

// The device buffers one frame of the host pipeline uses.
struct HostFrameBufs {
    float4 *rec;
    gbl::BeamParam *beams;
    float *wave;
    lidar_echo_t *echo;
    int32_t *counts;
};

// The pipeline's six streams, in the order of the join and done events.
static void pipeline_streams(lidar_t *l, cudaStream_t out[6])
{
    out[0] = l->aux_stream[0]; out[1] = l->aux_stream[1];
    out[2] = l->d2h_stream[0]; out[3] = l->d2h_stream[1];
    out[4] = l->setup_stream; out[5] = l->copy_stream;
}

// Creates the pipeline's streams and events on first use.
static lidar_status_t ensure_pipeline(lidar_t *l)
{
    cudaError_t e;
    cudaStream_t *streams[] = {&l->copy_stream, &l->d2h_stream[0], &l->d2h_stream[1], &l->aux_stream[0],
                               &l->aux_stream[1]};
    for (cudaStream_t *p : streams)
        if (!*p && (e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(l, e, "cudaStreamCreate(host pipeline)");
    if (!l->setup_stream) {
        int least = 0, greatest = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess ||
            (e = cudaStreamCreateWithPriority(&l->setup_stream, cudaStreamNonBlocking, greatest)) != cudaSuccess)
            return cuda_fail(l, e, "cudaStreamCreate(set-up stream)");
    }
    std::vector<cudaEvent_t *> evs = {&l->start_ev};
    for (cudaEvent_t &ev : l->join_ev) evs.push_back(&ev);
    for (auto &set : l->done_ev)
        for (cudaEvent_t &ev : set) evs.push_back(&ev);
    for (int i = 0; i < kHostChunks; ++i) evs.push_back(&l->chunk_ev[i]);
    for (int i = 0; i < kHostBands; ++i) { evs.push_back(&l->band_ev[i]); evs.push_back(&l->setup_ev[i]); }
    for (cudaEvent_t *ev : evs)
        if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(l, e, "cudaEventCreate(host pipeline)");
    return LIDAR_OK;
}

// Every stream of the pipeline starts after the caller's earlier work on `s`.
static lidar_status_t pipeline_start(lidar_t *l, cudaStream_t s)
{
    cudaError_t e;
    cudaStream_t st[6];
    pipeline_streams(l, st);
    if ((e = cudaEventRecord(l->start_ev, s)) != cudaSuccess) return cuda_fail(l, e, "cudaEventRecord");
    for (cudaStream_t x : st)
        if ((e = cudaStreamWaitEvent(x, l->start_ev, 0)) != cudaSuccess) return cuda_fail(l, e, "cudaStreamWaitEvent");
    return LIDAR_OK;
}

// Records ev[k] at the current end of pipeline stream k; if `join` is set,
// stream `s` (which may be the default stream, 0) waits for all six.
static lidar_status_t pipeline_mark(lidar_t *l, cudaEvent_t ev[6], bool join, cudaStream_t s)
{
    cudaError_t e;
    cudaStream_t st[6];
    pipeline_streams(l, st);
    for (int k = 0; k < 6; ++k)
        if ((e = cudaEventRecord(ev[k], st[k])) != cudaSuccess ||
            (join && (e = cudaStreamWaitEvent(s, ev[k], 0)) != cudaSuccess))
            return cuda_fail(l, e, "pipeline join");
    return LIDAR_OK;
}

// Enqueues one large frame on the pipeline streams, using the buffers B (no
// start or join: see simulate_host_pipelined and lidar_simulate_host_frames).
// dg holds the device staging planes of B, src the caller's host planes.
// prof: record the frame's per-kernel timing events (lidar_profile_enable).
static lidar_status_t enqueue_host_frame(lidar_t *l, const lidar_gbuffer_t *dg, const double R[9],
                                         const float *const src[7], float *const dst[7], const HostFrameBufs &B,
                                         float *wave, lidar_echo_t *echoes, int32_t *counts, bool prof,
                                         cudaEvent_t *end_ev)
{
    cudaError_t e;
    const bool tc = l->deposit != 0;
    const int G = tc ? l->G_tc : l->G;
    const int ng = (l->n_beams + G - 1) / G;
    const int K = kHostChunks, NB = kHostBands;

    // launch sizes: 91 % of the groups in K - 2 equal launches, then 6 % and
    // 3 %, so that little copying is left when the last launches end
    int bounds[kHostChunks + 1];
    bounds[0] = 0;
    for (int i = 1; i < K - 1; ++i) bounds[i] = std::min(l->n_beams, (int)((long)ng * 91 * i / (100 * (K - 2))) * G);
    bounds[K - 1] = std::min(l->n_beams, (int)((long)ng * 97 / 100) * G);
    bounds[K] = l->n_beams;
    int band_row[kHostBands + 1];
    for (int b = 0; b <= NB; ++b) band_row[b] = (int)((long)dg->V * b / NB);
    // the last band a chunk needs: its beams reach rows within the profile's
    // support radius of their elevation (the angle between two directions is
    // at least their elevation difference; the same rotation and row formula
    // as the beams' set-up, two rows wider on each side)
    int chunk_band[kHostChunks];
    const float r6 = (float)R[6], r7 = (float)R[7], r8 = (float)R[8];
    for (int i = 0; i < K; ++i) {
        // the largest height of a rotated unit direction (FP32; its error, ~1e-7
        // rad, is far below the two-row margin)
        float zmax = -2.f;
        const float *d = l->h_dirs.data() + 3 * (size_t)bounds[i];
        for (int b = bounds[i]; b < bounds[i + 1]; ++b, d += 3) zmax = std::max(zmax, r6 * d[0] + r7 * d[1] + r8 * d[2]);
        const double emax = std::asin(std::fmin(1.0, std::fmax(-1.0, (double)zmax)));
        double hi = std::ceil((emax + l->support_rad - dg->el0) / dg->del - 0.5) + 2;
        if (!(hi < dg->V - 1)) hi = dg->V - 1;  // also NaN
        int band = 0;
        while (band + 1 < NB && band_row[band + 1] <= (int)std::max(0.0, hi)) ++band;
        chunk_band[i] = band;
    }

    gbl::SetupArgs sa = setup_args(l, l, dg, R, B.rec, B.beams);
    gbl::FootprintArgs fa = frame_args(l, dg, sa);
    fa.rec = B.rec;
    fa.beams = B.beams;
    if (!wave) {
        // echo-only form: each CTA's waveforms stay in a slot of the pool
        fa.slot_pool = l->d_slot_pool;
        fa.slot_busy = l->d_slot_busy;
        fa.n_slots = l->n_slots;
        fa.slot_sms = kSlotSms;
        fa.slots_per_sm = l->slots_per_sm;
        fa.err = l->d_err;
    }
    const float *mp[7];
    bool mapped = true;
    for (int i = 0; i < 7 && mapped; ++i) mapped = (mp[i] = mapped_host(src[i])) != nullptr;
    if (mapped) {
        sa.range = mp[0]; sa.nx = mp[1]; sa.ny = mp[2]; sa.nz = mp[3];
        sa.rho = mp[4]; sa.retro = mp[5]; sa.amb = mp[6];
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    if (prof && l->prof) {
        size_t mark = l->ev_used;
        ev0 = next_event(l); ev1 = next_event(l); ev2 = next_event(l);
        if (!ev0 || !ev1 || !ev2) { l->ev_used = mark; ev0 = ev1 = ev2 = nullptr; }
    }
    *end_ev = ev2;  // recorded by the caller once its stream has joined the pipeline
    cudaStream_t ss = l->setup_stream, us = l->copy_stream;
    if (ev0) cudaEventRecord(ev0, ss);
    gbl::SetupArgs sb = sa;
    sb.pix_blocks = 0;  // the beams' set-up (reads no plane)
    if ((e = gbl::launch_setup(sb, ss)) != cudaSuccess) return cuda_fail(l, e, "setup kernel launch");
    int next = 0;
    for (int b = 0; b < NB; ++b) {
        const long p0 = (long)band_row[b] * dg->U, p1 = (long)band_row[b + 1] * dg->U;
        for (int i = 0; i < 7 && p1 > p0 && !mapped; ++i)
            if ((e = cudaMemcpyAsync(dst[i] + p0, src[i] + p0, (size_t)(p1 - p0) * sizeof(float), cudaMemcpyHostToDevice,
                                     us)) != cudaSuccess)
                return cuda_fail(l, e, "G-buffer upload");
        gbl::SetupArgs sp = sa;
        sp.n_beams = 0;
        sp.pix_begin = p0;
        sp.pix_end = p1;
        sp.pix_blocks = (int)std::max<long>(1, std::min<long>(sa.pix_blocks, (p1 - p0 + 255) / 256));
        if ((e = cudaEventRecord(l->band_ev[b], us)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ss, l->band_ev[b], 0)) != cudaSuccess ||
            (p1 > p0 && (e = gbl::launch_setup(sp, ss)) != cudaSuccess) ||
            (e = cudaEventRecord(l->setup_ev[b], ss)) != cudaSuccess)
            return cuda_fail(l, e, "setup kernel launch");
        if (b == NB - 1 && ev1) cudaEventRecord(ev1, ss);
        for (; next < K && chunk_band[next] <= b; ++next) {
            const int i = next, b0 = bounds[i], nb = bounds[i + 1] - bounds[i];
            cudaStream_t cs = l->aux_stream[i & 1];
            gbl::FootprintArgs fc = fa;
            fc.beams = B.beams + b0;
            fc.n_beams = nb;
            fc.wave = wave ? B.wave + (size_t)b0 * l->n_bins : nullptr;
            fc.echoes = B.echo + (size_t)b0 * l->max_echoes;
            fc.counts = B.counts + b0;
            if ((e = cudaStreamWaitEvent(cs, l->setup_ev[b], 0)) != cudaSuccess)
                return cuda_fail(l, e, "cudaStreamWaitEvent");
            if (nb > 0 && (e = gbl::launch_footprint(l->kind, G, tc, l->threads, tc ? l->smem_tc : l->smem, fc, cs)) !=
                              cudaSuccess)
                return cuda_fail(l, e, "footprint kernel launch");
            cudaStream_t ds = l->d2h_stream[i & 1];
            if ((e = cudaEventRecord(l->chunk_ev[i], cs)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ds, l->chunk_ev[i], 0)) != cudaSuccess)
                return cuda_fail(l, e, "cudaEventRecord");
            if (wave && nb > 0 && (e = cudaMemcpyAsync(wave + (size_t)b0 * l->n_bins, B.wave + (size_t)b0 * l->n_bins,
                                               (size_t)nb * l->n_bins * sizeof(float), cudaMemcpyDeviceToHost, ds)) !=
                              cudaSuccess)
                return cuda_fail(l, e, "result download");
        }
    }
    // echoes and counts (small) once every launch is done
    cudaStream_t ds = l->d2h_stream[0];
    for (int i = 1; i < K; i += 2)
        if ((e = cudaStreamWaitEvent(ds, l->chunk_ev[i], 0)) != cudaSuccess) return cuda_fail(l, e, "cudaStreamWaitEvent");
    if ((e = cudaMemcpyAsync(echoes, B.echo, (size_t)l->n_beams * l->max_echoes * sizeof(lidar_echo_t),
                             cudaMemcpyDeviceToHost, ds)) != cudaSuccess ||
        (e = cudaMemcpyAsync(counts, B.counts, (size_t)l->n_beams * sizeof(int32_t), cudaMemcpyDeviceToHost, ds)) !=
            cudaSuccess)
        return cuda_fail(l, e, "result download");
    return LIDAR_OK;
}

// One large frame of lidar_simulate_host: the pipeline starts after the
// caller's earlier work on `s`, runs the frame on the first buffer set, and `s`
// joins the ends of all six streams (the set-up and upload streams too, so
// that nothing reads the caller's planes after the return).
static lidar_status_t simulate_host_pipelined(lidar_t *l, const lidar_gbuffer_t *dg, const double R[9],
                                              const float *const src[7], float *const dst[7], float *wave,
                                              lidar_echo_t *echoes, int32_t *counts, cudaStream_t s)
{
    cudaError_t e;
    const bool tc = l->deposit != 0;
    lidar_status_t st = ensure_scratch(l, (size_t)dg->U * dg->V);
    if (st != LIDAR_OK) return st;
    if (!wave && (st = ensure_slots(l, tc ? l->G_tc : l->G, tc)) != LIDAR_OK) return st;  // echo-only form
    if ((st = ensure_pipeline(l)) != LIDAR_OK || (st = pipeline_start(l, s)) != LIDAR_OK) return st;
    const HostFrameBufs B{l->d_rec, l->d_beams, l->d_wave, l->d_echo, l->d_counts};
    cudaEvent_t end_ev = nullptr;
    if ((st = enqueue_host_frame(l, dg, R, src, dst, B, wave, echoes, counts, true, &end_ev)) != LIDAR_OK) return st;
    if ((st = pipeline_mark(l, l->join_ev, true, s)) != LIDAR_OK) return st;
    if (end_ev) cudaEventRecord(end_ev, s);
    return wave ? (((e = cudaStreamSynchronize(s)) != cudaSuccess) ? cuda_fail(l, e, "cudaStreamSynchronize") : LIDAR_OK)
                : lidar_sync(l, s);  // also reports a slot-claim timeout of the echo-only form
}

// The caller's host planes of frame g (src), the staging planes of a buffer
// set (dst), and the frame's G-buffer description over the staging planes (dg).
static void host_frame_planes(const lidar_gbuffer_t *g, float *planes, const float *src[7], float *dst[7],
                              lidar_gbuffer_t *dg)
{
    const size_t pixels = (size_t)g->U * g->V;
    const float *in[7] = {g->range, g->nx, g->ny, g->nz, g->rho_d, g->retro, g->ambient};
    for (int i = 0; i < 7; ++i) {
        src[i] = in[i];
        dst[i] = planes + (size_t)i * pixels;
    }
    *dg = *g;
    dg->range = dst[0]; dg->nx = dst[1]; dg->ny = dst[2]; dg->nz = dst[3];
    dg->rho_d = dst[4]; dg->retro = dst[5]; dg->ambient = dst[6];
}

// Frames of at least 8 x 152 beam groups (8 footprint launches of at least one
// CTA per SM) take the pipelined host path; smaller ones one pass on the
// caller's stream.
static bool pipelined_frame(const lidar_t *l)
{
    const int G = l->deposit != 0 ? l->G_tc : l->G;
    return (l->n_beams + G - 1) / G >= 8 * 152;
}

// Device buffers of the host entry points' buffer set `set` (0: the frame
// buffers of lidar_simulate_host; 1: the second set of
// lidar_simulate_host_frames) for frames of up to `pixels` pixels: staging
// planes, records, beam parameters, results (waveforms only if `wave`).
static lidar_status_t ensure_host_set(lidar_t *l, int set, size_t pixels, bool wave, HostFrameBufs *B, float **planes)
{
    cudaError_t e;
    float *&pl = set ? l->d_planes2 : l->d_planes;
    size_t &pcap = set ? l->planes2_cap : l->planes_cap;
    if (pixels > pcap) {
        cudaFree(pl);
        pl = nullptr;
        pcap = 0;
        if ((e = cudaMalloc(&pl, 7 * pixels * sizeof(float))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(G-buffer staging)");
        pcap = pixels;
    }
    lidar_echo_t *&echo = set ? l->d_echo2 : l->d_echo;
    int32_t *&counts = set ? l->d_counts2 : l->d_counts;
    if (!echo) {
        if ((e = cudaMalloc(&echo, (size_t)l->n_beams * l->max_echoes * sizeof(lidar_echo_t))) != cudaSuccess ||
            (e = cudaMalloc(&counts, (size_t)l->n_beams * sizeof(int32_t))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(output staging)");
    }
    float *&wv = set ? l->d_wave2 : l->d_wave;
    if (wave && !wv && (e = cudaMalloc(&wv, (size_t)l->n_beams * l->n_bins * sizeof(float))) != cudaSuccess)
        return cuda_fail(l, e, "cudaMalloc(output staging)");
    if (set == 0) {
        lidar_status_t st = ensure_scratch(l, pixels);
        if (st != LIDAR_OK) return st;
    } else {
        if (pixels > l->rec2_cap) {
            cudaFree(l->d_rec2);
            l->d_rec2 = nullptr;
            l->rec2_cap = 0;
            if ((e = cudaMalloc(&l->d_rec2, pixels * 2 * sizeof(float4))) != cudaSuccess)
                return cuda_fail(l, e, "cudaMalloc(per-pixel records)");
            l->rec2_cap = pixels;
        }
        if (!l->d_beams2 &&
            (e = cudaMalloc(&l->d_beams2, (size_t)l->n_beams * sizeof(gbl::BeamParam))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(beam parameters)");
    }
    *B = HostFrameBufs{set ? l->d_rec2 : l->d_rec, set ? l->d_beams2 : l->d_beams, wv, echo, counts};
    *planes = pl;
    return LIDAR_OK;
}

lidar_status_t lidar_simulate_host(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *wave,
                                   lidar_echo_t *echoes, int32_t *counts, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16)
        return fail(l, LIDAR_EINVAL, "the host entry points do not take the tcgen05 deposit");
    lidar_status_t st = check_gbuffer(l, g);
    if (st != LIDAR_OK) return st;
    double R[9];
    if ((st = check_pose(l, pose, R)) != LIDAR_OK) return st;
    if (!echoes || !counts) return fail(l, LIDAR_EINVAL, "output pointer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    size_t pixels = (size_t)g->U * g->V;
    cudaError_t e;
    HostFrameBufs B0;
    float *planes0 = nullptr;
    if ((st = ensure_host_set(l, 0, pixels, wave != nullptr, &B0, &planes0)) != LIDAR_OK) return st;
    const float *src[7];
    float *dst[7];
    lidar_gbuffer_t dg;
    host_frame_planes(g, planes0, src, dst, &dg);
    if (!pipelined_frame(l)) {
        // small frame: one pass on `stream`
        for (int i = 0; i < 7; ++i)
            if ((e = cudaMemcpyAsync(dst[i], src[i], pixels * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
                return cuda_fail(l, e, "G-buffer upload");
        if ((st = enqueue(l, &dg, R, wave ? l->d_wave : nullptr, l->d_echo, l->d_counts, s)) != LIDAR_OK) return st;
        if ((wave && (e = cudaMemcpyAsync(wave, l->d_wave, (size_t)l->n_beams * l->n_bins * sizeof(float),
                                          cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(echoes, l->d_echo, (size_t)l->n_beams * l->max_echoes * sizeof(lidar_echo_t),
                                 cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(counts, l->d_counts, (size_t)l->n_beams * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
            return cuda_fail(l, e, "result download");
        if (!wave) return lidar_sync(l, s);  // also reports a slot-claim timeout of the echo-only form
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(l, e, "cudaStreamSynchronize");
        return LIDAR_OK;
    }
    return simulate_host_pipelined(l, &dg, R, src, dst, wave, echoes, counts, s);
}

lidar_status_t lidar_simulate_host_frames(lidar_t *l, int n_frames, const lidar_gbuffer_t *g,
                                          const lidar_pose_t *pose, float *const *wave, lidar_echo_t *const *echoes,
                                          int32_t *const *counts, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16)
        return fail(l, LIDAR_EINVAL, "the host entry points do not take the tcgen05 deposit");
    if (n_frames < 0) return fail(l, LIDAR_EINVAL, "n_frames < 0");
    if (n_frames == 0) return LIDAR_OK;
    if (!g || !pose || !echoes || !counts) return fail(l, LIDAR_EINVAL, "frame array is NULL");
    std::vector<double> Rs(9 * (size_t)n_frames);
    size_t max_pixels = 0;
    lidar_status_t st;
    for (int f = 0; f < n_frames; ++f) {
        if ((st = check_gbuffer(l, g + f)) != LIDAR_OK || (st = check_pose(l, pose + f, Rs.data() + 9 * f)) != LIDAR_OK)
            return st;
        if (!echoes[f] || !counts[f] || (wave && !wave[f])) return fail(l, LIDAR_EINVAL, "output pointer is NULL");
        max_pixels = std::max(max_pixels, (size_t)g[f].U * g[f].V);
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (!pipelined_frame(l) || n_frames == 1) {
        // small frames (one pass each) or a single frame: lidar_simulate_host per frame
        for (int f = 0; f < n_frames; ++f)
            if ((st = lidar_simulate_host(l, g + f, pose + f, wave ? wave[f] : nullptr, echoes[f], counts[f], stream)) !=
                LIDAR_OK)
                return st;
        return LIDAR_OK;
    }
    const bool tc = l->deposit != 0;
    HostFrameBufs B[2];
    float *planes[2];
    for (int p = 0; p < 2; ++p)
        if ((st = ensure_host_set(l, p, max_pixels, wave != nullptr, &B[p], &planes[p])) != LIDAR_OK) return st;
    if (!wave && (st = ensure_slots(l, tc ? l->G_tc : l->G, tc)) != LIDAR_OK) return st;  // echo-only form
    if ((st = ensure_pipeline(l)) != LIDAR_OK || (st = pipeline_start(l, s)) != LIDAR_OK) return st;
    cudaError_t e;
    cudaStream_t streams[6];
    pipeline_streams(l, streams);
    for (int f = 0; f < n_frames; ++f) {
        const int p = f & 1;
        if (f >= 2)
            // frame f - 2 used the same buffers: every stream waits for all of it
            for (cudaStream_t x : streams)
                for (cudaEvent_t ev : l->done_ev[p])
                    if ((e = cudaStreamWaitEvent(x, ev, 0)) != cudaSuccess) return cuda_fail(l, e, "cudaStreamWaitEvent");
        const float *src[7];
        float *dst[7];
        lidar_gbuffer_t dg;
        host_frame_planes(g + f, planes[p], src, dst, &dg);
        cudaEvent_t end_ev = nullptr;
        if ((st = enqueue_host_frame(l, &dg, Rs.data() + 9 * f, src, dst, B[p], wave ? wave[f] : nullptr, echoes[f],
                                     counts[f], false, &end_ev)) != LIDAR_OK ||
            (st = pipeline_mark(l, l->done_ev[p], false, s)) != LIDAR_OK)
            return st;
    }
    // `s` joins the last frame of each set
    for (int p = 0; p < 2; ++p)
        for (cudaEvent_t ev : l->done_ev[p])
            if ((e = cudaStreamWaitEvent(s, ev, 0)) != cudaSuccess) return cuda_fail(l, e, "pipeline join");
    return wave ? (((e = cudaStreamSynchronize(s)) != cudaSuccess) ? cuda_fail(l, e, "cudaStreamSynchronize") : LIDAR_OK)
                : lidar_sync(l, s);  // also reports a slot-claim timeout of the echo-only form
}

lidar_status_t lidar_simulate_noalloc(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *wave,
                                      lidar_echoes_t *echoes, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    lidar_status_t st = check_gbuffer(l, g);
    if (st != LIDAR_OK) return st;
    if ((long)g->U * g->V > gbl::kNoAllocMaxPixels)
        return fail(l, LIDAR_EINVAL, "gbuffer has %ld pixels; lidar_simulate_noalloc takes at most %ld",
                    (long)g->U * g->V, gbl::kNoAllocMaxPixels);
    double R[9];
    if ((st = check_pose(l, pose, R)) != LIDAR_OK) return st;
    if (!wave || !echoes || !echoes->echoes || !echoes->counts)
        return fail(l, LIDAR_EINVAL, "output pointer is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(l, e, "cudaGetDevice");
    if (dev != l->device)
        return fail(l, LIDAR_EINVAL, "current device %d is not the device %d this lidar was created on", dev,
                    l->device);
    if (!l->noalloc_rec)
        return cuda_fail(l, l->noalloc_err, "no-allocation scratch was not placed at lidar_create");
    float4 *rec = l->noalloc_rec;
    // Run the regular path with the fixed array as its per-pixel scratch: its
    // capacity covers the G-buffer, so nothing is allocated; profiling events
    // (which would be created on demand) are off for this call. Every pixel's
    // record is rewritten before it is read, so nothing needs clearing.
    float4 *own = l->d_rec;
    size_t own_cap = l->rec_cap;
    bool prof = l->prof;
    l->d_rec = rec;
    l->rec_cap = (size_t)gbl::kNoAllocMaxPixels;
    l->prof = false;
    st = enqueue(l, g, R, wave, echoes->echoes, echoes->counts, (cudaStream_t)stream);
    l->d_rec = own;
    l->rec_cap = own_cap;
    l->prof = prof;
    return st;
}

lidar_status_t lidar_simulate_batch(lidar_t *l, const lidar_frame_t *frames, int32_t n_frames, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "executor is NULL");
    return batch_run(l, frames, n_frames, (cudaStream_t)stream, l->batch_G, l->batch_cps);
}

lidar_status_t lidar_autotune_batch(lidar_t *l, const lidar_frame_t *frames, int32_t n_frames, void *stream)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "executor is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, l->device);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess)
        return cuda_fail(l, e, "cudaEventCreate");
    float best = 1e30f;
    int bestG = l->batch_G, bestC = l->batch_cps;
    lidar_status_t st = LIDAR_OK;
    for (int G : {2, 4, 8, 16}) {
        if (l->deposit != 0 && G != 4 && G != 8) continue;
        size_t smem = gbl::footprint_smem_bytes(G, model_args(l));
        if ((long)smem > smem_optin) continue;
        for (int cps : {1, 2}) {
            if (cps * smem > 228 * 1024) continue;
            // one untimed run (graph capture), then two timed runs
            if ((st = batch_run(l, frames, n_frames, s, G, cps)) != LIDAR_OK) break;
            cudaEventRecord(a, s);
            for (int r = 0; r < 2 && st == LIDAR_OK; ++r) st = batch_run(l, frames, n_frames, s, G, cps);
            cudaEventRecord(b, s);
            if (st != LIDAR_OK) break;
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) { st = cuda_fail(l, e, "cudaEventSynchronize"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) { best = ms; bestG = G; bestC = cps; }
        }
        if (st != LIDAR_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != LIDAR_OK) return st;
    l->batch_G = bestG;
    l->batch_cps = bestC;
    return LIDAR_OK;
}

lidar_status_t lidar_set_echo_mode(lidar_t *l, int32_t mode)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (mode != LIDAR_ECHOES_NEAREST && mode != LIDAR_ECHOES_STRONGEST)
        return fail(l, LIDAR_EINVAL, "echo mode %d unknown", mode);
    l->echo_mode = mode;
    return LIDAR_OK;
}

lidar_status_t lidar_hold_echo_slots(lidar_t *l, int32_t held)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    const bool tc = l->deposit != 0;
    lidar_status_t st = ensure_slots(l, tc ? l->G_tc : l->G, tc);
    if (st != LIDAR_OK) return st;
    // a nonzero busy word is a held slot (claims compare against 0)
    cudaError_t e = cudaMemset(l->d_slot_busy, held ? 1 : 0, (size_t)l->n_slots * sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? LIDAR_OK : cuda_fail(l, e, "slot pool memset");
}

lidar_status_t lidar_set_deposit(lidar_t *l, int32_t mode)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (mode < LIDAR_DEPOSIT_ATOMIC || mode > LIDAR_DEPOSIT_TCGEN05_FP16)
        return fail(l, LIDAR_EINVAL, "deposit mode %d unknown", mode);
    if (mode >= LIDAR_DEPOSIT_TCGEN05_BF16) {
        if (l->n_bins > gbl::kUmmaMaxBins)
            return fail(l, LIDAR_EINVAL, "the tcgen05 deposit takes n_bins <= %d (got %d)", gbl::kUmmaMaxBins,
                        l->n_bins);
        const size_t smem = gbl::umma_smem_bytes(l->n_bins, l->M);
        if ((long)smem > 227L * 1024) return fail(l, LIDAR_EINVAL, "n_bins too large for the tcgen05 deposit");
        const bool bf16 = mode == LIDAR_DEPOSIT_TCGEN05_BF16;
        cudaError_t e = gbl::prepare_umma(l->kind, bf16, smem);
        if (e != cudaSuccess) return cuda_fail(l, e, "cudaFuncSetAttribute");
        // its error word (bounded pipeline waits) and the frame's weight maximum
        if ((!l->d_err && (e = cudaMalloc(&l->d_err, sizeof(int))) != cudaSuccess) ||
            (!l->d_wmax && (e = cudaMalloc(&l->d_wmax, sizeof(unsigned))) != cudaSuccess) ||
            (e = cudaMemset(l->d_err, 0, sizeof(int))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(tcgen05 deposit words)");
        if (!l->d_perm) {
            std::vector<int32_t> order = group_order(l);
            if ((e = cudaMalloc(&l->d_perm, order.size() * sizeof(int32_t))) != cudaSuccess ||
                (e = cudaMemcpy(l->d_perm, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                return cuda_fail(l, e, "beam group order upload");
        }
        l->smem_um = smem;
        l->deposit = mode;
        return LIDAR_OK;
    }
    if (mode != LIDAR_DEPOSIT_ATOMIC && (long)l->smem_tc > 227L * 1024)
        return fail(l, LIDAR_EINVAL, "n_bins too large for the tensor-core deposit");
    if (mode != LIDAR_DEPOSIT_ATOMIC) {
        cudaError_t e = gbl::prepare_footprint(l->kind, l->G_tc, true, l->smem_tc);
        if (e != cudaSuccess) return cuda_fail(l, e, "cudaFuncSetAttribute");
        l->batch_G = l->G_tc;
    }
    l->deposit = mode;
    return LIDAR_OK;
}

lidar_status_t lidar_batch_config(const lidar_t *l, int32_t *beams_per_cta, int32_t *ctas_per_sm)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "executor is NULL");
    if (beams_per_cta) *beams_per_cta = l->batch_G;
    if (ctas_per_sm) *ctas_per_sm = l->batch_cps > 0 ? l->batch_cps : 2;
    return LIDAR_OK;
}

lidar_status_t lidar_sync(lidar_t *l, void *stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(l, e, "cudaStreamSynchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(l, e, "asynchronous error");
    if (l && l->d_err) {
        int h = 0;
        if ((e = cudaMemcpy(&h, l->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(l, e, "error word download");
        if (h) {
            cudaMemset(l->d_err, 0, sizeof(int));
            if (l->deposit >= LIDAR_DEPOSIT_TCGEN05_BF16)
                return fail(l, LIDAR_ETIMEOUT,
                            "tcgen05 deposit: a CTA's pipeline wait gave up (code 0x%08x: wait site, stage, "
                            "stages claimed); its beams were not written", (unsigned)h);
            return fail(l, LIDAR_ETIMEOUT, "echo-only simulation: a CTA found no free waveform slot; its beams' "
                                           "echoes were not written");
        }
    }
    return LIDAR_OK;
}

lidar_status_t lidar_get_info(const lidar_t *l, int32_t *n_beams, int32_t *n_bins, int32_t *max_echoes,
                              double *profile_norm, double epw_coef[3])
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (n_beams) *n_beams = l->n_beams;
    if (n_bins) *n_bins = l->n_bins;
    if (max_echoes) *max_echoes = l->max_echoes;
    if (profile_norm) *profile_norm = l->Z;
    if (epw_coef) for (int i = 0; i < 3; ++i) epw_coef[i] = l->coef[i];
    return LIDAR_OK;
}

int32_t lidar_launches_per_simulate(const lidar_t *l) { return l ? 2 : 0; }

lidar_status_t lidar_profile_enable(lidar_t *l, int32_t enable)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    free_events(l);
    l->prof = enable != 0;
    return LIDAR_OK;
}

lidar_status_t lidar_profile_read(lidar_t *l, double total_ms[2], int32_t launches[2])
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    double t[2] = {0, 0};
    int32_t n[2] = {0, 0};
    for (size_t i = 0; i + 3 <= l->ev_used; i += 3) {
        cudaError_t e = cudaEventSynchronize(l->ev[i + 2]);
        if (e != cudaSuccess) return cuda_fail(l, e, "cudaEventSynchronize");
        float a = 0, b = 0;
        if ((e = cudaEventElapsedTime(&a, l->ev[i], l->ev[i + 1])) != cudaSuccess ||
            (e = cudaEventElapsedTime(&b, l->ev[i + 1], l->ev[i + 2])) != cudaSuccess)
            return cuda_fail(l, e, "cudaEventElapsedTime");
        t[0] += a; t[1] += b; n[0] += 1; n[1] += 1;
    }
    l->ev_used = 0;
    if (total_ms) { total_ms[0] = t[0]; total_ms[1] = t[1]; }
    if (launches) { launches[0] = n[0]; launches[1] = n[1]; }
    return LIDAR_OK;
}

const char *lidar_last_error(const lidar_t *l) { return l ? l->err : g_create_err; }

void lidar_destroy(lidar_t *l)
{
    if (!l) return;
    free_all(l);
    delete l;
}

}  // extern "C"
