/*
 * FP64 CPU oracle of the analytic LiDAR beam model (Dudzik et al., "Physically-
 * Based Simulation of Automotive LiDAR", IAVVC 2025, arXiv 2512.05932).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU path computes. Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Every loop follows the discretised definition directly: for every beam, the
 * whole G-buffer is visited (rows that are provably farther from the beam axis
 * than the profile support are skipped, an exact test), each pixel's return
 * is weighted by the profile at the pixel centre and spread over its range
 * interval, then the histogram is convolved with the pulse, ambient light is
 * added and echoes are read off with the threshold rule.
 *
 * Readings of the paper used here (each one is listed in the design notes):
 *  - Alg. 1 accumulates (the printed assignment inside the kernel loop is an
 *    accumulation: the signal is "composed of" the pixel contributions).
 *  - "contributes uniformly to a range interval" spreads the pixel's energy
 *    as a uniform density over its time-of-flight interval; the density is
 *    projected onto linear hat functions centred on the bin centres.
 *  - The kernel offset Phi - Psi_b of Eq. (centered kernel) is taken in the
 *    beam's local tangent frame with azimuthal-equidistant coordinates, and
 *    the beam centre is not rounded to the pixel grid.
 *  - rho_hat of a pixel = beta * |cos theta_i| / R^2 with beta = rho_d/pi + g.
 *  - The received power of a pixel is rho_hat times its exact solid angle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_C_LIGHT 299792458.0
#define ORC_PI 3.14159265358979323846
#define ORC_DEG (ORC_PI / 180.0)
#define ORC_MU_MIN 1e-3          /* grazing clamp of |d.n| in the range interval */
#define ORC_NEAR_REL 1e-4        /* guard band around the threshold */

enum { ORC_CLIPPED_START = 1u, ORC_CLIPPED_END = 2u, ORC_NEAR_THRESHOLD = 4u,
       ORC_PEAK_AMBIGUOUS = 8u };

typedef struct {
    int32_t kind; /* 0 radial analytic, 1 table, 2 separable H(u) V(v) */
    double sigma_deg, tail_amp, tail_core_deg, tail_pow, trunc_deg;
    int32_t tw, th;
    double pitch_deg;
    const float *table; /* kind 1: [th][tw], row j <-> v, column i <-> u;
                           kind 2: H[tw] (nodes along u) then V[th] (nodes along v) */
} orc_profile;

typedef struct {
    int32_t U, V;
    double az0, el0, daz, del;
    const float *range, *nx, *ny, *nz, *rho, *retro, *amb; /* [V][U] */
} orc_gbuffer;

typedef struct {
    int32_t n_bins;
    double dt, t0, fwhm, trunc_sigmas;
} orc_pulse;

typedef struct {
    double T, s_amb;
    double c0, c1, c2;
} orc_calib;

typedef struct {
    double range_m, epw_m, intensity, peak, r0, r1, x_peak;
    int32_t bin_peak, bin_start, bin_end;
    uint32_t flags;
} orc_echo;

/* ------------------------------------------------------------------------ */
/* Profile kappa*eta (Eq. centered kernel; Sec. III combined kernel)         */
/* ------------------------------------------------------------------------ */

/* Linear interpolation of n nodes t[0..n) at fractional index f, zero
 * beyond the end nodes (the value falls to 0 one node spacing outside). */
static double orc_lerp_nodes(const float *t, long n, double f)
{
    double f0 = floor(f), a = f - f0, val = 0.0;
    long i = (long)f0;
    if (i >= 0 && i < n) val += (1.0 - a) * (double)t[i];
    if (i + 1 >= 0 && i + 1 < n) val += a * (double)t[i + 1];
    return val;
}

/* Unnormalised profile value at local offset (u, v) in degrees. */
double orc_profile_raw(const orc_profile *p, double u, double v)
{
    if (p->kind == 0) {
        double th = sqrt(u * u + v * v);
        if (th > p->trunc_deg) return 0.0;
        double g = exp(-th * th / (2.0 * p->sigma_deg * p->sigma_deg));
        double t = 1.0;
        if (th > p->tail_core_deg) t = pow(th / p->tail_core_deg, -p->tail_pow);
        return g + p->tail_amp * t;
    }
    if (p->kind == 2) {
        /* separable kernel (Sec. III-C: horizontal times vertical profile) */
        double fi = u / p->pitch_deg + 0.5 * (p->tw - 1);
        double fj = v / p->pitch_deg + 0.5 * (p->th - 1);
        return orc_lerp_nodes(p->table, p->tw, fi) * orc_lerp_nodes(p->table + p->tw, p->th, fj);
    }
    /* bilinear interpolation of the table extended by zeros beyond its edge */
    double fi = u / p->pitch_deg + 0.5 * (p->tw - 1);
    double fj = v / p->pitch_deg + 0.5 * (p->th - 1);
    double i0 = floor(fi), j0 = floor(fj);
    double ax = fi - i0, ay = fj - j0;
    double val = 0.0;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            long i = (long)i0 + di, j = (long)j0 + dj;
            if (i < 0 || j < 0 || i >= p->tw || j >= p->th) continue;
            double wgt = (di ? ax : 1.0 - ax) * (dj ? ay : 1.0 - ay);
            val += wgt * (double)p->table[j * (long)p->tw + i];
        }
    return val;
}

/* Angular radius (degrees) outside of which the profile is zero. */
double orc_profile_support_deg(const orc_profile *p)
{
    if (p->kind == 0) return p->trunc_deg;
    double hu = (0.5 * (p->tw - 1) + 1.0) * p->pitch_deg;
    double hv = (0.5 * (p->th - 1) + 1.0) * p->pitch_deg;
    return sqrt(hu * hu + hv * hv);
}

/* Z = integral of the raw profile over the sphere, d omega = sin(theta) dtheta dphi.
 * Radial: composite Simpson in theta, split at the tail core and the
 * truncation. Table: the zero-extended table's cells, each split into 4x4
 * sub-cells, midpoint rule with the azimuthal-equidistant area element
 * d omega = sin(theta)/theta du dv. */
double orc_profile_norm(const orc_profile *p)
{
    if (p->kind == 0) {
        double edges[3] = {0.0, fmin(p->tail_core_deg, p->trunc_deg), p->trunc_deg};
        double Z = 0.0;
        for (int s = 0; s < 2; ++s) {
            double a = edges[s], b = edges[s + 1];
            if (b <= a) continue;
            int n = 200000;
            double h = (b - a) / n, acc = 0.0;
            for (int k = 0; k <= n; ++k) {
                double th = a + k * h;
                double f = orc_profile_raw(p, th, 0.0) * sin(th * ORC_DEG);
                acc += f * ((k == 0 || k == n) ? 1.0 : ((k & 1) ? 4.0 : 2.0));
            }
            Z += acc * h / 3.0 * ORC_DEG;
        }
        return 2.0 * ORC_PI * Z;
    }
    const int sub = 4;
    double pr = p->pitch_deg * ORC_DEG, Z = 0.0;
    for (int j = -1; j < p->th; ++j)
        for (int i = -1; i < p->tw; ++i)
            for (int sj = 0; sj < sub; ++sj)
                for (int si = 0; si < sub; ++si) {
                    double fi = i + (si + 0.5) / sub, fj = j + (sj + 0.5) / sub;
                    double u = (fi - 0.5 * (p->tw - 1)) * p->pitch_deg;
                    double v = (fj - 0.5 * (p->th - 1)) * p->pitch_deg;
                    double th = sqrt(u * u + v * v) * ORC_DEG;
                    double jac = th > 0 ? sin(th) / th : 1.0;
                    Z += orc_profile_raw(p, u, v) * jac;
                }
    return Z * pr * pr / (sub * sub);
}

/* ------------------------------------------------------------------------ */
/* Beam frame and local offsets (Eq. centered kernel, Sec. II-C pinhole vs   */
/* spherical: the kernel is adapted per beam in its own tangent frame)       */
/* ------------------------------------------------------------------------ */

typedef struct { double a[3], e1[3], e2[3]; } orc_frame;

static void cross3(const double *x, const double *y, double *o)
{
    o[0] = x[1] * y[2] - x[2] * y[1];
    o[1] = x[2] * y[0] - x[0] * y[2];
    o[2] = x[0] * y[1] - x[1] * y[0];
}

static void normalize3(double *x)
{
    double n = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    x[0] /= n; x[1] /= n; x[2] /= n;
}

/* Beam axis a = R dir and local axes E1 = R e1, E2 = R e2 where, in the sensor
 * frame, e1 = z x dir (normalised; y if dir is vertical) and e2 = dir x e1. */
void orc_beam_frame(const float *R, const float *dir, orc_frame *f)
{
    double d[3] = {dir[0], dir[1], dir[2]};
    normalize3(d);
    double e1[3] = {-d[1], d[0], 0.0};
    if (e1[0] * e1[0] + e1[1] * e1[1] < 1e-24) { e1[0] = 0; e1[1] = 1; e1[2] = 0; }
    normalize3(e1);
    double e2[3];
    cross3(d, e1, e2);
    for (int r = 0; r < 3; ++r) {
        f->a[r] = R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2];
        f->e1[r] = R[3 * r] * e1[0] + R[3 * r + 1] * e1[1] + R[3 * r + 2] * e1[2];
        f->e2[r] = R[3 * r] * e2[0] + R[3 * r + 1] * e2[1] + R[3 * r + 2] * e2[2];
    }
    normalize3(f->a);
}

/* Azimuthal-equidistant offset (u, v) in degrees of unit direction d. Returns 0
 * when d is in the back hemisphere of the beam. */
int orc_local_offset(const orc_frame *f, const double *d, double *u, double *v)
{
    double c = d[0] * f->a[0] + d[1] * f->a[1] + d[2] * f->a[2];
    double x = d[0] * f->e1[0] + d[1] * f->e1[1] + d[2] * f->e1[2];
    double y = d[0] * f->e2[0] + d[1] * f->e2[1] + d[2] * f->e2[2];
    if (c <= 0.0) return 0;
    double s = sqrt(x * x + y * y);
    double th = atan2(s, c);
    if (s > 0) { *u = th * x / s / ORC_DEG; *v = th * y / s / ORC_DEG; }
    else { *u = 0; *v = 0; }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel quantities (Eq. rho_hat, pixelRangeInterval of Alg. 1, range     */
/* correction r_corr = p.n/(v.n) r of Sec. II-D)                              */
/* ------------------------------------------------------------------------ */

static void dir_of(double az, double el, double *d)
{
    d[0] = cos(el) * cos(az); d[1] = cos(el) * sin(az); d[2] = sin(el);
}

/* Returns 1 if the pixel has a hit. w = rho_hat * d omega (received power per
 * unit profile weight), [t0, t1] its time-of-flight interval (s), a = L_amb
 * d omega (ambient, every pixel). */
int orc_pixel(const orc_gbuffer *g, int u, int v, double *w, double *t0, double *t1, double *a)
{
    long idx = (long)v * g->U + u;
    double az = g->az0 + (u + 0.5) * g->daz;
    double el = g->el0 + (v + 0.5) * g->del;
    /* exact solid angle of the pixel cell on the sphere */
    double domega = g->daz * (sin(el + 0.5 * g->del) - sin(el - 0.5 * g->del));
    double L = g->amb[idx];
    *a = (isfinite(L) ? L : 0.0) * domega;
    double rr = g->range[idx];
    *w = 0; *t0 = 0; *t1 = 0;
    if (!(isfinite(rr) && rr > 0.0)) return 0;
    double d[3];
    dir_of(az, el, d);
    double n[3] = {g->nx[idx], g->ny[idx], g->nz[idx]};
    double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    double beta = g->rho[idx] / ORC_PI + g->retro[idx];
    *w = beta * fabs(dn) / (rr * rr) * domega;
    /* orient the normal towards the sensor, clamp grazing incidence */
    double sgn = dn > 0 ? -1.0 : 1.0;
    double mu_p = fmax(-sgn * dn, ORC_MU_MIN);
    double rmin = rr, rmax = rr;
    for (int cj = -1; cj <= 1; cj += 2)
        for (int ci = -1; ci <= 1; ci += 2) {
            double dc[3];
            dir_of(az + 0.5 * ci * g->daz, el + 0.5 * cj * g->del, dc);
            double mu_c = fmax(-sgn * (dc[0] * n[0] + dc[1] * n[1] + dc[2] * n[2]), ORC_MU_MIN);
            double rc = rr * mu_p / mu_c;
            if (rc < rmin) rmin = rc;
            if (rc > rmax) rmax = rc;
        }
    *t0 = 2.0 * rmin / ORC_C_LIGHT;
    *t1 = 2.0 * rmax / ORC_C_LIGHT;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Range-bin deposit (Alg. 1 inner loop over [r0, r1])                       */
/* ------------------------------------------------------------------------ */

static double hat(double x) { double a = 1.0 - fabs(x); return a > 0 ? a : 0.0; }

/* D_k: mean of the hat function of bin k over [X0, X1], both in bin-centre
 * units (X = k at the centre of bin k). The interval is cut at the hat's
 * kinks; on each piece the hat is linear, so its mean there is its value at
 * the piece's midpoint. X1 == X0 gives the point value. */
double orc_deposit_weight(double X0, double X1, int k)
{
    double W = X1 - X0;
    if (!(W > 0.0)) return hat(X0 - k);
    double cuts[5] = {X0, k - 1.0, (double)k, k + 1.0, X1};
    double acc = 0.0, lo = X0;
    for (int c = 1; c < 5; ++c) {
        double hi = cuts[c];
        if (c < 4 && (hi <= lo || hi >= X1)) continue;
        if (c == 4) hi = X1;
        acc += (hi - lo) * hat(0.5 * (lo + hi) - k);
        lo = hi;
    }
    return acc / W;
}

/* ------------------------------------------------------------------------ */
/* Pulse varpi (EPW post-processing of Sec. II-C)                            */
/* ------------------------------------------------------------------------ */

/* Gaussian pulse of the given FWHM sampled at integer bin offsets -M..M,
 * M = ceil(trunc_sigmas * sigma_bins), normalised to unit sum. Returns M. */
int orc_pulse_taps(const orc_pulse *p, double *taps, int cap)
{
    double sigma = p->fwhm / (2.0 * sqrt(2.0 * log(2.0))) / p->dt;
    int M = (int)ceil(p->trunc_sigmas * sigma);
    if (2 * M + 1 > cap) return -1;
    double s = 0.0;
    for (int m = -M; m <= M; ++m) { taps[m + M] = exp(-0.5 * (m / sigma) * (m / sigma)); s += taps[m + M]; }
    for (int m = -M; m <= M; ++m) taps[m + M] /= s;
    return M;
}

/* xi_hat[k] = sum_m varpi[m] h[k - m] (zero outside the window) + A s_amb */
void orc_convolve(const double *h, int n, const double *taps, int M, double amb_level, double *out)
{
    for (int k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int m = -M; m <= M; ++m) {
            int j = k - m;
            if (j < 0 || j >= n) continue;
            acc += taps[m + M] * h[j];
        }
        out[k] = acc + amb_level;
    }
}

/* ------------------------------------------------------------------------ */
/* Echo extraction: maximal intervals with xi_hat > T (Sec. II-C), EPW, peak  */
/* ------------------------------------------------------------------------ */

static double bin_to_range(const orc_pulse *p, double x)
{
    return 0.5 * ORC_C_LIGHT * (p->t0 + (x + 0.5) * p->dt);
}

/* All runs in ascending bin order, at most max_out of them; returns the number
 * of runs written. */
int orc_extract_echoes(const double *xi, int n, const orc_pulse *p, const orc_calib *c,
                       orc_echo *out, int max_out)
{
    int cnt = 0;
    double T = c->T, eps = ORC_NEAR_REL * T;
    int k = 0;
    while (k < n && cnt < max_out) {
        if (!(xi[k] > T)) { ++k; continue; }
        int bs = k;
        while (k + 1 < n && xi[k + 1] > T) ++k;
        int be = k;
        ++k;
        orc_echo e;
        memset(&e, 0, sizeof e);
        e.bin_start = bs;
        e.bin_end = be;
        double x0, x1;
        if (bs > 0) x0 = (bs - 1) + (T - xi[bs - 1]) / (xi[bs] - xi[bs - 1]);
        else { x0 = 0.0; e.flags |= ORC_CLIPPED_START; }
        if (be < n - 1) x1 = be + (xi[be] - T) / (xi[be] - xi[be + 1]);
        else { x1 = n - 1.0; e.flags |= ORC_CLIPPED_END; }
        e.r0 = bin_to_range(p, x0);
        e.r1 = bin_to_range(p, x1);
        e.epw_m = e.r1 - e.r0;
        int kp = bs;
        for (int j = bs + 1; j <= be; ++j) if (xi[j] > xi[kp]) kp = j;
        e.bin_peak = kp;
        e.peak = xi[kp];
        double dlt = 0.0;
        if (kp > 0 && kp < n - 1) {
            double a = xi[kp - 1], b = xi[kp], cc = xi[kp + 1];
            if (a > 0 && b > 0 && cc > 0) {
                double la = log(a), lb = log(b), lc = log(cc);
                double den = la - 2.0 * lb + lc;
                if (den < 0) dlt = 0.5 * (la - lc) / den;
            } else {
                double den = a - 2.0 * b + cc;
                if (den < 0) dlt = 0.5 * (a - cc) / den;
            }
            if (dlt > 0.5) dlt = 0.5;
            if (dlt < -0.5) dlt = -0.5;
        }
        e.x_peak = kp + dlt;
        e.range_m = bin_to_range(p, kp + dlt);
        double E2 = e.epw_m * e.epw_m;
        e.intensity = exp(c->c0 + c->c1 * E2 + c->c2 * E2 * E2);
        for (int j = bs - 1; j <= be + 1; ++j)
            if (j >= 0 && j < n && fabs(xi[j] - T) <= eps) e.flags |= ORC_NEAR_THRESHOLD;
        for (int j = bs; j <= be; ++j)
            if (j != kp && xi[j] >= xi[kp] * (1.0 - ORC_NEAR_REL)) e.flags |= ORC_PEAK_AMBIGUOUS;
        out[cnt++] = e;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* EPW -> intensity calibration (Sec. II-C EPW; Sec. III-C threshold)         */
/* ------------------------------------------------------------------------ */

/* Sweep of a perpendicular point target of energy a (a single point deposit
 * at X = n/2 + phase, phase in {0, 1/4, 1/2, 3/4}) over 64 amplitudes
 * log-spaced from 50 T to 1e6 T, no ambient; least-squares fit of
 * ln a = c0 + c1 EPW^2 + c2 EPW^4 (EPW in metres) by the normal equations.
 * Returns the number of sweep points used, or -1. */
int orc_fit_epw(const orc_pulse *p, double T, double *coef)
{
    double taps[8192];
    int M = orc_pulse_taps(p, taps, 8192);
    if (M < 0) return -1;
    int n = 4 * M + 64;
    double *h = calloc(n, sizeof(double)), *xi = malloc(n * sizeof(double));
    double A[3][3] = {{0}}, b[3] = {0};
    orc_calib cal = {T, 0, 0, 0, 0};
    int used = 0;
    for (int ia = 0; ia < 64; ++ia) {
        double e = log10(50.0) + ia * (6.0 - log10(50.0)) / 63.0;
        double amp = T * pow(10.0, e);
        for (int ph = 0; ph < 4; ++ph) {
            double X = n / 2 + 0.25 * ph;
            memset(h, 0, n * sizeof(double));
            for (int k = 0; k < n; ++k) h[k] = amp * orc_deposit_weight(X, X, k);
            orc_convolve(h, n, taps, M, 0.0, xi);
            orc_echo ec[4];
            int ne = orc_extract_echoes(xi, n, p, &cal, ec, 4);
            if (ne != 1) continue;
            double E2 = ec[0].epw_m * ec[0].epw_m;
            double phi[3] = {1.0, E2, E2 * E2};
            double y = log(amp);
            for (int r = 0; r < 3; ++r) {
                b[r] += phi[r] * y;
                for (int q = 0; q < 3; ++q) A[r][q] += phi[r] * phi[q];
            }
            ++used;
        }
    }
    free(h); free(xi);
    /* Gaussian elimination with partial pivoting on the 3x3 system */
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r) if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int q = 0; q < 3; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        double t = b[col]; b[col] = b[piv]; b[piv] = t;
        for (int r = col + 1; r < 3; ++r) {
            double f = A[r][col] / A[col][col];
            for (int q = col; q < 3; ++q) A[r][q] -= f * A[col][q];
            b[r] -= f * b[col];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int q = r + 1; q < 3; ++q) s -= A[r][q] * coef[q];
        coef[r] = s / A[r][r];
    }
    return used;
}

/* ------------------------------------------------------------------------ */
/* Whole beam model (Alg. 1 with the post-processing of Sec. II-C)           */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_gbuffer *g;
    const orc_profile *p;
    double Z;
    const float *R, *dirs;
    const int32_t *beams;
    int n_sel;
    const orc_pulse *pu;
    const orc_calib *ca;
    double *h, *amb, *xi;
    orc_echo *echoes;
    int32_t *counts;
    int max_out;
    int tid, nthreads;
    const double *taps;
    int M;
} orc_job;

/* One beam: histogram h (before the pulse), ambient sum A and waveform xi. */
static void orc_one_beam(const orc_job *J, int sel)
{
    const orc_gbuffer *g = J->g;
    int nb = J->pu->n_bins;
    double *h = J->h + (long)sel * nb;
    double *xi = J->xi + (long)sel * nb;
    memset(h, 0, nb * sizeof(double));
    orc_frame f;
    int b = J->beams[sel];
    orc_beam_frame(J->R, J->dirs + 3 * (long)b, &f);
    double sup = orc_profile_support_deg(J->p) * ORC_DEG;
    double el_a = asin(fmax(-1.0, fmin(1.0, f.a[2])));
    double A = 0.0;
    for (int v = 0; v < g->V; ++v) {
        double el = g->el0 + (v + 0.5) * g->del;
        /* exact: the angle between two directions is at least their
         * elevation difference */
        if (fabs(el - el_a) > sup) continue;
        for (int u = 0; u < g->U; ++u) {
            double az = g->az0 + (u + 0.5) * g->daz;
            double d[3];
            dir_of(az, el, d);
            double uu, vv;
            if (!orc_local_offset(&f, d, &uu, &vv)) continue;
            double P = orc_profile_raw(J->p, uu, vv) / J->Z;
            if (!(P > 0.0)) continue;
            double w, t0, t1, a;
            int hit = orc_pixel(g, u, v, &w, &t0, &t1, &a);
            A += P * a;
            if (!hit) continue;
            double X0 = (t0 - J->pu->t0) / J->pu->dt - 0.5;
            double X1 = (t1 - J->pu->t0) / J->pu->dt - 0.5;
            long klo = (long)floor(X0) - 1, khi = (long)ceil(X1) + 1;
            if (klo < 0) klo = 0;
            if (khi > nb - 1) khi = nb - 1;
            for (long k = klo; k <= khi; ++k) h[k] += P * w * orc_deposit_weight(X0, X1, (int)k);
        }
    }
    J->amb[sel] = A;
    orc_convolve(h, nb, J->taps, J->M, A * J->ca->s_amb, xi);
    J->counts[sel] = orc_extract_echoes(xi, nb, J->pu, J->ca, J->echoes + (long)sel * J->max_out, J->max_out);
}

static void *orc_worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    for (int s = J->tid; s < J->n_sel; s += J->nthreads) orc_one_beam(J, s);
    return NULL;
}

/* Simulate the selected beams. h, xi: [n_sel][n_bins]; amb: [n_sel];
 * echoes: [n_sel][max_out]; counts: [n_sel]. Z = orc_profile_norm(p).
 * Returns 0 on success. */
int orc_simulate(const orc_gbuffer *g, const orc_profile *p, double Z, const float *R,
                 const float *dirs, const int32_t *beams, int n_sel, const orc_pulse *pu,
                 const orc_calib *ca, int nthreads, double *h, double *amb, double *xi,
                 orc_echo *echoes, int32_t *counts, int max_out)
{
    double *taps = malloc(16384 * sizeof(double));
    int M = orc_pulse_taps(pu, taps, 16384);
    if (M < 0) { free(taps); return -1; }
    if (nthreads < 1) nthreads = 1;
    orc_job *jobs = malloc(nthreads * sizeof(orc_job));
    pthread_t *th = malloc(nthreads * sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        orc_job J = {g, p, Z, R, dirs, beams, n_sel, pu, ca, h, amb, xi, echoes, counts,
                     max_out, t, nthreads, taps, M};
        jobs[t] = J;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    orc_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th); free(taps);
    return 0;
}

/* Per-pixel quantities of a whole G-buffer (for tests). */
void orc_pixels(const orc_gbuffer *g, double *w, double *t0, double *t1, double *a, int32_t *hit)
{
    for (int v = 0; v < g->V; ++v)
        for (int u = 0; u < g->U; ++u) {
            long i = (long)v * g->U + u;
            hit[i] = orc_pixel(g, u, v, &w[i], &t0[i], &t1[i], &a[i]);
        }
}

/* Local offsets of given directions for one beam (for tests). */
void orc_offsets(const float *R, const float *dir, const double *dirs3, int n, double *u, double *v,
                 int32_t *front)
{
    orc_frame f;
    orc_beam_frame(R, dir, &f);
    for (int i = 0; i < n; ++i) front[i] = orc_local_offset(&f, dirs3 + 3 * (long)i, &u[i], &v[i]);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (range stacking), nearest slice above threshold                    */
/* ------------------------------------------------------------------------ */

/* Per-pixel inputs of range stacking: intensity I = the pixel's received
 * power (rho_hat times its solid angle, 0 without a hit) and range index
 * floor(range / dr) (-1 without a hit). */
void orc_stack_inputs(const orc_gbuffer *g, double dr, double *I, int32_t *rbar)
{
    for (int v = 0; v < g->V; ++v)
        for (int u = 0; u < g->U; ++u) {
            long i = (long)v * g->U + u;
            double w, t0, t1, a;
            int hit = orc_pixel(g, u, v, &w, &t0, &t1, &a);
            I[i] = hit ? w : 0.0;
            rbar[i] = hit ? (int32_t)floor(g->range[i] / dr) : -1;
        }
}

/* Alg. 2: for s = s_max down to 1, the slice image (I where rbar == s, else
 * 0) is convolved with the centred kernel K[kh][kw] (zero outside the image:
 * out[v][u] = sum_{i,j} K[m + i][n + j] in[v - i][u - j], m = kh/2, n = kw/2),
 * and every pixel whose convolved value is >= thr takes s and that value.
 * Initial values: S = s_max, X = 0. Slices without a pixel are skipped (their
 * convolution is zero, below thr > 0). */
void orc_range_stack(int U, int V, const double *I, const int32_t *rbar, int kh, int kw, const double *K,
                     double thr, int s_max, int32_t *S, double *X)
{
    const int m = kh / 2, n = kw / 2;
    long np = (long)U * V;
    double *slice = malloc(np * sizeof(double));
    for (long i = 0; i < np; ++i) { S[i] = s_max; X[i] = 0.0; }
    for (int s = s_max; s >= 1; --s) {
        int any = 0;
        for (long i = 0; i < np; ++i) {
            slice[i] = rbar[i] == s ? I[i] : 0.0;
            if (rbar[i] == s) any = 1;
        }
        if (!any) continue;
        for (int v = 0; v < V; ++v)
            for (int u = 0; u < U; ++u) {
                double acc = 0.0;
                for (int i = -m; i <= m; ++i) {
                    int vv = v - i;
                    if (vv < 0 || vv >= V) continue;
                    for (int j = -n; j <= n; ++j) {
                        int uu = u - j;
                        if (uu < 0 || uu >= U) continue;
                        acc += K[(long)(m + i) * kw + (n + j)] * slice[(long)vv * U + uu];
                    }
                }
                if (acc >= thr) {
                    S[(long)v * U + u] = s;
                    X[(long)v * U + u] = acc;
                }
            }
    }
    free(slice);
}

/* Alg. 2 at single output pixels (v[q], u[q]), q < n: the same sums as
 * orc_range_stack (per slice s, sum over the kernel window of K * I on the
 * pixels of slice s, in the same (i, j) order, so the same rounding), and the
 * same answer: the nearest slice reaching the threshold (the last one the
 * far-to-near sweep writes), else s_max and 0. closest[q] = min over slices
 * s <= S of |sum_s - thr| / thr (how near a decision came to flipping). */
void orc_range_stack_at(int U, int V, const double *I, const int32_t *rbar, int kh, int kw, const double *K,
                        double thr, int s_max, int n, const int32_t *v, const int32_t *u, int32_t *S, double *X,
                        double *closest)
{
    const int m = kh / 2, h = kw / 2;
    double *acc = malloc((size_t)(s_max + 1) * sizeof(double));
    for (int q = 0; q < n; ++q) {
        for (int s = 0; s <= s_max; ++s) acc[s] = 0.0;
        for (int i = -m; i <= m; ++i) {
            int vv = v[q] - i;
            if (vv < 0 || vv >= V) continue;
            for (int j = -h; j <= h; ++j) {
                int uu = u[q] - j;
                if (uu < 0 || uu >= U) continue;
                int s = rbar[(long)vv * U + uu];
                if (s >= 1 && s <= s_max) acc[s] += K[(long)(m + i) * kw + (h + j)] * I[(long)vv * U + uu];
            }
        }
        S[q] = s_max;
        X[q] = 0.0;
        for (int s = 1; s <= s_max; ++s)
            if (acc[s] >= thr) { S[q] = s; X[q] = acc[s]; break; }
        double c = INFINITY;
        for (int s = 1; s <= S[q]; ++s) {
            double d = fabs(acc[s] - thr) / thr;
            if (d < c) c = d;
        }
        closest[q] = c;
    }
    free(acc);
}
