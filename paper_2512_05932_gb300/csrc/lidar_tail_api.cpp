// Host side of include/lidar_tail.h: the core/tail split (cell sums, per-beam
// bounds and prior, the split simulation with its exact re-run of beams that
// fail the acceptance test).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "lidar_host.h"
#include "lidar_internal.h"
#include "lidar_tail.h"
#include "lidar_tail_internal.h"

namespace gbl {

struct TailState {
    double core = 0.0;  // core radius (rad)
    int n_coarse = 0;
    // pulse constants of the acceptance test
    float pmax = 0.f, pl2 = 0.f, d1 = 0.f, d2 = 0.f, dd = 0.f;
    uint8_t *d_core = nullptr;      // [n_beams] all 1: every beam core-only in the split pass
    uint8_t *d_flags = nullptr;     // [n_beams]: 1 = re-run
    int *d_fb = nullptr;            // [1 + n_beams]: count, then the beams to re-run in order
    int *h_fb = nullptr;            // pinned copy of the count
    BeamParam *d_fb_beams = nullptr;
    float *d_box = nullptr;         // pulse averaged over the fine bins of a coarse bin (FootprintArgs::tail_box)
    int box_off = 0;
    int G_core = 4;                 // beams per CTA of the core pass (the sensor's)
    size_t smem_core = 0;
    int G_fb = 4;                   // beams per CTA of the exact re-run; the re-run beams are scattered,
    size_t smem_fb = 0;             // so each of a CTA's beams walks its own pixel box (lean phase 1)
    float4 *mip_s[kMipLevels] = {};
    float2 *mip_r[kMipLevels] = {};
    size_t mip_cap[kMipLevels] = {};
    float *d_rows = nullptr;        // lidar_simulate_surrogate: features, predicted tail, network input
    float *d_pred = nullptr;
    void *d_inputs = nullptr;
    float *d_wave = nullptr;        // waveform scratch of lidar_tail_exact
    lidar_echo_t *d_echo = nullptr;
    int32_t *d_counts = nullptr;
};

}  // namespace gbl

namespace gblh {

void tail_free(lidar_t *l)
{
    gbl::TailState *t = l->tail;
    if (!t) return;
    cudaFree(t->d_core);
    cudaFree(t->d_flags);
    cudaFree(t->d_fb);
    cudaFreeHost(t->h_fb);
    cudaFree(t->d_fb_beams);
    cudaFree(t->d_box);
    for (int i = 0; i < gbl::kMipLevels; ++i) {
        cudaFree(t->mip_s[i]);
        cudaFree(t->mip_r[i]);
    }
    cudaFree(t->d_rows);
    cudaFree(t->d_pred);
    cudaFree(t->d_inputs);
    cudaFree(t->d_wave);
    cudaFree(t->d_echo);
    cudaFree(t->d_counts);
    delete t;
    l->tail = nullptr;
}

}  // namespace gblh

using namespace gblh;

namespace {

lidar_status_t check_split(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, double R[9])
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (!l->tail) return fail(l, LIDAR_EINVAL, "lidar_tail_configure has not been called");
    lidar_status_t st = check_gbuffer(l, g);
    if (st != LIDAR_OK) return st;
    if (is_panorama(g) && g->U % 32 != 0)
        return fail(l, LIDAR_EINVAL, "a 2 pi panorama needs a width that is a multiple of 32 for the tail split");
    return check_pose(l, pose, R);
}

// Setup (pixels and/or beams) with every beam core-only or full.
lidar_status_t run_setup(lidar_t *l, const lidar_gbuffer_t *g, const double R[9], bool pixels, bool core,
                         cudaStream_t s)
{
    size_t np = (size_t)g->U * g->V;
    if (pixels) {
        lidar_status_t st = ensure_scratch(l, np);
        if (st != LIDAR_OK) return st;
    }
    gbl::SetupArgs sa = setup_args(l, l, g, R, l->d_rec, l->d_beams);
    if (!pixels) sa.pix_blocks = 0;
    sa.bin_records = 0;  // the split always uses the FP32 atomic deposit
    if (core) {
        sa.core_only = l->tail->d_core;
        sa.core_rad = l->tail->core;
    }
    cudaError_t e = gbl::launch_setup(sa, s);
    if (e != cudaSuccess) return cuda_fail(l, e, "setup kernel launch");
    return LIDAR_OK;
}

gbl::FootprintArgs frame_args(lidar_t *l, const lidar_gbuffer_t *g)
{
    gbl::FootprintArgs fa = model_args(l);
    fa.U = g->U; fa.V = g->V; fa.panorama = is_panorama(g) ? 1 : 0;
    fa.az0 = (float)g->az0; fa.el0 = (float)g->el0; fa.daz = (float)g->daz; fa.del = (float)g->del;
    fa.rec = l->d_rec;
    fa.beams = l->d_beams;
    fa.n_beams = l->n_beams;
    fa.inner2 = -1.f;
    fa.n_coarse = l->tail->n_coarse;
    fa.tail_stride = l->tail->n_coarse + 4;
    return fa;
}

lidar_status_t launch_fp(lidar_t *l, const gbl::FootprintArgs &fa, cudaStream_t s, bool rerun = false)
{
    const int G = rerun ? l->tail->G_fb : l->tail->G_core;
    const size_t smem = rerun ? l->tail->smem_fb : l->tail->smem_core;
    cudaError_t e = gbl::launch_footprint(l->kind, G, false, l->threads, smem, fa, s);
    if (e != cudaSuccess) return cuda_fail(l, e, "footprint kernel launch");
    return LIDAR_OK;
}

}  // namespace

extern "C" {

lidar_status_t lidar_tail_configure(lidar_t *l, double core_deg, int32_t n_coarse)
{
    if (!l) return fail(nullptr, LIDAR_EINVAL, "lidar is NULL");
    if (l->kind != LIDAR_PROFILE_RADIAL) return fail(l, LIDAR_EINVAL, "the tail split needs a radial profile");
    const double core = core_deg * kDeg;
    if (!(std::isfinite(core_deg) && core > 0.0 && core < l->support_rad))
        return fail(l, LIDAR_EINVAL, "core_deg must be in (0, truncation)");
    if (n_coarse < 1 || n_coarse > 1024 || l->n_bins % n_coarse != 0)
        return fail(l, LIDAR_EINVAL, "n_coarse must divide n_bins and be in [1, 1024]");
    tail_free(l);
    gbl::TailState *t = new (std::nothrow) gbl::TailState();
    if (!t) return fail(l, LIDAR_ENOMEM, "host allocation failed");
    l->tail = t;
    t->core = core;
    t->n_coarse = n_coarse;
    // pulse constants from the FP32 taps the kernels use
    std::vector<float> tp(l->tp_len);
    cudaError_t e = cudaMemcpy(tp.data(), l->d_taps, tp.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { tail_free(l); return cuda_fail(l, e, "pulse taps download"); }
    const int M = l->M;
    auto p = [&](int m) -> double { return (m < -M || m > M) ? 0.0 : (double)tp[l->tp_off + m]; };
    double pmax = 0, s2 = 0, d1 = 0, d2 = 0, dd = 0;
    for (int m = -M - 2; m <= M + 2; ++m) {
        pmax = std::max(pmax, p(m));
        s2 += p(m) * p(m);
        d1 = std::max(d1, std::fabs(p(m + 1) - p(m)));
        d2 = std::max(d2, std::fabs(p(m + 2) - p(m)));
        dd = std::max(dd, std::fabs(p(m + 1) - 2 * p(m) + p(m - 1)));
    }
    const double up = 1.0 + 1e-5;
    t->pmax = (float)(pmax * up); t->pl2 = (float)(std::sqrt(s2) * up);
    t->d1 = (float)(d1 * up); t->d2 = (float)(d2 * up); t->dd = (float)(dd * up);
    // B(x) = (1/cf) sum_{j < cf} p(x - j), x in [-M - 7, M + cf + 6]
    const int cf = l->n_bins / n_coarse;
    t->box_off = (M + 7 + 3) & ~3;  // multiple of 4: aligned 16-byte loads in the kernel
    std::vector<float> box(((t->box_off + M + cf + 7) + 3) & ~3, 0.f);
    for (int x = -M - 7; x <= M + cf + 6; ++x) {
        double acc = 0;
        for (int j = 0; j < cf; ++j) acc += p(x - j);
        box[x + t->box_off] = (float)(acc / cf);
    }
    t->G_core = l->G;
    {
        // four re-run beams per CTA where their histograms fit, else one
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, l->device);
        if ((long)gbl::footprint_smem_bytes(4, model_args(l)) > optin) t->G_fb = 1;
    }
    t->smem_fb = gbl::footprint_smem_bytes(t->G_fb, model_args(l));
    t->smem_core = gbl::footprint_smem_bytes(t->G_core, model_args(l));
    if ((e = gbl::prepare_footprint(l->kind, t->G_fb, false, t->smem_fb)) != cudaSuccess ||
        (e = gbl::prepare_footprint(l->kind, t->G_core, false, t->smem_core)) != cudaSuccess) {
        tail_free(l);
        return cuda_fail(l, e, "cudaFuncSetAttribute");
    }
    std::vector<uint8_t> ones(l->n_beams, 1);
    if ((e = cudaMalloc(&t->d_core, l->n_beams)) != cudaSuccess ||
        (e = cudaMemcpy(t->d_core, ones.data(), l->n_beams, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&t->d_flags, l->n_beams)) != cudaSuccess ||
        (e = cudaMalloc(&t->d_fb, (size_t)(l->n_beams + 1) * sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&t->h_fb, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&t->d_fb_beams, (size_t)l->n_beams * sizeof(gbl::BeamParam))) != cudaSuccess ||
        (e = cudaMalloc(&t->d_box, box.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMemcpy(t->d_box, box.data(), box.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
        tail_free(l);
        return cuda_fail(l, e, "cudaMalloc(tail split buffers)");
    }
    return LIDAR_OK;
}

lidar_status_t lidar_tail_features(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *rows,
                                   void *inputs, void *stream)
{
    double R[9];
    lidar_status_t st = check_split(l, g, pose, R);
    if (st != LIDAR_OK) return st;
    if (!rows) return fail(l, LIDAR_EINVAL, "rows is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    gbl::TailState *t = l->tail;
    if ((st = run_setup(l, g, R, false, true, s)) != LIDAR_OK) return st;
    // cell sums
    gbl::MipArgs ma{};
    ma.U = g->U; ma.V = g->V;
    ma.az0 = (float)g->az0; ma.el0 = (float)g->el0; ma.daz = (float)g->daz; ma.del = (float)g->del;
    ma.sv = (float)std::sin(0.5 * g->del);
    ma.range = g->range; ma.nx = g->nx; ma.ny = g->ny; ma.nz = g->nz;
    ma.rho = g->rho_d; ma.retro = g->retro; ma.amb = g->ambient;
    cudaError_t e;
    for (int i = 0; i < gbl::kMipLevels; ++i) {
        const int side = 4 << i;
        ma.ncx[i] = (g->U + side - 1) / side;
        ma.ncy[i] = (g->V + side - 1) / side;
        const size_t n = (size_t)ma.ncx[i] * ma.ncy[i];
        if (n > t->mip_cap[i]) {
            cudaFree(t->mip_s[i]);
            cudaFree(t->mip_r[i]);
            t->mip_s[i] = nullptr; t->mip_r[i] = nullptr; t->mip_cap[i] = 0;
            if ((e = cudaMalloc(&t->mip_s[i], n * sizeof(float4))) != cudaSuccess ||
                (e = cudaMalloc(&t->mip_r[i], n * sizeof(float2))) != cudaSuccess)
                return cuda_fail(l, e, "cudaMalloc(cell sums)");
            t->mip_cap[i] = n;
        }
        ma.s[i] = t->mip_s[i];
        ma.r[i] = t->mip_r[i];
    }
    if ((e = gbl::launch_tail_mips(ma, s)) != cudaSuccess) return cuda_fail(l, e, "cell-sum kernel launch");
    // per-beam bounds, prior and network input
    gbl::PrepArgs pa{};
    pa.U = g->U; pa.V = g->V; pa.panorama = is_panorama(g) ? 1 : 0;
    pa.daz = (float)g->daz; pa.del = (float)g->del;
    pa.beams = l->d_beams;
    pa.n_beams = l->n_beams;
    pa.kg = l->kg; pa.trunc2 = l->trunc2; pa.tail_amp = l->tail_amp; pa.tc2_inv = l->tc2_inv;
    pa.tail_hp = l->tail_hp; pa.invZ = (float)(1.0 / l->Z);
    pa.core = (float)t->core;
    pa.trunc = (float)l->support_rad;
    // cell radius bound (half-extent between the outer pixel centres), per level
    auto cell_rho = [&](int side) {
        const double h = 0.5 * (side - 1);
        return 1.0001 * std::sqrt(std::pow(h * g->daz, 2) + std::pow(h * g->del, 2));
    };
    pa.rho_top = (float)cell_rho(4 << (gbl::kQuadLevels - 1));
    // a cell is refined while its nearest point is closer than 8 of its
    // radii: there a power-law profile changes by more than ~1.5x across it
    pa.refine[0] = 0.f;
    for (int i = 1; i < gbl::kQuadLevels; ++i) pa.refine[i] = (float)(8.0 * cell_rho(4 << i));
    for (int i = 0; i < gbl::kMipLevels; ++i) {
        pa.ncx[i] = ma.ncx[i]; pa.ncy[i] = ma.ncy[i];
        pa.s[i] = ma.s[i]; pa.r[i] = ma.r[i];
    }
    pa.x_scale = (float)(2.0 / (kC * l->dt));
    pa.x_off = (float)(-l->t0 / l->dt - 0.5);
    pa.inv_cf = (float)((double)t->n_coarse / l->n_bins);
    pa.inv_nb = (float)(1.0 / l->n_bins);
    pa.n_coarse = t->n_coarse;
    pa.prior = rows;
    pa.inputs = inputs;
    if ((e = gbl::launch_tail_prep(pa, s)) != cudaSuccess) return cuda_fail(l, e, "tail prep kernel launch");
    return LIDAR_OK;
}

lidar_status_t lidar_tail_exact(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, float *rows,
                                void *stream)
{
    double R[9];
    lidar_status_t st = check_split(l, g, pose, R);
    if (st != LIDAR_OK) return st;
    if (!rows) return fail(l, LIDAR_EINVAL, "rows is NULL");
    gbl::TailState *t = l->tail;
    cudaError_t e;
    if (!t->d_wave) {
        if ((e = cudaMalloc(&t->d_wave, (size_t)l->n_beams * l->n_bins * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&t->d_echo, (size_t)l->n_beams * l->max_echoes * sizeof(lidar_echo_t))) != cudaSuccess ||
            (e = cudaMalloc(&t->d_counts, (size_t)l->n_beams * sizeof(int32_t))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(tail waveform scratch)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = run_setup(l, g, R, true, false, s)) != LIDAR_OK) return st;
    gbl::FootprintArgs fa = frame_args(l, g);
    const float c2 = (float)t->core;
    fa.inner2 = c2 * c2;
    fa.coarse_out = rows;
    fa.wave = t->d_wave; fa.echoes = t->d_echo; fa.counts = t->d_counts;
    return launch_fp(l, fa, s);
}

lidar_status_t lidar_simulate_split(lidar_t *l, const lidar_gbuffer_t *g, const lidar_pose_t *pose, const float *tail,
                                    float *wave, lidar_echoes_t *echoes, int32_t *n_fallback, void *stream)
{
    double R[9];
    lidar_status_t st = check_split(l, g, pose, R);
    if (st != LIDAR_OK) return st;
    if (!tail || !wave || !echoes || !echoes->echoes || !echoes->counts)
        return fail(l, LIDAR_EINVAL, "tail or output pointer is NULL");
    gbl::TailState *t = l->tail;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    // pass 1: exact core of every beam + the given tail, acceptance test
    if ((st = run_setup(l, g, R, true, true, s)) != LIDAR_OK) return st;
    if ((e = cudaMemsetAsync(t->d_flags, 0, l->n_beams, s)) != cudaSuccess) return cuda_fail(l, e, "cudaMemsetAsync");
    gbl::FootprintArgs fa = frame_args(l, g);
    const float c = (float)t->core;
    fa.core2 = c * c;
    fa.tail_in = tail;
    fa.tail_box = t->d_box;
    fa.tb_off = t->box_off;
    fa.g_pmax = t->pmax; fa.g_pl2 = t->pl2; fa.g_d1 = t->d1; fa.g_d2 = t->d2; fa.g_dd = t->dd;
    fa.g_l2 = 5e-4f;
    fa.g_dr = 2.5e-4f;
    fa.fb_flags = t->d_flags;
    fa.wave = wave; fa.echoes = echoes->echoes; fa.counts = echoes->counts;
    if ((st = launch_fp(l, fa, s)) != LIDAR_OK) return st;
    if ((e = gbl::launch_compact(t->d_flags, l->n_beams, t->d_fb, s)) != cudaSuccess)
        return cuda_fail(l, e, "compaction kernel launch");
    if ((e = cudaMemcpyAsync(t->h_fb, t->d_fb, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(l, e, "re-run count download");
    const int nfb = *t->h_fb;
    if (n_fallback) *n_fallback = nfb;
    if (nfb <= 0) return LIDAR_OK;
    // pass 2: the failing beams with the full profile, written to their own rows
    gbl::SetupArgs sa = setup_args(l, l, g, R, l->d_rec, t->d_fb_beams);
    sa.pix_blocks = 0;
    sa.bin_records = 0;
    sa.n_beams = nfb;
    sa.beam_ids = t->d_fb + 1;
    if ((e = gbl::launch_setup(sa, s)) != cudaSuccess) return cuda_fail(l, e, "setup kernel launch");
    gbl::FootprintArgs fb = frame_args(l, g);
    fb.beams = t->d_fb_beams;
    fb.n_beams = nfb;
    fb.out_ids = t->d_fb + 1;
    fb.wave = wave; fb.echoes = echoes->echoes; fb.counts = echoes->counts;
    return launch_fp(l, fb, s, true);
}

lidar_status_t lidar_simulate_surrogate(lidar_t *l, lidar_tailnet_t *net, const lidar_gbuffer_t *g,
                                        const lidar_pose_t *pose, float *wave, lidar_echoes_t *echoes,
                                        int32_t *n_fallback, void *stream)
{
    double R[9];
    lidar_status_t st = check_split(l, g, pose, R);
    if (st != LIDAR_OK) return st;
    gbl::TailState *t = l->tail;
    const size_t rs = (size_t)t->n_coarse + 4;
    cudaError_t e;
    if (!t->d_rows) {
        if ((e = cudaMalloc(&t->d_rows, l->n_beams * rs * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&t->d_pred, l->n_beams * rs * sizeof(float))) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(surrogate rows)");
    }
    if (net && !t->d_inputs) {
        if ((e = cudaMalloc(&t->d_inputs, (size_t)l->n_beams * LIDAR_TAIL_INPUT_CELLS * 4)) != cudaSuccess)
            return cuda_fail(l, e, "cudaMalloc(network input)");
    }
    if ((st = lidar_tail_features(l, g, pose, t->d_rows, net ? t->d_inputs : nullptr, stream)) != LIDAR_OK) return st;
    const float *tail = t->d_rows;
    if (net) {
        if ((st = lidar_tailnet_predict(net, t->d_inputs, t->d_rows, l->n_beams, t->d_pred, stream)) != LIDAR_OK)
            return fail(l, st, "tail network: %s", lidar_tailnet_last_error(net));
        tail = t->d_pred;
    }
    if ((st = lidar_simulate_split(l, g, pose, tail, wave, echoes, n_fallback, stream)) != LIDAR_OK) return st;
    if (net && (st = lidar_tailnet_sync(net, stream)) != LIDAR_OK)
        return fail(l, st, "tail network: %s", lidar_tailnet_last_error(net));
    return LIDAR_OK;
}

}  // extern "C"
