// Footprint deposit on the 5th-generation tensor cores (tcgen05, sm_103a),
// included by lidar_kernels.cu (it uses that file's profile evaluation,
// layout helpers and phases 2-4).
//
// A CTA takes a group of kUN = 16 beams. Their histograms h_b[k] live in
// tensor memory for the whole deposit phase: TMEM lane l of column
// blk * 16 + j holds bin 128 blk + l of beam j (FP32). The union pixel box is
// walked in tiles of kUK = 64 consecutive pixels of a row, and for every
// 128-bin block the tile's deposits reach, one 128 x 16 x 64 product
//     h[128 blk .. +127][j] += sum_p A[k][p] * B[p][j]
// is issued: A[k][p] = w_p D_k(p), the pixel's power times its hat weight on
// bin k (the setup kernel's record, beam-independent: written once per pixel
// per CTA, not once per (beam, pixel) pair), B[p][j] = P_j(p), the profile
// weight of beam j at pixel p (Eq. centered kernel). Operands are 16-bit
// (BF16, or FP16 with power-of-two scales), products are accumulated in FP32.
//
// Roles: warp 0, lane 0 issues the MMAs (one stage after the other); warps
// 1..kUP are producers. A producer warp takes a tile from a counter, builds
// B (lane (j, h): beam j, pixels 32h..32h+31, profile in FP32, ambient
// sum_p P_j(p) L_amb dω in FP32), then for each block the tile reaches
// claims the next stage of a kUS-deep ring (a sequence number from a shared
// counter; before reusing a stage it waits until the issuer has issued the
// stage's previous fill, then on its "empty" barrier), clears the rows its A
// buffer held, writes the tile's hat weights (lane p: pixels p, p + 32) and B,
// and arrives on the stage's "full" mbarrier; the issuer takes the stages in
// sequence order, issues four K = 16 MMAs per stage and commits them to the
// stage's "empty" mbarrier. Operand
// buffers use the K-major 128-byte swizzled layout (16-byte chunk c of row r
// at chunk c ^ (r & 7)), rows of 64 16-bit values.
// After the last tile, the histograms are read back (tcgen05.ld) kUG beams at
// a time into shared memory and finished by the phases of the FP32 kernel
// (window edges, pulse convolution + ambient, echoes).
//
// Scaling (FP16): B is multiplied by 2^eB so that the profile's maximum maps
// to about 2^14, A by 2^eA so that the frame's largest record weight does;
// both are per-CTA constants, so every product of the accumulation carries
// the same factor 2^(eA + eB), removed in FP32 at read-back. BF16 shares
// FP32's exponent range and runs unscaled.
//
// Every mbarrier wait is bounded; on expiry the CTA records an error in
// A.err (reported as LIDAR_ETIMEOUT by lidar_sync), waits (bounded) for its
// MMAs, frees its tensor memory and returns without writing its beams.

namespace umd {

constexpr int kUN = 16;                        // beams per CTA (MMA N)
constexpr int kUK = 64;                        // pixels per tile (MMA K: four steps of 16)
constexpr int kUMr = 128;                      // bins per block (MMA M, TMEM lanes)
constexpr int kUS = 8;                         // stages of the operand ring
constexpr int kUP = 16;                        // producer warps
constexpr int kUThreads = 32 * (kUP + 1);
constexpr uint32_t kUA = kUMr * 128;           // A buffer: 128 rows x 128 bytes
constexpr uint32_t kUB = kUN * 128;            // B buffer: 16 rows x 128 bytes
constexpr long kUWait = 1L << 22;              // bounded mbarrier polls
constexpr int kUTab = 128;                     // columns per offset-table stripe (2 tiles)

struct UmSmem {  // at a 1024-byte aligned offset (swizzle atoms)
    unsigned char a[kUS][kUA];
    unsigned char b[kUS][kUB];
    uint64_t full[kUS], empty[kUS], done;
    int blk[kUS];
    int clr_lo[kUS], clr_hi[kUS];  // rows of the stage's A written by its last use
    uint32_t tmem;
    int seq, seq_total, prod_done, abort, touched, ctr;
    int issued;  // stages whose MMAs the issuer has issued and committed (monotonic)
    int where;  // first wait that gave up: site << 28 | its sequence number << 14 | stages claimed
    float scale_a, scale_b;
};

// Records the first wait that gave up (for the error word) and stops the pipeline.
__device__ __forceinline__ void um_fail(UmSmem &S, int site, int seq)
{
    atomicCAS(&S.where, 0, (site << 28) | ((seq & 0x3FFF) << 14) | (*(volatile int *)&S.seq & 0x3FFF));
    atomicExch(&S.abort, 1);
}

struct UmLayout {
    Layout fin;       // hbuf / taps of the finishing phases (kUG beams at a time)
    int G;            // kUG
    size_t off_um, off_hbuf, off_taps, off_amb, off_nrm, off_tmass, off_supp, off_tsupp, off_tab, off_bp, off_pix,
        total;
};

// Beams per finishing round: the largest of 8, 4, 2 whose histograms fit
// next to the ring and the tables.
__host__ __device__ inline UmLayout um_layout(int n_bins, int M)
{
    UmLayout L;
    int G = 8;
    for (;; G >>= 1) {
        L.fin = make_layout(G, n_bins, M);
        L.G = G;
        size_t off = sizeof(UmSmem) + 1024;  // + alignment slack
        L.off_um = 0;
        L.off_hbuf = off; off += (size_t)G * L.fin.HB * 4;
        L.off_taps = off; off += (size_t)(skew_pos(L.fin.taps_len) + 1) * 4;
        L.off_amb = off; off += kUN * 4;
        L.off_nrm = off; off += kUN * 4;
        L.off_tmass = off; off += kUN * 4;
        L.off_supp = off; off += kUN * 8;
        L.off_tsupp = off; off += kUN * 8;
        off = (off + 15) & ~(size_t)15;
        L.off_tab = off; off += (size_t)kUN * kUTab * sizeof(float2);
        L.off_bp = off; off += (size_t)kUN * sizeof(BeamParam);
        L.off_pix = off; off += (size_t)kUP * kUK * sizeof(float2);
        L.total = off;
        if (L.total <= 227 * 1024 || G == 2) break;
    }
    return L;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 128-byte swizzled operand: start >> 4, LBO 16 (unused), SBO 1024
// (8 rows x 128 B), descriptor version, swizzle mode 2.
__device__ __forceinline__ uint64_t um_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// kind::f16 instruction descriptor: FP32 accumulator, A and B both BF16
// (bf16 = true) or both FP16, K-major, N = 16, M = 128.
__device__ __forceinline__ uint32_t um_idesc(bool bf16)
{
    const uint32_t ab = bf16 ? ((1u << 7) | (1u << 10)) : 0u;
    return (1u << 4) | ab | ((uint32_t)(kUN >> 3) << 17) | ((uint32_t)(kUMr >> 4) << 24);
}

__device__ __forceinline__ bool um_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t parity)
{
    for (long i = 0; i < kUWait; ++i) {
        if (um_try(bar, parity)) return true;
        if (i >= 8) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void um_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void um_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void um_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Producer-warp barrier (named barrier 1; the issuer warp does not take part).
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kUP) : "memory"); }

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    uint32_t r;
    if (BF16) asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

template <bool BF16>
__device__ __forceinline__ unsigned short pack1(float v)
{
    return (unsigned short)(pack2<BF16>(v, 0.f) & 0xFFFFu);
}

// Byte offset of element (row r, column k < 64) in a 128-byte swizzled
// K-major buffer of 16-bit values.
__device__ __forceinline__ uint32_t swz(int r, int k)
{
    return (uint32_t)(r * 128 + ((((k >> 3) ^ r) & 7) << 4) + ((k & 7) << 1));
}

}  // namespace umd

// One group of kUN beams of one frame on the tensor cores. Every thread of
// the CTA calls it; tmem is the CTA's allocation (at least nblk * 16 columns),
// `item` counts the groups this CTA has run before (mbarrier phases).
template <int KIND, bool BF16>
__device__ void footprint_umma_group(const FootprintArgs &A, const int group, unsigned char *smem_raw,
                                     umd::UmSmem &S, const umd::UmLayout &UL, uint32_t tmem, int item)
{
    using namespace umd;
    const int nb = A.n_bins, M = A.M;
    const Layout &Ly = UL.fin;
    float *hbuf = reinterpret_cast<float *>(smem_raw + UL.off_hbuf);
    float *taps = reinterpret_cast<float *>(smem_raw + UL.off_taps);
    float *amb_s = reinterpret_cast<float *>(smem_raw + UL.off_amb);
    float *nrm2_s = reinterpret_cast<float *>(smem_raw + UL.off_nrm);
    float *tmass_s = reinterpret_cast<float *>(smem_raw + UL.off_tmass);
    int *supp = reinterpret_cast<int *>(smem_raw + UL.off_supp);
    int *tsupp = reinterpret_cast<int *>(smem_raw + UL.off_tsupp);
    float2 *tab = reinterpret_cast<float2 *>(smem_raw + UL.off_tab);
    BeamParam *bp = reinterpret_cast<BeamParam *>(smem_raw + UL.off_bp);
    float2 *pixall = reinterpret_cast<float2 *>(smem_raw + UL.off_pix);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b0 = group * kUN;
    const int gcount = min(kUN, A.n_beams - b0);
    const int nblk = (nb + kUMr - 1) / kUMr;  // <= 32 (checked by the host)

    // ---- phase 0: parameters, union box ----------------------------------
    for (int i = tid; i < Ly.taps_len; i += blockDim.x) {
        int m = i - Ly.taps_off;
        taps[skew_pos(i)] = (m >= -M && m <= M) ? A.taps_pad[A.tp_off + m] : 0.f;
    }
    if (tid < kUN) {
        amb_s[tid] = 0.f;
        nrm2_s[tid] = 0.f;
        tmass_s[tid] = 0.f;
        BeamParam P;
        if (tid < gcount) P = A.beams[b0 + tid];
        else { P = BeamParam{}; P.valid = 0; }
        bp[tid] = P;
    }
    if (tid == 0) {
        S.seq_total = -1;
        S.prod_done = 0;
        S.touched = 0;
    }
    __syncthreads();
    if (tid < kUN && A.panorama) {
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
    int R0 = 1 << 30, R1 = -(1 << 30), C0 = 1 << 30, C1 = -(1 << 30);
    for (int j = 0; j < gcount; ++j) {
        const BeamParam &P = bp[j];
        if (!P.valid) continue;
        R0 = min(R0, P.row0); R1 = max(R1, P.row1);
        C0 = min(C0, P.col0); C1 = max(C1, P.col1);
    }
    const uint32_t idesc = um_idesc(BF16);
    const int seq0 = S.seq;  // stages of earlier groups of this CTA (read before any claim)
    __syncthreads();

    if (warp == 0) {
        // ---- MMA issuer ----------------------------------------------------
        if (lane == 0) {
            int seq = seq0;
            uint32_t touched = 0;
            long polls = 0;
            for (;;) {
                const int s = seq % kUS;
                const uint32_t par = (uint32_t)((seq / kUS) & 1);
                if (!um_try(su32(&S.full[s]), par)) {
                    if (*(volatile int *)&S.prod_done && *(volatile int *)&S.seq_total == seq) break;
                    if (*(volatile int *)&S.abort) break;
                    if (++polls > kUWait) { um_fail(S, 1, seq); break; }
                    if (polls > 8) __nanosleep(32);
                    continue;
                }
                polls = 0;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int blk = S.blk[s];
                const uint32_t acc0 = (touched >> blk) & 1u;
                const uint32_t a0 = su32(S.a[s]), bb0 = su32(S.b[s]);
#pragma unroll
                for (int kk = 0; kk < kUK / 16; ++kk)
                    um_mma(tmem + (uint32_t)(blk * kUN), um_desc(a0 + 32u * kk), um_desc(bb0 + 32u * kk), idesc,
                           (kk > 0 || acc0) ? 1u : 0u);
                touched |= 1u << blk;
                um_commit(su32(&S.empty[s]));
                ++seq;
                __threadfence_block();
                *(volatile int *)&S.issued = seq;
            }
            S.touched = (int)touched;
            um_commit(su32(&S.done));  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        // ---- producers -----------------------------------------------------
        const int pw = warp - 1, ptid = tid - 32;
        // the tile's pixels as this warp's lanes loaded them: (record word 0, ambient)
        float2 *pix = pixall + pw * kUK;
        const int j = lane & 15, h = lane >> 4;  // B: beam j, pixels 32h .. 32h + 31 of a tile
        const BeamParam P = bp[j];
        const bool jok = (j < gcount) && P.valid;
        const float t2max = P.pad0 ? A.core2 : A.trunc2;
        const float sa = S.scale_a, sb = S.scale_b;
        float amb_acc = 0.f;
        for (int cs = C0; cs <= C1 && R0 <= R1; cs += kUTab) {
            const int ce = min(C1, cs + kUTab - 1);
            const int ncs = ce - cs + 1;
            prod_sync();  // previous stripe's table no longer read
            for (int i = ptid; i < kUN * ncs; i += 32 * kUP) {
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
                tab[jj * kUTab + cc] = make_float2(sD, vers);
            }
            if (ptid == 0) S.ctr = kUP;
            prod_sync();
            const float2 *tjc = tab + j * kUTab - cs;
            const int ntile = (ncs + kUK - 1) / kUK;
            const int nunits = (R1 - R0 + 1) * ntile;
            // after an abort the loops below do no work, but every producer
            // still reaches the stripe barriers
            for (int unit = *(volatile int *)&S.abort ? nunits : pw; unit < nunits;) {
                const int row = R0 + unit / ntile;
                const int c_lo = cs + (unit - (unit / ntile) * ntile) * kUK;
                const int c_hi = min(ce, c_lo + kUK - 1);
                const float4 *recrow = A.rec + 2 * (size_t)row * A.U;
                // (1) the tile's records: lane p holds pixels p and p + 32;
                // mask of the 128-bin blocks their deposits reach
                float4 q0[2], q1[2];
                uint32_t bmask = 0;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int c = c_lo + lane + 32 * i;
                    int cw = c;
                    if (A.panorama) {
                        if (cw < 0) cw += A.U;
                        else if (cw >= A.U) cw -= A.U;
                        if ((unsigned)cw >= (unsigned)A.U) { cw = c % A.U; if (cw < 0) cw += A.U; }
                    }
                    const bool in = c <= c_hi;
                    q0[i] = in ? __ldg(recrow + 2 * cw) : make_float4(__uint_as_float(kNoDeposit), 0.f, 0.f, 0.f);
                    q1[i] = in ? __ldg(recrow + 2 * cw + 1) : make_float4(__uint_as_float(kNoDeposit), 0.f, 0.f, 0.f);
                    pix[lane + 32 * i] = make_float2(q0[i].x, q0[i].y);
                    const uint32_t kab = __float_as_uint(q0[i].x);
                    if (kab != kNoDeposit) {
                        const int f = (int)(kab & 0xFFFFu) - kBinBias;
                        const bool narrow = __float_as_uint(q1[i].x) != kNoDeposit;
                        const int lo = max(f, 0);
                        const int hi = min(narrow ? f + 3 : (int)(kab >> 16) - kBinBias + 1, nb - 1);
                        if (lo <= hi) {
                            const int bl = lo / kUMr, bh = hi / kUMr;  // 0 <= bl <= bh < nblk <= 32
                            bmask |= (bh == 31 ? 0xFFFFFFFFu : ((1u << (bh + 1)) - 1u)) & ~((1u << bl) - 1u);
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bmask |= __shfl_xor_sync(0xffffffffu, bmask, o);
                __syncwarp();  // the pixel table is written
                // (2) B: beam j at pixels 32h .. 32h + 31, profile and ambient in FP32
                uint32_t bw[16];
                const float cosEl = cosf(A.el0 + ((float)row + 0.5f) * A.del);
                float sdEl, cdEl;
                sincosf(((float)(row - P.ri) - P.rf) * A.del, &sdEl, &cdEl);
                const float Kv = P.sin_elb * cosEl, Kc = P.cos_elb * cosEl;
                const float ax = P.cg * cosEl, bx = P.sg * Kv, cx = P.sg * sdEl;
                const float ay = -P.sg * cosEl, by = P.cg * Kv, cy = P.cg * sdEl;
                const bool rowok = jok && row >= P.row0 && row <= P.row1;
                const int my_lo = max(c_lo, P.col0), my_hi = min(c_hi, P.col1);
#pragma unroll
                for (int t2 = 0; t2 < 16; ++t2) {
                    float pv[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int tc = 32 * h + 2 * t2 + e;  // column within the tile
                        const int c = c_lo + tc;
                        bool ok = rowok && c >= my_lo && c <= my_hi;
                        // the record's first word and ambient, from the warp's pixel table
                        const float2 ka = ok ? pix[tc] : make_float2(__uint_as_float(kNoDeposit), 0.f);
                        const bool dep = __float_as_uint(ka.x) != kNoDeposit;
                        ok = ok && (dep || ka.y != 0.f);
                        const float2 tt = tjc[ok ? c : cs];
                        ok = ok && fmaf(-Kc, tt.y, cdEl) > 0.f;
                        const float x = fmaf(ax, tt.x, fmaf(bx, tt.y, cx));
                        const float y = fmaf(ay, tt.x, fmaf(by, tt.y, cy));
                        const float Pw = profile_finish<KIND>(A, profile_fetch<KIND>(A, x, y, ok, t2max));
                        amb_acc = fmaf(Pw, ka.y, amb_acc);
                        pv[e] = dep ? Pw * sb : 0.f;
                    }
                    bw[t2] = pack2<BF16>(pv[0], pv[1]);
                }
                // (3) one stage per 128-bin block the tile reaches
                while (bmask) {
                    const int blk = __ffs(bmask) - 1;
                    bmask &= bmask - 1;
                    int seq = 0;
                    if (lane == 0) seq = atomicAdd(&S.seq, 1);
                    seq = __shfl_sync(0xffffffffu, seq, 0);
                    const int s = seq % kUS;
                    // Stage reuse: stage s was last filled with seq - kUS. Its "empty"
                    // barrier can be waited on by parity only once the issuer has
                    // issued that fill (before, the barrier may be two phases behind
                    // and an old phase of the same parity would pass the wait), so
                    // first wait for the issuer to reach it.
                    int okw = 1;
                    if (lane == 0 && seq >= kUS) {
                        long w = 0;
                        while (*(volatile int *)&S.issued <= seq - kUS && !*(volatile int *)&S.abort) {
                            if (++w > kUWait) break;
                            if (w > 8) __nanosleep(32);
                        }
                        __threadfence_block();
                        if (*(volatile int *)&S.issued <= seq - kUS) {
                            um_fail(S, 4, seq);
                            okw = 0;
                        } else if (!um_wait(su32(&S.empty[s]), (uint32_t)(((seq / kUS) - 1) & 1))) {
                            um_fail(S, 2, seq);
                            okw = 0;
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, okw, 0)) break;  // the issuer stops at this stage
                    unsigned char *Ab = S.a[s];
                    // clear the rows the stage's previous tile wrote
                    const int r0 = S.clr_lo[s], r1 = S.clr_hi[s];
                    for (int i = lane; i < (r1 - r0 + 1) * 8; i += 32)
                        *reinterpret_cast<uint4 *>(Ab + (r0 + i / 8) * 128 + (i % 8) * 16) = make_uint4(0u, 0u, 0u, 0u);
                    __syncwarp();
                    // A: this lane's two pixels' weights on the block's bins
                    const int kb0 = blk * kUMr;
                    int rlo = kUMr, rhi = -1;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const uint32_t kab = __float_as_uint(q0[i].x);
                        if (kab == kNoDeposit) continue;
                        const int col = lane + 32 * i;
                        const int f = (int)(kab & 0xFFFFu) - kBinBias;
                        const bool narrow = __float_as_uint(q1[i].x) != kNoDeposit;
                        const int g = narrow ? f + 2 : (int)(kab >> 16) - kBinBias;
                        // bins f, f+1 (h0, h1) and g, g+1 (h2, h3); a wide run between them
                        const float hv[4] = {q0[i].z, q0[i].w, q1[i].y, q1[i].z};
                        const int kv[4] = {f, f + 1, g, g + 1};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int r = kv[e] - kb0;
                            if (kv[e] >= 0 && kv[e] < nb && r >= 0 && r < kUMr && hv[e] != 0.f) {
                                *reinterpret_cast<unsigned short *>(Ab + swz(r, col)) = pack1<BF16>(hv[e] * sa);
                                rlo = min(rlo, r); rhi = max(rhi, r);
                            }
                        }
                        if (!narrow && q1[i].w != 0.f) {
                            const unsigned short cv = pack1<BF16>(q1[i].w * sa);
                            const int ks = max(f + 2, max(kb0, 0)), ke = min(g - 1, min(kb0 + kUMr - 1, nb - 1));
                            for (int k = ks; k <= ke; ++k)
                                *reinterpret_cast<unsigned short *>(Ab + swz(k - kb0, col)) = cv;
                            if (ks <= ke) { rlo = min(rlo, ks - kb0); rhi = max(rhi, ke - kb0); }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        rlo = min(rlo, __shfl_xor_sync(0xffffffffu, rlo, o));
                        rhi = max(rhi, __shfl_xor_sync(0xffffffffu, rhi, o));
                    }
                    // B: beam j's 32 weights as four 16-byte chunks
                    unsigned char *Bb = S.b[s];
#pragma unroll
                    for (int cch = 0; cch < 4; ++cch) {
                        const int chunk = 4 * h + cch;
                        *reinterpret_cast<uint4 *>(Bb + j * 128 + (((chunk ^ j) & 7) << 4)) =
                            make_uint4(bw[4 * cch], bw[4 * cch + 1], bw[4 * cch + 2], bw[4 * cch + 3]);
                    }
                    // make the generic-proxy writes visible to the tensor core
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        S.clr_lo[s] = rlo <= rhi ? rlo : 0;
                        S.clr_hi[s] = rlo <= rhi ? rhi : -1;
                        S.blk[s] = blk;
                        um_arrive(su32(&S.full[s]));
                    }
                }
                __syncwarp();  // this tile's pixel-table reads come before the next tile's writes
                int nu = nunits;
                if (lane == 0 && !*(volatile int *)&S.abort) nu = atomicAdd(&S.ctr, 1);
                unit = __shfl_sync(0xffffffffu, nu, 0);
            }
        }
        // ambient: lanes j and j + 16 hold beam j
        amb_acc += __shfl_xor_sync(0xffffffffu, amb_acc, 16);
        if (lane < kUN && amb_acc != 0.f) atomicAdd(amb_s + lane, amb_acc);
        prod_sync();
        if (ptid == 0) {
            S.seq_total = S.seq;
            __threadfence_block();
            *(volatile int *)&S.prod_done = 1;
        }
    }
    // ---- wait for every MMA, read the histograms back, finish --------------
    const bool ok_done = um_wait(su32(&S.done), (uint32_t)(item & 1));
    if (!ok_done) um_fail(S, 3, item);
    const bool ok = __syncthreads_and(ok_done && !*(volatile int *)&S.abort) != 0;
    if (!ok) {
        if (tid == 0 && A.err) atomicCAS(A.err, 0, S.where ? S.where : 1);
        return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t touched = (uint32_t)S.touched;
    const float unscale = 1.f / (S.scale_a * S.scale_b);
    const int G = UL.G;
    for (int r0 = 0; r0 < gcount; r0 += G) {
        for (int i = tid; i < G * Ly.HB; i += blockDim.x) hbuf[i] = 0.f;
        __syncthreads();
        if (warp < 8) {
            // warp w reads TMEM lanes 32 (w % 4) .. +31 of blocks w / 4, w / 4 + 2, ...
            const int quarter = warp & 3;
            for (int blk = warp >> 2; blk < nblk; blk += 2) {
                if (!((touched >> blk) & 1u)) continue;
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(blk * kUN);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int k = blk * kUMr + 32 * quarter + lane;
                if (k < nb) {
#pragma unroll
                    for (int jj = 0; jj < kUN; ++jj)
                        if (jj >= r0 && jj < r0 + G)
                            hbuf[(jj - r0) * Ly.HB + skew_pos(k + Ly.pad)] = __uint_as_float(v[jj]) * unscale;
                }
            }
        }
        __syncthreads();
        footprint_finish(A, Ly, hbuf, taps, amb_s + r0, supp + 2 * r0, tsupp + 2 * r0, nrm2_s + r0, tmass_s + r0,
                         bp + r0, b0 + r0, min(G, gcount - r0), G, r0, kUN);
        __syncthreads();
    }
}

// Prepares a CTA for footprint_umma_group: barriers, cleared operand buffers,
// the power-of-two scales and the tensor-memory allocation (warp 0).
template <bool BF16>
__device__ uint32_t umma_cta_begin(const FootprintArgs &A, umd::UmSmem &S, uint32_t ncols)
{
    using namespace umd;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kUS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.empty[s])));
            S.clr_lo[s] = 0;
            S.clr_hi[s] = -1;
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
        S.where = 0;
        S.seq = 0;
        S.issued = 0;
        float sa = 1.f, sb = 1.f;
        if (!BF16) {
            // FP16: the largest operand of each side near 2^14
            int e;
            const float wmax = A.umma_wmax ? __uint_as_float(*A.umma_wmax) : 0.f;
            if (wmax > 0.f) { frexpf(wmax, &e); sa = ldexpf(1.f, 14 - e); }
            if (A.umma_pmax > 0.f) { frexpf(A.umma_pmax, &e); sb = ldexpf(1.f, 14 - e); }
        }
        S.scale_a = sa;
        S.scale_b = sb;
    }
    // operand buffers start cleared (each use clears only what the last one wrote)
    for (int i = tid; i < (int)(kUS * kUA / 16); i += blockDim.x)
        reinterpret_cast<uint4 *>(S.a)[i] = make_uint4(0u, 0u, 0u, 0u);
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return S.tmem;
}

__device__ __forceinline__ void umma_cta_end(uint32_t tmem, uint32_t ncols)
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
    }
}

__host__ __device__ inline uint32_t umma_cols(int n_bins)
{
    const int need = ((n_bins + umd::kUMr - 1) / umd::kUMr) * umd::kUN;
    uint32_t c = 32;
    while ((int)c < need) c <<= 1;
    return c;
}

template <int KIND, bool BF16>
__global__ void __launch_bounds__(umd::kUThreads, 1) footprint_umma_kernel(FootprintArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = umd::su32(smem_raw);
    umd::UmSmem &S = *reinterpret_cast<umd::UmSmem *>(smem_raw + ((1024u - (raw & 1023u)) & 1023u));
    const umd::UmLayout UL = umd::um_layout(A.n_bins, A.M);
    const uint32_t ncols = umma_cols(A.n_bins);
    const uint32_t tmem = umma_cta_begin<BF16>(A, S, ncols);
    footprint_umma_group<KIND, BF16>(A, blockIdx.x, smem_raw, S, UL, tmem, 0);
    umma_cta_end(tmem, ncols);
}

// Batched form: a persistent grid of one CTA per SM taking (frame, group)
// items from a counter (as footprint_batch_kernel), with one tensor-memory
// allocation and one barrier ring for all its items.
template <int KIND, bool BF16>
__global__ void __launch_bounds__(umd::kUThreads, 1)
    footprint_umma_batch_kernel(FootprintArgs base, const FrameDesc *frames, const int2 *items, int n_items,
                                int *counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const uint32_t raw = umd::su32(smem_raw);
    umd::UmSmem &S = *reinterpret_cast<umd::UmSmem *>(smem_raw + ((1024u - (raw & 1023u)) & 1023u));
    const umd::UmLayout UL = umd::um_layout(base.n_bins, base.M);
    const uint32_t ncols = umma_cols(base.n_bins);
    // the per-frame scale of A is set per item below; the CTA-level set-up
    // computes the profile's
    const uint32_t tmem = umma_cta_begin<BF16>(base, S, ncols);
    for (int done = 0;; ++done) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (it >= n_items || S.abort) break;
        const int2 fg = items[it];
        const FrameDesc F = frames[fg.x];
        FootprintArgs A = base;
        A.U = F.U; A.V = F.V; A.panorama = F.panorama;
        A.az0 = F.az0; A.el0 = F.el0; A.daz = F.daz; A.del = F.del;
        A.rec = F.rec; A.beams = F.beams; A.n_beams = F.n_beams;
        A.wave = F.wave; A.echoes = F.echoes; A.counts = F.counts;
        if (threadIdx.x == 0 && !BF16) {
            int e;
            const float wmax = F.wmax ? __uint_as_float(*F.wmax) : 0.f;
            S.scale_a = 1.f;
            if (wmax > 0.f) { frexpf(wmax, &e); S.scale_a = ldexpf(1.f, 14 - e); }
        }
        __syncthreads();
        footprint_umma_group<KIND, BF16>(A, fg.y, smem_raw, S, UL, tmem, done);
        __syncthreads();  // shared memory is reused by the next item
    }
    umma_cta_end(tmem, ncols);
}

static_assert(umd::kUN == kUmmaBeams, "tcgen05 deposit group size");
static_assert(umd::kUMr * 32 == kUmmaMaxBins, "32 blocks of 128 bins fill 512 TMEM columns at 16 beams");
