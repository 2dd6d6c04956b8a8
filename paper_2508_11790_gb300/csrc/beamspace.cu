// Beamspace transform and window gather (Eq. VerDFT, Eq. BeamTransform,
// Eq. OverallWindow, Eq. ApplyWindow).
//
// Every (record, bin) vector of N elements (contiguous in the channelised
// cube) is zero-padded to M points and transformed by an M-point Stockham
// FFT in shared memory; a CTA takes VPB consecutive vectors.  The windowed
// variant then writes, for every target, the W_t beams of its window
// (start_g + w mod M) straight from shared memory into the packed training
// or test window arrays; the full variant writes all M beams.
#include "beamspace_dev.cuh"
#include "internal.h"

namespace bs {

// kFull: write all M beams to out[v][m]; else gather windows (PREC = storage
// precision of the training windows).
template <int M, bool kFull, int PREC>
__global__ void __launch_bounds__(BsCfg<M>::nthr, BsCfg<M>::minb)
    beamspace_kernel(const float2 *__restrict__ y, int64_t nvec, int N, const float2 *__restrict__ tw,
                     float scale, float2 *__restrict__ out, GatherArgs ga) {
    using RP = Radix<M>;
    constexpr int vpb = BsCfg<M>::vpb;
    constexpr int nthr = BsCfg<M>::nthr;
    constexpr int pl = BsCfg<M>::pl;
    extern __shared__ float2 sm[];
    // per-target gather entries of this CTA (uniform path), filled before the
    // FFT so that the table loads overlap the butterflies
    __shared__ long long tab_base[kTabT];
    __shared__ int tab_sw[kTabT];     // start | (W << 16)
    __shared__ int tab_n[kTabT];      // outputs of this target in this CTA (0: none)
    const int tid = threadIdx.x;
    const int64_t vid0 = (int64_t)blockIdx.x * vpb;
    int s_cta = 0, v0_cta = 0;
    bool train_cta = false;
    if constexpr (!kFull) {
        if (ga.uniform && vid0 < ga.nvec) {
            const int p = (int)((ga.vbase + vid0) >> ga.log2F);
            const int q = (int)((ga.vbase + vid0) & ((1 << ga.log2F) - 1));
            s_cta = q >> ga.log2B;
            const int i0 = q & ((1 << ga.log2B) - 1);
            train_cta = p < ga.P_train;
            v0_cta = train_cta ? (p << ga.log2B) + i0 : ((p - ga.P_train) << ga.log2B) + i0;
            const int nv = (ga.nvec - vid0 < (int64_t)vpb) ? (int)(ga.nvec - vid0) : vpb;
            for (int t = tid; t < ga.T && t < kTabT; t += nthr)
                fill_target_entry(ga, t, s_cta, v0_cta, nv, train_cta, tab_base, tab_sw, tab_n);
        }
    }

    auto gload = [&](int c, int n) -> float2 {
        const int64_t v = vid0 + c;
        if (n >= N || v >= nvec) return make_float2(0.f, 0.f);
        return __ldcs(&y[v * N + n]);
    };
    auto sload = [&](int c, int m) -> float2 { return sm[c * pl + padrow(m)]; };
    auto sstore = [&](int c, int m, float2 v) { sm[c * pl + padrow(m)] = v; };

    if constexpr (RP::npass == 1) {
        stockham_pass<M, RP::r0, 1, vpb, nthr, false, false>(tid, tw, gload, sstore);
    } else if constexpr (RP::npass == 2) {
        stockham_pass<M, RP::r0, 1, vpb, nthr, false, false>(tid, tw, gload, sstore);
        __syncthreads();
        stockham_pass<M, RP::r1, RP::r0, vpb, nthr, false, true>(tid, tw, sload, sstore);
    } else {
        stockham_pass<M, RP::r0, 1, vpb, nthr, false, false>(tid, tw, gload, sstore);
        __syncthreads();
        stockham_pass<M, RP::r1, RP::r0, vpb, nthr, false, true>(tid, tw, sload, sstore);
        __syncthreads();
        stockham_pass<M, RP::r2, RP::r0 * RP::r1, vpb, nthr, false, true>(tid, tw, sload, sstore);
    }
    __syncthreads();

    if constexpr (kFull) {
        for (int e = tid; e < vpb * M; e += nthr) {
            const int c = e / M, m = e % M;
            const int64_t v = vid0 + c;
            if (v < nvec) out[v * M + m] = cscale(sload(c, m), scale);
        }
    } else if (ga.uniform) {
        // All vpb vectors share record p and subband s (bins i0 .. i0+vpb-1).
        // Flat loop over the (target, vector c, beam w) entries of the gather
        // table; the vpb * W_t outputs of target t form one contiguous run of
        // the window array (element k = c * W_t + w from the target's base).
        if (vid0 >= ga.nvec) return;
        const int nv = (ga.nvec - vid0 < (int64_t)vpb) ? (int)(ga.nvec - vid0) : vpb;
        for (int e = tid; e < ga.ngather; e += nthr) {
            const int packed = __ldg(&ga.gather[e]);
            const int t = packed >> 10, c = (packed >> 5) & 31, w = packed & 31;
            long long base;
            int sw, nout;
            if (t < kTabT) {
                base = tab_base[t];
                sw = tab_sw[t];
                nout = tab_n[t];
            } else {
                fill_target_entry(ga, t, s_cta, v0_cta, nv, train_cta, &base, &sw, &nout, 0);
            }
            const int W = sw >> 16;
            const int k = c * W + w;
            if (k >= nout) continue;
            const float2 val = cscale(sload(c, ((sw & 0xFFFF) + w) & (M - 1)), scale);
            if (train_cta) store_train<PREC>(ga.ztr, base + k, val, ga.store_scale);
            else ga.zte[base + k] = val;
        }
    } else {
        const int Fm1 = (1 << ga.log2F) - 1, Bm1 = (1 << ga.log2B) - 1;
        for (int e = tid; e < ga.ngather; e += nthr) {
            const int packed = __ldg(&ga.gather[e]);
            const int t = packed >> 10, c = (packed >> 5) & 31, w = packed & 31;
            const int64_t g0 = (int64_t)t * ga.L;
            const int W = __ldg(&ga.Wg[g0]);
            const int64_t vid = vid0 + c;
            if (vid >= nvec) continue;
            const int p = (int)((ga.vbase + vid) >> ga.log2F);
            const int q = (int)((ga.vbase + vid) & Fm1);
            const int s = q >> ga.log2B, i = q & Bm1;
            const int64_t g = g0 + s;
            const int m = (__ldg(&ga.start[g]) + w) & (M - 1);
            const float2 val = cscale(sload(c, m), scale);
            if (p < ga.P_train) {
                const int vv = (p << ga.log2B) + i;
                if (vv < __ldg(&ga.Kg[g]))
                    store_train<PREC>(ga.ztr, __ldg(&ga.ztr_off[g]) + (int64_t)vv * W + w, val, ga.store_scale);
            } else {
                const int vv = ((p - ga.P_train) << ga.log2B) + i;
                ga.zte[__ldg(&ga.zte_off[g]) + (int64_t)vv * W + w] = val;
            }
        }
    }
}

template <int M, bool kFull, int PREC>
static bs_status launch_bs_t(const float2 *y, int64_t nvec, int N, const float2 *tw, float2 *out,
                             const GatherArgs &ga, cudaStream_t st) {
    using C = BsCfg<M>;
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            return cuda_error(cudaFuncSetAttribute(beamspace_kernel<M, kFull, PREC>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem),
                              "beamspace attribute");
        }))
        return s;
    const int64_t blocks = (nvec + C::vpb - 1) / C::vpb;
    if (blocks > 0x7FFFFFFF) return set_error(BS_EUNSUPPORTED, "too many vectors");
    if (blocks == 0) return BS_OK;
    beamspace_kernel<M, kFull, PREC><<<(unsigned)blocks, C::nthr, C::smem, st>>>(
        y, nvec, N, tw, 1.0f / sqrtf((float)M), out, ga);
    return check_launch("beamspace launch");
}

template <bool kFull, int PREC>
static bs_status launch_bs(int M, const float2 *y, int64_t nvec, int N, const float2 *tw, float2 *out,
                           const GatherArgs &ga, cudaStream_t st) {
    switch (M) {
        case 16: return launch_bs_t<16, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 32: return launch_bs_t<32, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 64: return launch_bs_t<64, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 128: return launch_bs_t<128, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 256: return launch_bs_t<256, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 512: return launch_bs_t<512, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 1024: return launch_bs_t<1024, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 2048: return launch_bs_t<2048, kFull, PREC>(y, nvec, N, tw, out, ga, st);
        case 4096: return launch_bs_t<4096, kFull, PREC>(y, nvec, N, tw, out, ga, st);
    }
    return set_error(BS_EUNSUPPORTED, "M not supported");
}

static int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

bs_status launch_beamspace(const bs_plan *p, const float2 *xc, void *ztr, float2 *zte, cudaStream_t st, int p0,
                           int np) {
    if (np < 0) np = p->P - p0;
    GatherArgs ga;
    ga.nvec = (int64_t)np * p->Fs;   // Fs = Ls B bins per record (F without a shard)
    ga.vbase = (int64_t)p0 * p->Fs;
    xc += ga.vbase * p->cfg.N;   // the kernels index vectors of this range
    ga.log2F = ilog2(p->Fs);
    ga.log2B = ilog2(p->B);
    ga.L = p->Ls;
    ga.T = p->cfg.T;
    ga.P_train = p->cfg.P_train;
    ga.uniform = (p->B % p->vpb) == 0;
    ga.gather = p->d_gather;
    ga.gsub = reinterpret_cast<const longlong2 *>(p->d_gsub);
    ga.ngather = (int)p->gather.size();
    ga.Wg = p->d_Wg;
    ga.Kg = p->d_Kg;
    ga.start = p->d_start;
    ga.ztr_off = p->d_ztr_off;
    ga.zte_off = p->d_zte_off;
    ga.ztr = ztr;
    ga.zte = zte;
    ga.store_scale = p->cfg.store_scale;
    if (p->planar) return launch_beamspace2d(p, xc, ga, st);
    bool used = false;
    bs_status s = BS_OK;
    // -1: the first variant that applies, in the order tensor cores, warp per
    // transform, bulk-copy-staged, one-shot; 0..3 start the search there
    const int v = p->tune_beamspace;
    if (v < 0 || v == 3) {
        s = launch_beamspace_tc(p, xc, ga, st, &used);
        if (s || used) return s;
    }
    if (v <= 0 || v == 3) {
        s = launch_beamspace_warp(p, xc, ga, st, &used);
        if (s || used) return s;
    }
    if (v <= 1 || v == 3) {
        s = launch_beamspace_tma(p, xc, ga, st, &used);
        if (s || used) return s;
    }
    switch (p->cfg.precision) {
        case BS_PREC_FP32: return launch_bs<false, BS_PREC_FP32>(p->cfg.M, xc, ga.nvec, p->cfg.N, p->d_twM, nullptr, ga, st);
        case BS_PREC_FP16: return launch_bs<false, BS_PREC_FP16>(p->cfg.M, xc, ga.nvec, p->cfg.N, p->d_twM, nullptr, ga, st);
        default: return launch_bs<false, BS_PREC_BF16>(p->cfg.M, xc, ga.nvec, p->cfg.N, p->d_twM, nullptr, ga, st);
    }
}

bs_status launch_beamspace_full(const bs_plan *p, const float2 *y, int64_t nvec, float2 *yb,
                                cudaStream_t st) {
    GatherArgs ga{};
    return launch_bs<true, BS_PREC_FP32>(p->cfg.M, y, nvec, p->cfg.N, p->d_twM, yb, ga, st);
}

bs_status launch_fft_rows(const bs_plan *p, const float2 *y, int64_t nvec, float2 *yb, cudaStream_t st) {
    GatherArgs ga{};
    return launch_bs<true, BS_PREC_FP32>(p->cfg.F, y, nvec, p->cfg.F, p->d_twF, yb, ga, st);
}

}  // namespace bs
