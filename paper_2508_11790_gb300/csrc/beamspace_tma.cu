// Persistent beamspace transform and window gather for M = 512 .. 4096
// (Eq. VerDFT, Eq. BeamTransform, Eq. OverallWindow, Eq. ApplyWindow).
//
// Same result as the one-shot kernel of beamspace.cu (every (record, bin)
// vector zero-padded to M points, M-point DFT scaled by 1/sqrt(M), then the
// W_t beams start_g + w (mod M) of every target written to the packed
// window arrays), organised for throughput:
//
// * one CTA per resident slot loops over groups of vpb consecutive vectors
//   (vpb * M = 4096 points); the group's vpb * N input elements are
//   contiguous in the channelised cube and arrive by one 1-D bulk copy
//   into a double-buffered staging area, issued two groups ahead;
// * the three Stockham passes (radix 16, 16, M/256) keep every thread on
//   the same butterfly index in every group, so the twiddle factors of
//   passes 2 and 3 are read from the table once, into registers;
// * when N <= M/2 the upper half of every radix-16 input of pass 1 is the
//   zero padding, and the first radix-2 stage of that DFT is skipped;
// * pass 1 writes work buffer X1, pass 2 reads X1 and writes X2, and pass 3
//   writes each output to the X2 slot it read it from (Stockham with
//   Ns = 256 and 256 butterflies per vector), so a group takes three CTA
//   barriers; the gather entries of the group are loaded during pass 2 and
//   stored to shared memory after pass 3, off the critical path;
// * each thread keeps its (fixed) share of the gather table in registers,
//   decoded once.
//
// Shared memory per CTA: 2 x vpb x padded(M) x 8 bytes of work buffers plus
// 2 x vpb x N x 8 bytes of staging (102 KB at M = 2048, N = 1024): two CTAs
// per SM.
#include "beamspace_dev.cuh"
#include "internal.h"
#include "tma.cuh"

#include <algorithm>

namespace bs {

constexpr int kGatherRegs = 8;   // gather entries per thread held in registers

template <int M>
struct BsTmaCfg {
    using RP = Radix<M>;
    static_assert(RP::npass == 3, "three-pass sizes only (M = 512 .. 4096)");
    static constexpr int vpb = BsCfg<M>::vpb;
    static constexpr int nthr = 256;
    static constexpr int Q = M / 16;    // butterflies per vector in passes 1 and 2
    static constexpr int R2 = RP::r2;   // radix of pass 3 (M / 256)
    static constexpr int pl = padded_len(M);
    static constexpr size_t work_bytes = (size_t)vpb * pl * sizeof(float2);
    static_assert(vpb * Q == nthr, "one pass-1/2 butterfly per thread");
    static_assert(work_bytes % 16 == 0, "staging area must start 16-byte aligned");
};

// 16-point DFT (natural order in and out) of v[0..7] with v[8..15] = 0: the
// first radix-2 decimation-in-frequency stage reduces to e = v, o = v w^k.
__device__ __forceinline__ void dft16_upper_zero(float2 (&v)[16]) {
    float2 e[8], o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        e[k] = v[k];
        o[k] = twiddle16(k, v[k]);
    }
    RegDFT<8>::run(e);
    RegDFT<8>::run(o);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[2 * k] = e[k];
        v[2 * k + 1] = o[k];
    }
}

template <int M, bool kHalf>
__global__ void __launch_bounds__(256, 2)
    beamspace_tma_kernel(const float2 *__restrict__ y, int N, const float2 *__restrict__ tw, float scale,
                         int prec, GatherArgs ga, int *__restrict__ err) {
    using C = BsTmaCfg<M>;
    constexpr int vpb = C::vpb, Q = C::Q, R2 = C::R2, pl = C::pl;
    constexpr int QP = Q + Q / 16;   // padded distance of rows r Q and (r+1) Q
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *X1 = reinterpret_cast<float2 *>(smraw);                    // pass-1 output
    float2 *X2 = reinterpret_cast<float2 *>(smraw + C::work_bytes);     // passes 2-3, gather
    float2 *stg = reinterpret_cast<float2 *>(smraw + 2 * C::work_bytes);
    const int stage_elems = vpb * N;
    uint64_t *bar = reinterpret_cast<uint64_t *>(stg + 2 * (size_t)stage_elems);
    __shared__ GatherEnt tab[kTabT];
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    const int64_t ngroups = ga.nvec / vpb;   // the caller guarantees nvec % vpb == 0
    const int64_t G = gridDim.x;
    int64_t g = blockIdx.x;
    if (g >= ngroups) return;
    const unsigned stage_bytes = (unsigned)stage_elems * (unsigned)sizeof(float2);

    auto issue = [&](int64_t gg, int s) {   // thread 0 only
        mbar_arrive_expect_tx(&bar[s], stage_bytes);
        bulk_load(stg + (size_t)s * stage_elems, y + gg * vpb * (int64_t)N, stage_bytes, &bar[s]);
    };
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
        issue(g, 0);
        if (g + G < ngroups) issue(g + G, 1);
    }

    // Twiddles of this thread's butterflies: pass 2 (Ns = 16, R = 16) uses
    // w^(r (j mod 16) M/256), pass 3 (Ns = 256, R = R2) w^(r j), j = tid.
    float2 w2[16], w3[R2];
    {
        const int e2 = (tid & 15) * (M / 256);
#pragma unroll
        for (int r = 1; r < 16; ++r) w2[r] = __ldg(&tw[r * e2]);
#pragma unroll
        for (int r = 1; r < R2; ++r) w3[r] = __ldg(&tw[r * tid]);
    }
    const float sc_tr = (prec == BS_PREC_FP32) ? scale : scale * ga.store_scale;
    // Every group uses the same gather table and thread tid always takes
    // entries tid + k * 256: its first kGatherRegs entries stay in registers
    // (re-reading the table for every group would go to L2: the L1 left
    // beside the shared memory of two CTAs does not keep it).  An entry
    // (t, c, w) with t < kTabT is held decoded: t | k << 8 | c << 17 | w << 21
    // with k = c W_t + w its position in the target's run; others keep the
    // table's packing with bit 30 set; -1: no entry.
    int gent[kGatherRegs];
#pragma unroll
    for (int k = 0; k < kGatherRegs; ++k) {
        const int e = tid + k * C::nthr;
        int v = -1;
        if (e < ga.ngather) {
            const int packed = __ldg(&ga.gather[e]);
            const int t = packed >> 10, c = (packed >> 5) & 31, w = packed & 31;
            if (t < kTabT) {
                const int W = __ldg(&ga.Wg[(int64_t)t * ga.L]);
                v = t | ((c * W + w) << 8) | (c << 17) | (w << 21);
            } else {
                v = packed | (1 << 30);
            }
        }
        gent[k] = v;
    }
    if (tid == 0) ok_s = mbar_wait_bounded(&bar[0], 0) ? 1 : 0;
    __syncthreads();

    // Three CTA barriers per group.  Thread 0 waits for the next group's copy
    // before the third barrier, so its status is known to all threads after it.
    for (unsigned it = 0; g < ngroups; g += G, ++it) {
        const int s = (int)(it & 1u);
        if (!ok_s) {   // uniform: record, wait (bounded) for the copies in flight, leave
            if (tid == 0) {
                atomicOr(err, 1);
                mbar_wait_bounded(&bar[s], (it >> 1) & 1u);
                if (g + G < ngroups) mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1u);
            }
            return;
        }
        mbar_try_wait(&bar[s], (it >> 1) & 1u);   // completed phase: each thread acquires the copy
        const int64_t vid0 = ga.vbase + g * vpb;   // in the whole cube
        const int p = (int)(vid0 >> ga.log2F);
        const int q = (int)(vid0 & ((1 << ga.log2F) - 1));
        const int sb = q >> ga.log2B;
        const int i0 = q & ((1 << ga.log2B) - 1);
        const bool train = p < ga.P_train;
        const int v0 = train ? (p << ga.log2B) + i0 : ((p - ga.P_train) << ga.log2B) + i0;

        // pass 1: radix 16, Ns = 1; output t = 16 j + r lands at padrow(t) = 17 j + r
        {
            const int c = tid / Q, j = tid % Q;
            const float2 *src = stg + (size_t)s * stage_elems + c * N;
            float2 v[16];
            if constexpr (kHalf) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int n = j + r * Q;
                    v[r] = (n < N) ? src[n] : make_float2(0.f, 0.f);
                }
                dft16_upper_zero(v);
            } else {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int n = j + r * Q;
                    v[r] = (n < N) ? src[n] : make_float2(0.f, 0.f);
                }
                RegDFT<16>::run(v);
            }
            float2 *dst = X1 + c * pl + 17 * j;
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[r] = v[r];
        }
        __syncthreads();   // (1) staging buffer s consumed, X1 complete
        if (tid == 0 && g + 2 * G < ngroups) {
            fence_proxy_async();
            issue(g + 2 * G, s);
        }
        // this group's gather entries (subband-major table: one contiguous
        // read for consecutive targets); loads issued here, stored after pass 3
        long long e_base = 0;
        int e_sw = 0, e_n = 0;
        const bool filler = tid < ga.T && tid < kTabT;
        if (filler) {
            const longlong2 *gs = ga.gsub + 2 * ((int64_t)sb * ga.T + tid);
            const longlong2 o = __ldg(gs), m = __ldg(gs + 1);
            const int W = (int)(m.x >> 16), K = (int)m.y;
            e_sw = (int)m.x;
            e_n = train ? ((v0 >= K) ? 0 : min(vpb * W, (K - v0) * W)) : vpb * W;
            e_base = (train ? o.x : o.y) + (long long)v0 * W;
        }

        // pass 2: radix 16, Ns = 16, X1 -> X2
        {
            const int c = tid / Q, j = tid % Q;
            const float2 *col = X1 + c * pl + j + (j >> 4);
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = col[r * QP];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w2[r]);
            RegDFT<16>::run(v);
            const int base = (j >> 4) * 256 + (j & 15);
            float2 *dst = X2 + c * pl + base + (base >> 4);   // padrow(base + 16 r) = base + base/16 + 17 r
#pragma unroll
            for (int r = 0; r < 16; ++r) dst[17 * r] = v[r];
        }
        __syncthreads();   // (2) X2 complete

        // pass 3: radix R2, Ns = 256; butterfly j = tid of every vector reads
        // and writes rows j + 256 r (padded: j + j/16 + 272 r) of X2
#pragma unroll
        for (int b = 0; b < vpb; ++b) {
            float2 *col = X2 + b * pl + tid + (tid >> 4);
            float2 v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = col[272 * r];
#pragma unroll
            for (int r = 1; r < R2; ++r) v[r] = cmul(v[r], w3[r]);
            RegDFT<R2>::run(v);
#pragma unroll
            for (int r = 0; r < R2; ++r) col[272 * r] = v[r];
        }
        if (filler) tab[tid] = GatherEnt{e_base, e_sw, e_n};
        if (tid == 0 && g + G < ngroups) ok_s = mbar_wait_bounded(&bar[s ^ 1], ((it + 1) >> 1) & 1u) ? 1 : 0;
        __syncthreads();   // (3) beams and gather entries complete; next copy's status known

        // window gather: the vpb * W_t outputs of target t are one run of the
        // window array (element k = c * W_t + w from the target's base)
        auto put = [&](long long idx, float2 val) {
            if (!train) {
                ga.zte[idx] = cscale(val, scale);
            } else if (prec == BS_PREC_FP16) {
                store_train<BS_PREC_FP16>(ga.ztr, idx, val, sc_tr);
            } else if (prec == BS_PREC_BF16) {
                store_train<BS_PREC_BF16>(ga.ztr, idx, val, sc_tr);
            } else {
                store_train<BS_PREC_FP32>(ga.ztr, idx, cscale(val, sc_tr), 1.f);
            }
        };
        auto gather_packed = [&](int packed) {   // table packing (t << 10) | (c << 5) | w
            const int t = packed >> 10, c = (packed >> 5) & 31, w = packed & 31;
            long long base;
            int sw, nout;
            if (t < kTabT) {
                const GatherEnt te = tab[t];
                base = te.base;
                sw = te.sw;
                nout = te.n;
            } else {
                fill_target_entry(ga, t, sb, v0, vpb, train, &base, &sw, &nout, 0);
            }
            const int k = c * (sw >> 16) + w;
            if (k >= nout) return;
            put(base + k, X2[c * pl + padrow(((sw & 0xFFFF) + w) & (M - 1))]);
        };
#pragma unroll
        for (int k = 0; k < kGatherRegs; ++k) {
            const int v = gent[k];
            if (v < 0) continue;
            if (v & (1 << 30)) {
                gather_packed(v & ~(1 << 30));
                continue;
            }
            const GatherEnt te = tab[v & 255];
            const int kk = (v >> 8) & 511;
            if (kk >= te.n) continue;
            const int c = (v >> 17) & 15, w = (v >> 21) & 31;
            put(te.base + kk, X2[c * pl + padrow(((te.sw & 0xFFFF) + w) & (M - 1))]);
        }
        for (int e = tid + kGatherRegs * C::nthr; e < ga.ngather; e += C::nthr) gather_packed(__ldg(&ga.gather[e]));
    }
}

template <int M, bool kHalf>
static bs_status launch_tma_t(const bs_plan *p, const float2 *y, const GatherArgs &ga, cudaStream_t st) {
    using C = BsTmaCfg<M>;
    const size_t smem_max = 2 * C::work_bytes + 2 * (size_t)C::vpb * M * sizeof(float2) + 16;
    const size_t smem = 2 * C::work_bytes + 2 * (size_t)C::vpb * p->cfg.N * sizeof(float2) + 16;
    static PerDevice occ;
    int blocks_per_sm = 1;
    if (bs_status s = occ.get(
            [&](int *v) {
                cudaError_t e = cudaFuncSetAttribute(beamspace_tma_kernel<M, kHalf>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
                if (e != cudaSuccess) return cuda_error(e, "beamspace (TMA) attribute");
                int nb = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, beamspace_tma_kernel<M, kHalf>, C::nthr,
                                                                  smem_max);
                if (e != cudaSuccess) return cuda_error(e, "beamspace (TMA) occupancy");
                *v = std::max(nb, 1);
                return BS_OK;
            },
            &blocks_per_sm))
        return s;
    const int64_t ngroups = ga.nvec / C::vpb;
    if (ngroups == 0) return BS_OK;
    const int grid = (int)std::min<int64_t>(ngroups, (int64_t)p->num_sms * blocks_per_sm);
    beamspace_tma_kernel<M, kHalf><<<grid, C::nthr, smem, st>>>(y, p->cfg.N, p->d_twM, 1.0f / sqrtf((float)M),
                                                               p->cfg.precision, ga, p->d_err);
    return check_launch("beamspace (TMA) launch");
}

template <int M>
static bs_status launch_tma_m(const bs_plan *p, const float2 *y, const GatherArgs &ga, cudaStream_t st) {
    if (2 * p->cfg.N <= M) return launch_tma_t<M, true>(p, y, ga, st);
    return launch_tma_t<M, false>(p, y, ga, st);
}

bs_status launch_beamspace_tma(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                               bool *used) {
    *used = false;
    const int M = p->cfg.M;
    if ((p->cfg.flags & BS_FLAG_NO_TMA) || !ga.uniform || (p->cfg.N & 1) ||
        (reinterpret_cast<uintptr_t>(xc) & 15) || M < 512 || M > 4096 || ga.nvec % p->vpb)
        return BS_OK;
    *used = true;
    switch (M) {
        case 512: return launch_tma_m<512>(p, xc, ga, st);
        case 1024: return launch_tma_m<1024>(p, xc, ga, st);
        case 2048: return launch_tma_m<2048>(p, xc, ga, st);
        default: return launch_tma_m<4096>(p, xc, ga, st);
    }
}

}  // namespace bs
