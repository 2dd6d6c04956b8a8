// Channeliser (Sec. III-A): F-point FFT over fast time of every element of
// every record, written subband-major so that the beamspace stage reads
// each (record, bin) vector of N elements contiguously.
//
// x, xc: [P][F][N] cf32.  xc[p][q][n] with q = s*B + i holds FFT bin
// k = (q - F/2) mod F, i.e. the FFT output in signed-frequency order; this
// is produced by multiplying the input by (-1)^t (shift theorem), so no
// extra permutation pass is needed.
//
// A subband shard writes only bins q0 .. q0 + Fs - 1 of each record, to rows
// q - q0 of a cube of Fs rows per record (Fs = F without a shard).
//
// One CTA transforms NT consecutive elements (columns) of one record: the
// first Stockham pass reads the columns straight from HBM (NT*8-byte
// segments of each row), the middle passes run in padded shared memory and
// the last pass writes straight to HBM.
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

#include <algorithm>

namespace bs {

// Columns per CTA: NT = 8192 / F clamped to [4, 32], so that one tile holds
// 8192 points (69.6 KB of padded shared memory) and two CTAs fit on an SM:
// one CTA's loads overlap the other's butterflies.  With 512 threads every
// radix-16 pass is one butterfly per thread (<= 64 registers).
template <int F>
struct ChCfg {
    static constexpr int NT = (8192 / F > 32) ? 32 : ((8192 / F < 4) ? 4 : 8192 / F);
    static constexpr int nthr = (NT * F / 16 < 512) ? NT * F / 16 : 512;
    static constexpr size_t smem = (size_t)padded_len(F) * NT * sizeof(float2);
    static constexpr int minb = (smem <= 100 * 1024) ? 2 : 1;
};

template <int F>
__global__ void __launch_bounds__(ChCfg<F>::nthr, ChCfg<F>::minb)
    channelize_kernel(const float2 *__restrict__ x, float2 *__restrict__ xc, int N,
                      const float2 *__restrict__ tw, float scale, int q0, int Fs) {
    using RP = Radix<F>;
    constexpr int NT = ChCfg<F>::NT;
    constexpr int nthr = ChCfg<F>::nthr;
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x;
    const int n0 = blockIdx.x * NT;
    const float2 *xin = x + (size_t)blockIdx.y * F * N;
    float2 *xout = xc + (size_t)blockIdx.y * Fs * N;

    auto gload = [&](int c, int t) -> float2 {
        const int n = n0 + c;
        if (n >= N) return make_float2(0.f, 0.f);
        const float2 v = __ldcs(&xin[(size_t)t * N + n]);
        return (t & 1) ? make_float2(-v.x, -v.y) : v;   // (-1)^t: signed-frequency order
    };
    auto sload = [&](int c, int t) -> float2 { return sm[padrow(t) * NT + c]; };
    auto sstore = [&](int c, int t, float2 v) { sm[padrow(t) * NT + c] = v; };
    auto gstore = [&](int c, int q, float2 v) {
        const int n = n0 + c;
        if (n < N && q >= q0 && q < q0 + Fs) xout[(size_t)(q - q0) * N + n] = cscale(v, scale);
    };

    if constexpr (RP::npass == 1) {
        stockham_pass<F, RP::r0, 1, NT, nthr, true, false>(tid, tw, gload, gstore);
    } else if constexpr (RP::npass == 2) {
        stockham_pass<F, RP::r0, 1, NT, nthr, true, false>(tid, tw, gload, sstore);
        __syncthreads();
        stockham_pass<F, RP::r1, RP::r0, NT, nthr, true, false>(tid, tw, sload, gstore);
    } else {
        stockham_pass<F, RP::r0, 1, NT, nthr, true, false>(tid, tw, gload, sstore);
        __syncthreads();
        stockham_pass<F, RP::r1, RP::r0, NT, nthr, true, true>(tid, tw, sload, sstore);
        __syncthreads();
        stockham_pass<F, RP::r2, RP::r0 * RP::r1, NT, nthr, true, false>(tid, tw, sload, gstore);
    }
}

// Persistent TMA variant: one CTA per SM loops over (record, column tile)
// tiles.  The raw tile (F rows x NT columns) arrives in a dense staging
// buffer by TMA; pass 0 reads it into the padded work buffer, after which
// the staging buffer is free and the next tile's TMA is issued, so the HBM
// reads of tile i+1 overlap passes 1-2 (and the HBM writes) of tile i.  The
// last pass writes a dense output tile in shared memory, which leaves by
// TMA tensor stores (NT x 8-byte rows, clipped at N): scattered 8-byte
// stores from every thread had filled the global store queue.
template <int F>
struct ChTmaCfg {
    static constexpr int NT = ChCfg<F>::NT;
    static constexpr int nthr = ChCfg<F>::nthr;
    static constexpr int box_rows = F < 256 ? F : 256;
    static constexpr size_t stage_bytes = (size_t)F * NT * sizeof(float2);
    static constexpr size_t work_bytes = (size_t)padded_len(F) * NT * sizeof(float2);
    static constexpr size_t smem = 2 * stage_bytes + work_bytes + 16;   // staging, work, output tile
};

template <int F>
__global__ void __launch_bounds__(ChTmaCfg<F>::nthr, 1)
    channelize_tma_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap omap, int N,
                          int P, const float2 *__restrict__ tw, float scale, int *__restrict__ err, int q0,
                          int Fs, int obox) {
    using RP = Radix<F>;
    using C = ChTmaCfg<F>;
    constexpr int NT = C::NT;
    constexpr int nthr = C::nthr;
    extern __shared__ __align__(128) unsigned char smraw[];
    float2 *stg = reinterpret_cast<float2 *>(smraw);
    float2 *sm = reinterpret_cast<float2 *>(smraw + C::stage_bytes);
    float2 *ob = reinterpret_cast<float2 *>(smraw + C::stage_bytes + C::work_bytes);   // dense output tile
    uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + 2 * C::stage_bytes + C::work_bytes);
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    const int ntn = (N + NT - 1) / NT;
    const long long ntiles = (long long)P * ntn;
    long long tile = blockIdx.x;
    if (tile >= ntiles) return;

    auto issue = [&](long long tl) {   // thread 0 only
        const int p = (int)(tl / ntn), n0 = (int)(tl % ntn) * NT;
        mbar_arrive_expect_tx(bar, (unsigned)C::stage_bytes);
#pragma unroll 1
        for (int r0 = 0; r0 < F; r0 += C::box_rows)
            tma_load_2d(stg + (size_t)r0 * NT, &tmap, bar, 2 * n0, p * F + r0);
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_proxy_async();
        issue(tile);
    }
    __syncthreads();

    unsigned phase = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const int p = (int)(tile / ntn), n0 = (int)(tile % ntn) * NT;
        if (tid == 0) ok_s = mbar_wait_bounded(bar, phase) ? 1 : 0;
        __syncthreads();
        if (!ok_s) {   // uniform: record the failure, wait (bounded) for the copy, leave
            if (tid == 0) {
                atomicOr(err, 1);
                mbar_wait_bounded(bar, phase);
                bulk_wait0();
            }
            return;
        }
        mbar_try_wait(bar, phase);   // completed phase: each thread acquires the TMA writes
        phase ^= 1u;
        auto gload = [&](int c, int t) -> float2 {
            const float2 v = stg[t * NT + c];
            return (t & 1) ? make_float2(-v.x, -v.y) : v;   // (-1)^t: signed-frequency order
        };
        auto sload = [&](int c, int t) -> float2 { return sm[padrow(t) * NT + c]; };
        auto sstore = [&](int c, int t, float2 v) { sm[padrow(t) * NT + c] = v; };
        auto ostore = [&](int c, int q, float2 v) { ob[q * NT + c] = cscale(v, scale); };
        static_assert(RP::npass == 3, "TMA channeliser needs F >= 512");
        stockham_pass<F, RP::r0, 1, NT, nthr, true, false>(tid, tw, gload, sstore);
        __syncthreads();   // staging consumed
        if (tid == 0 && tile + gridDim.x < ntiles) {
            fence_proxy_async();
            issue(tile + gridDim.x);
        }
        stockham_pass<F, RP::r1, RP::r0, NT, nthr, true, true>(tid, tw, sload, sstore);
        if (tid == 0) bulk_wait_read0();   // the previous tile's output has left the output buffer
        __syncthreads();
        stockham_pass<F, RP::r2, RP::r0 * RP::r1, NT, nthr, true, false>(tid, tw, sload, ostore);
        __syncthreads();   // output tile complete; work buffer consumed before the next tile's pass 0
        if (tid == 0) {    // the shard's rows of the output tile to xc by TMA (columns beyond N clipped)
            fence_proxy_async();
#pragma unroll 1
            for (int r0 = 0; r0 < Fs; r0 += obox)
                tma_store_2d(&omap, ob + (size_t)(q0 + r0) * NT, 2 * n0, p * Fs + r0);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

template <int F>
static bs_status launch_ch_tma(const bs_plan *pl, const float2 *x, int P, int N, float2 *xc, cudaStream_t st,
                               bool *used) {
    using C = ChTmaCfg<F>;
    *used = false;
    if ((N & 1) || (reinterpret_cast<uintptr_t>(x) & 15) || C::smem > 220 * 1024) return BS_OK;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return BS_OK;
    if (reinterpret_cast<uintptr_t>(xc) & 15) return BS_OK;
    CUtensorMap tmap, omap;
    const int Fs = pl->Fs, q0 = pl->s0 * pl->B;
    const int obox = Fs < C::box_rows ? Fs : C::box_rows;   // q0 and Fs are multiples of obox
    const cuuint64_t gdim[2] = {(cuuint64_t)2 * N, (cuuint64_t)P * F};
    const cuuint64_t odim[2] = {(cuuint64_t)2 * N, (cuuint64_t)P * Fs};
    const cuuint64_t gstride[1] = {(cuuint64_t)N * sizeof(float2)};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * C::NT), (cuuint32_t)C::box_rows};
    const cuuint32_t obx[2] = {(cuuint32_t)(2 * C::NT), (cuuint32_t)obox};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(x), gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, xc, odim, gstride, obx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return BS_OK;   // fall back to the non-TMA kernel
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            return cuda_error(cudaFuncSetAttribute(channelize_tma_kernel<F>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem),
                              "channelize attribute");
        }))
        return s;
    const long long tiles = (long long)P * ((N + C::NT - 1) / C::NT);
    const int grid = (int)std::min<long long>(tiles, pl->num_sms);
    channelize_tma_kernel<F><<<grid, C::nthr, C::smem, st>>>(tmap, omap, N, P, pl->d_twF, 1.0f / sqrtf((float)F),
                                                            pl->d_err, q0, Fs, obox);
    *used = true;
    return check_launch("channelize (TMA) launch");
}

template <int F>
static bs_status launch_ch(const float2 *x, int P, int N, float2 *xc, const float2 *tw, int q0, int Fs,
                           cudaStream_t st) {
    using C = ChCfg<F>;
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            return cuda_error(cudaFuncSetAttribute(channelize_kernel<F>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem),
                              "channelize attribute");
        }))
        return s;
    dim3 grid((N + C::NT - 1) / C::NT, P);
    channelize_kernel<F><<<grid, C::nthr, C::smem, st>>>(x, xc, N, tw, 1.0f / sqrtf((float)F), q0, Fs);
    return check_launch("channelize launch");
}

bs_status launch_channelize(const bs_plan *p, const float2 *x, int P, float2 *xc, cudaStream_t st) {
    const int N = p->cfg.N;
    const int q0 = p->s0 * p->B, Fs = p->Fs;
    if (!(p->cfg.flags & BS_FLAG_NO_TMA)) {
        bool used = false;
        bs_status s = BS_OK;
        switch (p->cfg.F) {
            case 512: s = launch_ch_tma<512>(p, x, P, N, xc, st, &used); break;
            case 1024: s = launch_ch_tma<1024>(p, x, P, N, xc, st, &used); break;
            case 2048: s = launch_ch_tma<2048>(p, x, P, N, xc, st, &used); break;
            default: break;
        }
        if (s || used) return s;
    }
    switch (p->cfg.F) {
        case 16: return launch_ch<16>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 32: return launch_ch<32>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 64: return launch_ch<64>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 128: return launch_ch<128>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 256: return launch_ch<256>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 512: return launch_ch<512>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 1024: return launch_ch<1024>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 2048: return launch_ch<2048>(x, P, N, xc, p->d_twF, q0, Fs, st);
        case 4096: return launch_ch<4096>(x, P, N, xc, p->d_twF, q0, Fs, st);
    }
    return set_error(BS_EUNSUPPORTED, "F not supported");
}

}  // namespace bs
