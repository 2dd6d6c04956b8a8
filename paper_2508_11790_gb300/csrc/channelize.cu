// Channeliser (Sec. III-A): F-point FFT over fast time of every element of
// every record, written subband-major so that the beamspace stage reads
// each (record, bin) vector of N elements contiguously.
//
// x, xc: [P][F][N] cf32.  xc[p][q][n] with q = s*B + i holds FFT bin
// k = (q - F/2) mod F, i.e. the FFT output in signed-frequency order; this
// is produced by multiplying the input by (-1)^t (shift theorem), so no
// extra permutation pass is needed.
//
// One CTA transforms NT consecutive elements (columns) of one record: the
// first Stockham pass reads the columns straight from HBM (NT*8-byte
// segments of each row), the middle passes run in padded shared memory and
// the last pass writes straight to HBM.
#include "common.cuh"
#include "internal.h"

namespace bs {

template <int F>
struct ChCfg {
    // columns per CTA: 8 (64-byte row segments) up to F = 2048, 4 at F = 4096
    // (shared memory), more for short FFTs
    static constexpr int NT = (F >= 4096) ? 4 : (4096 / F > 32) ? 32 : ((4096 / F < 8) ? 8 : 4096 / F);
    static constexpr int nthr = (NT * F / 16 < 512) ? NT * F / 16 : 512;
    static constexpr size_t smem = (size_t)padded_len(F) * NT * sizeof(float2);
};

template <int F>
__global__ void __launch_bounds__(ChCfg<F>::nthr)
    channelize_kernel(const float2 *__restrict__ x, float2 *__restrict__ xc, int N,
                      const float2 *__restrict__ tw, float scale) {
    using RP = Radix<F>;
    constexpr int NT = ChCfg<F>::NT;
    constexpr int nthr = ChCfg<F>::nthr;
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x;
    const int n0 = blockIdx.x * NT;
    const size_t rec = (size_t)blockIdx.y * F * N;
    const float2 *xin = x + rec;
    float2 *xout = xc + rec;

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
        if (n < N) xout[(size_t)q * N + n] = cscale(v, scale);
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

template <int F>
static bs_status launch_ch(const float2 *x, int P, int N, float2 *xc, const float2 *tw,
                           cudaStream_t st) {
    using C = ChCfg<F>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(channelize_kernel<F>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (e != cudaSuccess) return cuda_error(e, "channelize attribute");
        attr_set = true;
    }
    dim3 grid((N + C::NT - 1) / C::NT, P);
    channelize_kernel<F><<<grid, C::nthr, C::smem, st>>>(x, xc, N, tw, 1.0f / sqrtf((float)F));
    return check_launch("channelize launch");
}

bs_status launch_channelize(const bs_plan *p, const float2 *x, int P, float2 *xc, cudaStream_t st) {
    const int N = p->cfg.N;
    switch (p->cfg.F) {
        case 16: return launch_ch<16>(x, P, N, xc, p->d_twF, st);
        case 32: return launch_ch<32>(x, P, N, xc, p->d_twF, st);
        case 64: return launch_ch<64>(x, P, N, xc, p->d_twF, st);
        case 128: return launch_ch<128>(x, P, N, xc, p->d_twF, st);
        case 256: return launch_ch<256>(x, P, N, xc, p->d_twF, st);
        case 512: return launch_ch<512>(x, P, N, xc, p->d_twF, st);
        case 1024: return launch_ch<1024>(x, P, N, xc, p->d_twF, st);
        case 2048: return launch_ch<2048>(x, P, N, xc, p->d_twF, st);
        case 4096: return launch_ch<4096>(x, P, N, xc, p->d_twF, st);
    }
    return set_error(BS_EUNSUPPORTED, "F not supported");
}

}  // namespace bs
