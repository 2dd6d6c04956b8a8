// Beamformer output (Sec. II-B, applied per pair to the windowed test
// vectors): out[g][v'] = c_g^H z_test[g][v'] = sum_w conj(c_g[w]) z[v'][w].
//
// One thread per output.  The windows of a warp's 32 consecutive outputs
// are one contiguous span of the test-window array (pair-major, then
// vector, then beam), so the warp first copies that span to shared memory
// with coalesced loads and each thread then reads its W_g entries there
// (per-thread loads of 8 W contiguous bytes would touch 32 sectors per
// instruction).  Memory bound (8 W + 8 bytes per output).
#include "common.cuh"
#include "internal.h"

namespace bs {

// WM: the largest window (16, or 32 with half as many warps per CTA), so a
// warp's span of 32 outputs x W_g entries fits its shared-memory buffer.
template <int WM>
struct ApplyCfg {
    static constexpr int threads = WM <= 16 ? 256 : 128;
    static constexpr int span = 32 * WM;   // float2 per warp
};

template <int WM>
__global__ void __launch_bounds__(ApplyCfg<WM>::threads)
    apply_kernel(const float2 *__restrict__ z, const int64_t *__restrict__ zte_off,
                 const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                 const float2 *__restrict__ c, float2 *__restrict__ out, int64_t total, int Vte) {
    __shared__ float2 span[ApplyCfg<WM>::threads / 32][ApplyCfg<WM>::span];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t idx0 = (int64_t)blockIdx.x * blockDim.x + warp * 32;
    if (idx0 >= total) return;   // uniform per warp
    const int64_t idx = idx0 + lane;
    const bool valid = idx < total;
    const int64_t gi = valid ? idx : total - 1;   // invalid lanes repeat the last output's window
    const int64_t g = gi / Vte;
    const int v = (int)(gi - g * Vte);
    const int W = __ldg(&Wg[g]);
    const int64_t start = __ldg(&zte_off[g]) + (int64_t)v * W;
    const int64_t s0 = __shfl_sync(0xFFFFFFFFu, start, 0);
    const int64_t e31 = __shfl_sync(0xFFFFFFFFu, start + W, 31);
    const int n = (int)(e31 - s0);   // <= 32 * WM
    float2 *buf = span[warp];
    for (int e = lane; e < n; e += 32) buf[e] = __ldcs(&z[s0 + e]);
    __syncwarp();
    const float2 *zv = buf + (start - s0);
    const float2 *cg = c + __ldg(&woff[g]);
    float re = 0.f, im = 0.f;
    for (int w = 0; w < W; ++w) {
        const float2 a = zv[w];
        const float2 b = __ldg(&cg[w]);
        // conj(b) * a
        re = fmaf(b.x, a.x, fmaf(b.y, a.y, re));
        im = fmaf(b.x, a.y, fmaf(-b.y, a.x, im));
    }
    if (valid) out[idx] = make_float2(re, im);
}

bs_status launch_apply(const bs_plan *p, const float2 *zte, const float2 *c, float2 *out, cudaStream_t st) {
    const int64_t total = p->pairs * p->Vte;
    if (total == 0) return BS_OK;
    if (p->Wmax > 32) return set_error(BS_EUNSUPPORTED, "W > 32");
    if (p->Wmax <= 16) {
        constexpr int thr = ApplyCfg<16>::threads;
        apply_kernel<16><<<(unsigned)((total + thr - 1) / thr), thr, 0, st>>>(zte, p->d_zte_off, p->d_Wg, p->d_woff, c,
                                                                             out, total, p->Vte);
    } else {
        constexpr int thr = ApplyCfg<32>::threads;
        apply_kernel<32><<<(unsigned)((total + thr - 1) / thr), thr, 0, st>>>(zte, p->d_zte_off, p->d_Wg, p->d_woff, c,
                                                                             out, total, p->Vte);
    }
    return check_launch("apply launch");
}

}  // namespace bs
