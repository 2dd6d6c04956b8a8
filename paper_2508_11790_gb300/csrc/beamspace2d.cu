// Planar-array beamspace transform and window gather (Eq. ArrayFactor,
// Eq. VerDFT, Eq. HorDFT, Eq. OverallDFT, Eq. BeamTransform, Eq.
// OverallWindow read as S_h (x) S_v, Eq. ApplyWindow).
//
// Elements n = n_x Nz + n_z, beams m = m_x Mz + m_z, window entries
// w = w_x Wz + w_z.  One warp per (record, bin) vector, several per CTA: the
// vector's N = Nx Nz elements are staged in the warp's shared memory; the
// vertical DFT (Mz points of Nz, D_v) runs as direct sums into Mz rows of
// Mx points, zero beyond Nx, and the horizontal one (Mx points, D_h^T) as a
// radix-2 Stockham FFT along every row (log2 Mx passes, two buffers,
// twiddles from an exact per-CTA table), leaving all M = Mx Mz beams with
// row m_z holding m_x in natural order.  The window gather then takes the
// plan's flat (target, entry) list a lane per entry and writes every
// target's Wx x Wz window to the packed window arrays with the conventions
// of the linear-array kernels.  Only warp barriers inside the vector loop.
// Planar plans are limited to N <= 1024 and M <= 2048 (the paper's array
// is 4 x 32).
#include "beamspace_dev.cuh"
#include "internal.h"

#include <algorithm>

namespace bs {

__global__ void __launch_bounds__(128)
    beamspace2d_kernel(const float2 *__restrict__ y, int Nx, int Nz, int Mx, int Mz, float scale, int prec,
                       GatherArgs ga, const int32_t *__restrict__ start_z, const int32_t *__restrict__ Wz,
                       const int32_t *__restrict__ glist, int sumW) {
    extern __shared__ float2 sm2[];
    const int N = Nx * Nz, M = Mx * Mz;
    float2 *twx = sm2;             // [Mx / 2] e^{-2 pi i k / Mx}
    float2 *twz = twx + Mx / 2;    // [Mz]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *ys = twz + Mz + (size_t)warp * (N + 2 * M);   // [N]
    float2 *b0 = ys + N;                                  // [Mz][Mx]
    float2 *b1 = b0 + M;                                  // [Mz][Mx]
    for (int k = tid; k < Mx / 2; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)Mx, &sn, &cs);
        twx[k] = make_float2(cs, sn);
    }
    for (int k = tid; k < Mz; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)Mz, &sn, &cs);
        twz[k] = make_float2(cs, sn);
    }
    __syncthreads();
    const int64_t vid = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (vid >= ga.nvec) return;   // no CTA barrier below
    for (int n = lane; n < N; n += 32) ys[n] = __ldcs(&y[vid * N + n]);
    __syncwarp();
    for (int e = lane; e < M; e += 32) {   // vertical DFT of every column n_x; zero past Nx
        const int mz = e / Mx, nx = e % Mx;
        float2 acc = make_float2(0.f, 0.f);
        if (nx < Nx)
            for (int nz = 0; nz < Nz; ++nz) acc = cadd(acc, cmul(ys[nx * Nz + nz], twz[(mz * nz) & (Mz - 1)]));
        b0[e] = acc;
    }
    __syncwarp();
    // horizontal FFT of every row: radix-2 Stockham passes (sub-transform
    // size Ns = 1, 2, .., Mx/2), ping-pong between b0 and b1
    float2 *src = b0, *dst = b1;
    const int half = Mx >> 1;
    for (int Ns = 1; Ns < Mx; Ns <<= 1) {
        for (int e = lane; e < M / 2; e += 32) {
            const int row = e / half, j = e % half;
            const float2 *x = src + row * Mx;
            const int k = j & (Ns - 1);
            const float2 a = x[j];
            const float2 b = cmul(x[j + half], twx[k * (half / Ns)]);
            float2 *o = dst + row * Mx + ((j - k) << 1) + k;
            o[0] = cadd(a, b);
            o[Ns] = csub(a, b);
        }
        __syncwarp();
        float2 *t = src;
        src = dst;
        dst = t;
    }
    const float2 *yb = src;   // [Mz][Mx]: beam m = m_x Mz + m_z at m_z Mx + m_x

    // window gather: a lane per entry of the flat (target, entry) list
    const int64_t v = ga.vbase + vid;
    const int p = (int)(v >> ga.log2F);
    const int q = (int)(v & ((1 << ga.log2F) - 1));
    const int s = q >> ga.log2B, i = q & ((1 << ga.log2B) - 1);
    const bool train = p < ga.P_train;
    const int v0 = train ? (p << ga.log2B) + i : ((p - ga.P_train) << ga.log2B) + i;
    const float sc_tr = (prec == BS_PREC_FP32) ? 1.f : ga.store_scale;
    for (int e = lane; e < sumW; e += 32) {
        const int packed = __ldg(&glist[e]);
        const int t = packed >> 8, w = packed & 255;
        const int64_t g = (int64_t)t * ga.L + s;
        const int W = __ldg(&ga.Wg[g]);
        const int wz = __ldg(&Wz[t]);
        const int mx = (__ldg(&ga.start[g]) + w / wz) & (Mx - 1);
        const int mz = (__ldg(&start_z[g]) + w % wz) & (Mz - 1);
        const float2 val = cscale(yb[mz * Mx + mx], scale);
        if (!train) {
            ga.zte[__ldg(&ga.zte_off[g]) + (int64_t)v0 * W + w] = val;
        } else if (v0 < __ldg(&ga.Kg[g])) {
            const int64_t idx = __ldg(&ga.ztr_off[g]) + (int64_t)v0 * W + w;
            if (prec == BS_PREC_FP16) store_train<BS_PREC_FP16>(ga.ztr, idx, val, sc_tr);
            else if (prec == BS_PREC_BF16) store_train<BS_PREC_BF16>(ga.ztr, idx, val, sc_tr);
            else store_train<BS_PREC_FP32>(ga.ztr, idx, val, 1.f);
        }
    }
}

bs_status launch_beamspace2d(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st) {
    const int Nx = p->Nx, Nz = p->Nz, Mx = p->Mx, Mz = p->Mz;
    if (ga.nvec == 0) return BS_OK;
    const size_t per_warp = ((size_t)Nx * Nz + 2 * (size_t)Mx * Mz) * sizeof(float2);
    const size_t tables = ((size_t)Mx / 2 + Mz) * sizeof(float2);
    // up to 4 vectors (warps) per CTA while their buffers stay within 48 KB
    int nw = (int)std::min<size_t>(4, std::max<size_t>(1, (48 * 1024 - tables) / per_warp));
    const size_t smem = tables + (size_t)nw * per_warp;
    const int64_t blocks = (ga.nvec + nw - 1) / nw;
    if (blocks > 0x7FFFFFFF) return set_error(BS_EUNSUPPORTED, "too many vectors");
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(beamspace2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "planar beamspace attribute");
    }
    beamspace2d_kernel<<<(unsigned)blocks, 32 * nw, smem, st>>>(xc, Nx, Nz, Mx, Mz, 1.0f / sqrtf((float)(Mx * Mz)),
                                                              p->cfg.precision, ga, p->d_start_z, p->d_Wz,
                                                              p->d_glist, p->sumW);
    return check_launch("planar beamspace launch");
}

}  // namespace bs
