// Planar-array beamspace transform and window gather (Eq. ArrayFactor,
// Eq. VerDFT, Eq. HorDFT, Eq. OverallDFT, Eq. BeamTransform, Eq.
// OverallWindow read as S_h (x) S_v, Eq. ApplyWindow).
//
// Elements n = n_x Nz + n_z, beams m = m_x Mz + m_z, window entries
// w = w_x Wz + w_z.  One CTA per (record, bin) vector: its N = Nx Nz elements
// are staged in shared memory, the vertical DFT (Mz points of Nz, D_v) and
// then the horizontal one (Mx points of Nx, D_h^T) run as direct sums with
// twiddles from two small exact tables, leaving all M = Mx Mz beams in
// shared memory; each target's Wx x Wz window is then written to the packed
// window arrays with the conventions of the linear-array kernels.  Planar
// plans are limited to N <= 1024 and M <= 2048 (the paper's array is 4 x 32).
#include "beamspace_dev.cuh"
#include "internal.h"

#include <algorithm>

namespace bs {

__global__ void __launch_bounds__(128)
    beamspace2d_kernel(const float2 *__restrict__ y, int Nx, int Nz, int Mx, int Mz, float scale, int prec,
                       GatherArgs ga, const int32_t *__restrict__ start_z, const int32_t *__restrict__ Wz) {
    extern __shared__ float2 sm2[];
    const int N = Nx * Nz, M = Mx * Mz;
    float2 *ys = sm2;              // [N]
    float2 *yv = ys + N;           // [Nx][Mz]
    float2 *yb = yv + Nx * Mz;     // [Mx][Mz]
    float2 *twx = yb + M;          // [Mx] e^{-j 2 pi k / Mx}
    float2 *twz = twx + Mx;        // [Mz]
    const int tid = threadIdx.x;
    const int64_t vid = blockIdx.x;
    for (int n = tid; n < N; n += 128) ys[n] = __ldcs(&y[vid * N + n]);
    for (int k = tid; k < Mx; k += 128) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)Mx, &sn, &cs);
        twx[k] = make_float2(cs, sn);
    }
    for (int k = tid; k < Mz; k += 128) {
        float sn, cs;
        sincospif(-2.f * (float)k / (float)Mz, &sn, &cs);
        twz[k] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int e = tid; e < Nx * Mz; e += 128) {   // vertical DFT of every column n_x
        const int nx = e / Mz, mz = e % Mz;
        float2 acc = make_float2(0.f, 0.f);
        for (int nz = 0; nz < Nz; ++nz) acc = cadd(acc, cmul(ys[nx * Nz + nz], twz[(mz * nz) & (Mz - 1)]));
        yv[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < M; e += 128) {         // horizontal DFT of every vertical beam m_z
        const int mx = e / Mz, mz = e % Mz;
        float2 acc = make_float2(0.f, 0.f);
        for (int nx = 0; nx < Nx; ++nx) acc = cadd(acc, cmul(yv[nx * Mz + mz], twx[(mx * nx) & (Mx - 1)]));
        yb[e] = cscale(acc, scale);
    }
    __syncthreads();

    // window gather: a warp per target, a lane per window entry (W <= 16)
    const int64_t v = ga.vbase + vid;
    const int p = (int)(v >> ga.log2F);
    const int q = (int)(v & ((1 << ga.log2F) - 1));
    const int s = q >> ga.log2B, i = q & ((1 << ga.log2B) - 1);
    const bool train = p < ga.P_train;
    const int v0 = train ? (p << ga.log2B) + i : ((p - ga.P_train) << ga.log2B) + i;
    const float sc_tr = (prec == BS_PREC_FP32) ? 1.f : ga.store_scale;
    const int lane = tid & 31, warp = tid >> 5;
    for (int t = warp; t < ga.T; t += 4) {
        const int64_t g = (int64_t)t * ga.L + s;
        const int W = __ldg(&ga.Wg[g]);
        if (lane >= W) continue;
        const int wz = __ldg(&Wz[t]);
        const int mx = (__ldg(&ga.start[g]) + lane / wz) & (Mx - 1);
        const int mz = (__ldg(&start_z[g]) + lane % wz) & (Mz - 1);
        const float2 val = yb[mx * Mz + mz];
        if (!train) {
            ga.zte[__ldg(&ga.zte_off[g]) + (int64_t)v0 * W + lane] = val;
        } else if (v0 < __ldg(&ga.Kg[g])) {
            const int64_t idx = __ldg(&ga.ztr_off[g]) + (int64_t)v0 * W + lane;
            if (prec == BS_PREC_FP16) store_train<BS_PREC_FP16>(ga.ztr, idx, val, sc_tr);
            else if (prec == BS_PREC_BF16) store_train<BS_PREC_BF16>(ga.ztr, idx, val, sc_tr);
            else store_train<BS_PREC_FP32>(ga.ztr, idx, val, 1.f);
        }
    }
}

bs_status launch_beamspace2d(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st) {
    const int Nx = p->Nx, Nz = p->Nz, Mx = p->Mx, Mz = p->Mz;
    const size_t smem = ((size_t)Nx * Nz + (size_t)Nx * Mz + (size_t)Mx * Mz + Mx + Mz) * sizeof(float2);
    if (ga.nvec == 0) return BS_OK;
    if (ga.nvec > 0x7FFFFFFF) return set_error(BS_EUNSUPPORTED, "too many vectors");
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(beamspace2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "planar beamspace attribute");
    }
    beamspace2d_kernel<<<(unsigned)ga.nvec, 128, smem, st>>>(xc, Nx, Nz, Mx, Mz, 1.0f / sqrtf((float)(Mx * Mz)),
                                                            p->cfg.precision, ga, p->d_start_z, p->d_Wz);
    return check_launch("planar beamspace launch");
}

}  // namespace bs
