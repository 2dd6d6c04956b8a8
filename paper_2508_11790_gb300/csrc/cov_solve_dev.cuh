// Fused loaded covariance + MVDR solve over (target, subband) pairs of uneven
// window size W and training count K, in one persistent launch
// (Eq. EmpiricalCov on the windowed vectors, Eq. BeamCorrMVDR).
//
// Every half-warp is an independent worker: it takes the next pair from a
// work queue (an atomic head over a pair order sorted by decreasing cost
// W^2 K, so the tail of the launch is made of cheap pairs) and
//   1. forms the lower triangle of sum_k z_k z_k^H: its 16 lanes take
//      (3x3 tile, k-slice) tasks; a task loads 6 window entries per vector
//      (read-only path) and does 9 complex multiply-adds; FP32 sums cover
//      kCsFold = 4 vectors and are folded into double-float (hi, lo)
//      (with 16 the worst C4 weight error was 1.9e-3);
//   2. reduces the slices in double-float and forms R = sum / K + delta I in
//      double-float, stored as FP64 in its shared memory (optionally also in
//      global memory);
//   3. solves (solve_pair: FP32 Cholesky, FP64-residual refinement, FP64
//      escalation) and writes c and info.
// No CTA-wide barrier is involved, so one half-warp's solve overlaps the
// other half-warps' covariance work; the covariance never goes to HBM.
#pragma once
#include "common.cuh"
#include "internal.h"
#include "solve_dev.cuh"

namespace bs {

constexpr int kCsFold = 4;   // vectors per FP32 partial sum

__device__ __forceinline__ void df_acc(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}

template <int PREC>
__device__ __forceinline__ float2 load_window_cs(const void *z, int64_t idx, float inv_sc) {
    if constexpr (PREC == BS_PREC_FP32) {
        return __ldcs(reinterpret_cast<const float2 *>(z) + idx);
    } else if constexpr (PREC == BS_PREC_FP16) {
        const float2 f = __half22float2(reinterpret_cast<const __half2 *>(z)[idx]);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    } else {
        const float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(z)[idx]);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    }
}

struct CovSolveArgs {
    const void *z;
    const int64_t *ztr_off;
    const int32_t *Wg, *Kg;
    const int64_t *woff, *roff;
    const float2 *at32, *atlo;
    const double2 *at64;
    const int32_t *order;     // pair order of the queue (NULL: identity)
    int64_t pairs;
    const float *delta_pair;  // NULL: delta
    double delta;
    DF delta_df;              // delta as a double-float
    float inv_sc;
    double kappa_max;
    int refine, allow_f64;
    float2 *c;
    int32_t *info;
    double2 *R;               // optional FP64 covariance output
    int *head;                // work-queue head, 0 at launch
};

// Per half-warp shared memory: the FP64 covariance of its pair and a
// scratch area used first for the slice partials, then by the solve.
struct HalfWarpSmem {
    double2 R[WMAX * WMAX];
    union {
        float red[21][9][4];             // (task, entry, {hr, lr, hi, li})
        double2 solve[WMAX][WMAX + 1];   // solve_pair scratch
    } u;
};

template <int PREC, int NTH>
__global__ void __launch_bounds__(NTH) cov_solve_kernel(CovSolveArgs a) {
    extern __shared__ __align__(16) unsigned char cs_smem[];
    HalfWarpSmem *hws = reinterpret_cast<HalfWarpSmem *>(cs_smem);
    const int hw = threadIdx.x >> 4;
    const int lane = threadIdx.x & 15;
    const unsigned mask = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    HalfWarpSmem &S = hws[hw];

    for (;;) {
        long long idx = 0;
        if (lane == 0) idx = atomicAdd(a.head, 1);
        idx = __shfl_sync(mask, idx, 0, 16);
        if (idx >= a.pairs) break;   // uniform over the half-warp
        const int64_t g = a.order ? (int64_t)a.order[idx] : (int64_t)idx;
        const int W = a.Wg[g], K = a.Kg[g];
        const int nb3 = (W + 2) / 3;
        const int nblk = nb3 * (nb3 + 1) / 2;          // 3x3 tiles of the lower triangle
        const int H = nblk >= 16 ? 1 : 16 / nblk;      // k-slices
        const int ntask = nblk * H;
        const int64_t zb = a.ztr_off[g];

        for (int task = lane; task < ntask; task += 16) {
            const int tile = task % nblk, h = task / nblk;
            int bi = 0, rem = tile;
            while (rem > bi) { rem -= bi + 1; ++bi; }
            const int i0 = 3 * bi, j0 = 3 * rem;
            float ar[3][3], ai[3][3], hr[3][3], lr[3][3], hi[3][3], li[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) ar[r][q] = ai[r][q] = hr[r][q] = lr[r][q] = hi[r][q] = li[r][q] = 0.f;
            int cnt = 0;
            for (int v = h; v < K; v += H) {
                const int64_t base = zb + (int64_t)v * W;
                float2 zi[3], zj[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    zi[r] = (i0 + r < W) ? load_window_cs<PREC>(a.z, base + i0 + r, a.inv_sc) : make_float2(0.f, 0.f);
                    zj[r] = (j0 + r < W) ? load_window_cs<PREC>(a.z, base + j0 + r, a.inv_sc) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {   // z_i conj(z_j)
                        ar[r][q] = fmaf(zi[r].x, zj[q].x, fmaf(zi[r].y, zj[q].y, ar[r][q]));
                        ai[r][q] = fmaf(zi[r].y, zj[q].x, fmaf(-zi[r].x, zj[q].y, ai[r][q]));
                    }
                if (++cnt == kCsFold) {
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            df_acc(hr[r][q], lr[r][q], ar[r][q]);
                            df_acc(hi[r][q], li[r][q], ai[r][q]);
                            ar[r][q] = ai[r][q] = 0.f;
                        }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    df_acc(hr[r][q], lr[r][q], ar[r][q]);
                    df_acc(hi[r][q], li[r][q], ai[r][q]);
                    float *o = S.u.red[task][3 * r + q];
                    o[0] = hr[r][q];
                    o[1] = lr[r][q];
                    o[2] = hi[r][q];
                    o[3] = li[r][q];
                }
        }
        __syncwarp(mask);

        // slice reduction and the loaded covariance in double-float; FP64 only
        // for the stored value of each entry
        const float Kf = (float)K;
        const float qk = 1.f / Kf;
        const DF invK = df_norm(qk, fmaf(-qk, Kf, 1.f) / Kf);   // 1/K (K < 2^24)
        const DF dl = a.delta_pair ? DF{a.delta_pair[g], 0.f} : a.delta_df;
        const int E = W * (W + 1) / 2;
        for (int e = lane; e < E; e += 16) {
            int i = 0, r2 = e;
            while (r2 > i) { r2 -= i + 1; ++i; }
            const int j = r2;
            const int b = (i / 3) * (i / 3 + 1) / 2 + j / 3;
            const int ee = 3 * (i % 3) + (j % 3);
            float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
            for (int hh = 0; hh < H; ++hh) {
                const float *o = S.u.red[hh * nblk + b][ee];
                df_acc(sh, sl, o[0]);
                sl += o[1];
                df_acc(th, tl, o[2]);
                tl += o[3];
            }
            const DF re = df_mul(df_norm(sh, sl), invK);
            if (i == j) {
                S.R[i * W + i] = make_double2(df_to_double(df_add(re, dl)), 0.0);
            } else {
                const double rd = df_to_double(re), id = df_to_double(df_mul(df_norm(th, tl), invK));
                S.R[i * W + j] = make_double2(rd, id);
                S.R[j * W + i] = make_double2(rd, __longlong_as_double(__double_as_longlong(id) ^ (1ll << 63)));
            }
        }
        __syncwarp(mask);
        if (a.R) {
            double2 *Rg = a.R + a.roff[g];
            for (int e = lane; e < W * W; e += 16) Rg[e] = S.R[e];
        }
        const int64_t wo = a.woff[g];
        solve_pair(mask, lane, W, S.R, a.at32 + wo, a.atlo + wo, a.at64 + wo, a.c + wo, a.info + g, a.kappa_max, a.refine,
                   a.allow_f64, S.u.solve);
        __syncwarp(mask);
    }
}

template <int PREC, int NTH>
bs_status launch_cs_t(const CovSolveArgs &a, int grid, cudaStream_t st) {
    constexpr size_t smem = (NTH / 16) * sizeof(HalfWarpSmem);
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            return cuda_error(cudaFuncSetAttribute(cov_solve_kernel<PREC, NTH>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              "cov_solve attribute");
        }))
        return s;
    cov_solve_kernel<PREC, NTH><<<grid, NTH, smem, st>>>(a);
    return check_launch("cov_solve launch");
}

// One explicit instantiation per precision lives in its own translation
// unit (cov_solve_fp32.cu, cov_solve_fp16.cu, cov_solve_bf16.cu) so that the
// three compile in parallel.
template <int PREC>
bs_status launch_cs_prec(const CovSolveArgs &a, int grid, cudaStream_t st);

}  // namespace bs
