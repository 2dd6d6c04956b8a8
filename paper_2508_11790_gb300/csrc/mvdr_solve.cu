// Stand-alone MVDR solve (Eq. BeamCorrMVDR) of every pair from its stored
// FP64 covariance: one half-warp per pair (W <= 16), eight pairs per CTA,
// or one warp per pair (16 < W <= 32).  The solve itself (FP32 Cholesky,
// compensated refinement, FP64 escalation) is solve_pair_fixed() in
// solve_dev.cuh.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "solve_dev.cuh"

namespace bs {

constexpr int SOLVE_PAIRS_PER_CTA = 8;

__global__ void __launch_bounds__(SOLVE_PAIRS_PER_CTA * 16, 4)
    mvdr_solve_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                      const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                      const float2 *__restrict__ at32, const float2 *__restrict__ atlo,
                      const double2 *__restrict__ at64, float2 *__restrict__ c, int32_t *__restrict__ info,
                      int64_t pairs, double kappa_max, int refine, int allow_f64, const int32_t *__restrict__ order,
                      const float *__restrict__ dpre) {
    __shared__ double2 scratch[SOLVE_PAIRS_PER_CTA][WMAX][WMAX + 1];
    const int hw = threadIdx.x >> 4;
    const int lane = threadIdx.x & 15;
    const unsigned mask = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    const int64_t slot = (int64_t)blockIdx.x * SOLVE_PAIRS_PER_CTA + hw;
    if (slot >= pairs) return;   // uniform over the half-warp
    const int64_t g = order ? (int64_t)order[slot] : slot;   // pairs grouped by W
    const int64_t wo = woff[g];
    solve_pair_inline(mask, lane, Wg[g], R + roff[g], at32 + wo, atlo + wo, at64 + wo, c + wo, info + g, kappa_max,
                      refine, allow_f64, scratch[hw], dpre ? dpre + wo : nullptr);
}

// Windows of 17..32 beams: one warp per pair, solved at WT = 24 or 32 with
// the pair's covariance copied to shared memory padded to WT x WT.  The
// padding has zero off-diagonal entries, R_00 on its diagonal and the
// preconditioner entry of row 0, so its Cholesky pivots equal the pair's
// first pivot (the pivot ratio that decides FP64 escalation is the pair's);
// with zero steering entries there the padded solution entries are exactly
// zero, and the first W entries are the W x W solve.
constexpr int WIDE_WARPS = 4;
struct WideSmem {
    double2 R[WMAX_WIDE * WMAX_WIDE];
    double2 scratch[WMAX_WIDE][WMAX_WIDE + 1];
    double2 a64[WMAX_WIDE];
    float2 a32[WMAX_WIDE], alo[WMAX_WIDE], c[WMAX_WIDE];
    float d[WMAX_WIDE];
};

template <int WT>
__device__ __forceinline__ void solve_wide(int lane, int W, const double2 *Rg, const float2 *a32, const float2 *alo,
                                           const double2 *a64, const float *dg, float2 *cg, int32_t *info,
                                           double kappa_max, int refine, int allow_f64, WideSmem &S) {
    for (int e = lane; e < WT * WT; e += 32) {
        const int i = e / WT, j = e % WT;
        S.R[e] = (i < W && j < W) ? Rg[i * W + j] : (i == j ? Rg[0] : make_double2(0.0, 0.0));
    }
    const bool row = lane < W;
    S.a32[lane] = row ? a32[lane] : make_float2(0.f, 0.f);
    S.alo[lane] = row ? alo[lane] : make_float2(0.f, 0.f);
    S.a64[lane] = row ? a64[lane] : make_double2(0.0, 0.0);
    if (dg) S.d[lane] = row ? dg[lane] : dg[0];
    __syncwarp();
    solve_pair_fixed<WT, 32>(0xFFFFFFFFu, lane, S.R, S.a32, S.alo, S.a64, S.c, info, kappa_max, refine, allow_f64,
                             S.scratch, dg ? S.d : nullptr);
    __syncwarp();
    if (row) cg[lane] = S.c[lane];
}

__global__ void __launch_bounds__(WIDE_WARPS * 32)
    mvdr_solve_wide_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                           const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                           const float2 *__restrict__ at32, const float2 *__restrict__ atlo,
                           const double2 *__restrict__ at64, float2 *__restrict__ c, int32_t *__restrict__ info,
                           int64_t slot0, int64_t slot1, double kappa_max, int refine, int allow_f64,
                           const int32_t *__restrict__ order, const float *__restrict__ dpre) {
    extern __shared__ __align__(16) unsigned char wide_smem[];
    WideSmem &S = reinterpret_cast<WideSmem *>(wide_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t slot = slot0 + (int64_t)blockIdx.x * WIDE_WARPS + (threadIdx.x >> 5);
    if (slot >= slot1) return;   // uniform over the warp
    const int64_t g = order ? (int64_t)order[slot] : slot;
    const int W = Wg[g];
    const int64_t wo = woff[g];
    const float *dg = dpre ? dpre + wo : nullptr;
    if (W <= 24)
        solve_wide<24>(lane, W, R + roff[g], at32 + wo, atlo + wo, at64 + wo, dg, c + wo, info + g, kappa_max, refine,
                       allow_f64, S);
    else
        solve_wide<32>(lane, W, R + roff[g], at32 + wo, atlo + wo, at64 + wo, dg, c + wo, info + g, kappa_max, refine,
                       allow_f64, S);
}

// Plain FP32 per-pair solve: one thread factorises and solves its pair in
// shared memory (no refinement, no FP64), c = v / |u|^2.
__global__ void plain_solve_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                                   const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                                   const float2 *__restrict__ at32, float2 *__restrict__ c,
                                   int32_t *__restrict__ info) {
    __shared__ float2 Lm[WMAX_WIDE][WMAX_WIDE];
    __shared__ float2 u[WMAX_WIDE], v[WMAX_WIDE];
    const int64_t g = blockIdx.x;
    const int W = Wg[g];
    const double2 *Rg = R + roff[g];
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        const double2 r = Rg[e];
        Lm[e / W][e % W] = make_float2((float)r.x, (float)r.y);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int fail = 0;
    for (int k = 0; k < W && !fail; ++k) {
        float d = Lm[k][k].x;
        for (int m = 0; m < k; ++m) d -= Lm[k][m].x * Lm[k][m].x + Lm[k][m].y * Lm[k][m].y;
        if (!(d > 0.f)) { fail = k + 1; break; }
        d = sqrtf(d);
        Lm[k][k] = make_float2(d, 0.f);
        for (int i = k + 1; i < W; ++i) {
            float2 s = Lm[i][k];
            for (int m = 0; m < k; ++m) s = csub(s, cmulc(Lm[i][m], Lm[k][m]));
            Lm[i][k] = cscale(s, 1.f / d);
        }
    }
    if (fail) {
        for (int i = 0; i < W; ++i) c[woff[g] + i] = make_float2(nanf(""), nanf(""));
        info[g] = fail;
        return;
    }
    float nu = 0.f;
    for (int i = 0; i < W; ++i) {
        float2 s = at32[woff[g] + i];
        for (int m = 0; m < i; ++m) s = csub(s, cmul(Lm[i][m], u[m]));
        u[i] = cscale(s, 1.f / Lm[i][i].x);
        nu += u[i].x * u[i].x + u[i].y * u[i].y;
    }
    for (int i = W - 1; i >= 0; --i) {
        float2 s = u[i];
        for (int m = i + 1; m < W; ++m) s = csub(s, conjmul(Lm[m][i], v[m]));
        v[i] = cscale(s, 1.f / Lm[i][i].x);
    }
    for (int i = 0; i < W; ++i) c[woff[g] + i] = cscale(v[i], 1.f / nu);
    info[g] = 0;
}

bs_status launch_mvdr_solve(const bs_plan *p, const double2 *R, float2 *c, int32_t *info, cudaStream_t st,
                            const float *dpre) {
    const int64_t G = p->pairs;
    if (p->Wmax > WMAX_WIDE) return set_error(BS_EUNSUPPORTED, "W > 32");
    if (p->cfg.flags & BS_FLAG_PLAIN) {
        plain_solve_kernel<<<(unsigned)G, 32, 0, st>>>(R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, c, info);
        return check_launch("plain solve launch");
    }
    const int refine = (p->cfg.flags & BS_FLAG_NO_REFINE) ? 0 : 1;
    const int f64 = (p->cfg.flags & BS_FLAG_NO_FP64) ? 0 : 1;
    const int32_t *order = p->Wmin == p->Wmax ? nullptr : p->d_order_w;   // pairs grouped by W, smallest first
    const int64_t nsmall = p->nsmall;                                       // pairs with W <= 16 come first
    if (nsmall > 0) {
        const unsigned blocks = (unsigned)((nsmall + SOLVE_PAIRS_PER_CTA - 1) / SOLVE_PAIRS_PER_CTA);
        mvdr_solve_kernel<<<blocks, SOLVE_PAIRS_PER_CTA * 16, 0, st>>>(
            R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, p->d_atlo, p->d_at64, c, info, nsmall, p->cfg.kappa_max,
            refine, f64, order, dpre);
        if (bs_status s = check_launch("solve launch")) return s;
    }
    if (nsmall < G) {
        constexpr size_t smem = WIDE_WARPS * sizeof(WideSmem);
        static PerDevice attr;
        if (bs_status s = attr.get([](int *) {
                return cuda_error(cudaFuncSetAttribute(mvdr_solve_wide_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "solve (wide) attribute");
            }))
            return s;
        const unsigned blocks = (unsigned)((G - nsmall + WIDE_WARPS - 1) / WIDE_WARPS);
        mvdr_solve_wide_kernel<<<blocks, WIDE_WARPS * 32, smem, st>>>(
            R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, p->d_atlo, p->d_at64, c, info, nsmall, G, p->cfg.kappa_max,
            refine, f64, order, dpre);
        if (bs_status s = check_launch("solve (wide) launch")) return s;
    }
    return BS_OK;
}

}  // namespace bs
