// Stand-alone MVDR solve (Eq. BeamCorrMVDR) of every pair from its stored
// FP64 covariance: one half-warp per pair, eight pairs per CTA.  The solve
// itself (FP32 Cholesky, FP64-residual refinement, FP64 escalation) is
// solve_pair() in solve_dev.cuh.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "solve_dev.cuh"

namespace bs {

constexpr int SOLVE_PAIRS_PER_CTA = 8;

__global__ void __launch_bounds__(SOLVE_PAIRS_PER_CTA * 16, 5)
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
    solve_pair(mask, lane, Wg[g], R + roff[g], at32 + wo, atlo + wo, at64 + wo, c + wo, info + g, kappa_max, refine,
               allow_f64, scratch[hw], dpre ? dpre + wo : nullptr);
}

// Plain FP32 per-pair solve: one thread factorises and solves its pair in
// shared memory (no refinement, no FP64), c = v / |u|^2.
__global__ void plain_solve_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                                   const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                                   const float2 *__restrict__ at32, float2 *__restrict__ c,
                                   int32_t *__restrict__ info) {
    __shared__ float2 Lm[WMAX][WMAX];
    __shared__ float2 u[WMAX], v[WMAX];
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
    if (p->Wmax > WMAX) return set_error(BS_EUNSUPPORTED, "W > 16");
    if (p->cfg.flags & BS_FLAG_PLAIN) {
        plain_solve_kernel<<<(unsigned)G, 32, 0, st>>>(R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, c, info);
        return check_launch("plain solve launch");
    }
    const unsigned blocks = (unsigned)((G + SOLVE_PAIRS_PER_CTA - 1) / SOLVE_PAIRS_PER_CTA);
    mvdr_solve_kernel<<<blocks, SOLVE_PAIRS_PER_CTA * 16, 0, st>>>(
        R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, p->d_atlo, p->d_at64, c, info, G, p->cfg.kappa_max,
        (p->cfg.flags & BS_FLAG_NO_REFINE) ? 0 : 1, (p->cfg.flags & BS_FLAG_NO_FP64) ? 0 : 1,
        p->Wmin == p->Wmax ? nullptr : p->d_order_w, dpre);
    return check_launch("solve launch");
}

}  // namespace bs
