// Stand-alone MVDR solve (Eq. BeamCorrMVDR) of every pair from its stored
// FP64 covariance: one launch per window size present, pairs visited in
// the plan's W-grouped order.  An 8-lane group solves a pair of W <= 8, a
// half-warp one of 8 < W <= 16, a warp one of 16 < W <= 32.  The solve
// itself (FP32 Cholesky, compensated refinement, FP64 escalation) is
// solve_pair_body() in solve_dev.cuh.
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "solve_dev.cuh"

namespace bs {

// The pairs of one window size W <= 16, solved by a kernel compiled for
// that size alone: one kernel holding the bodies of all sixteen sizes
// behind a switch stalled mostly on instruction fetch.  GW = 8 lanes per
// pair for W <= 8 (sixteen pairs per CTA), else 16 (eight pairs per CTA).
template <int WT>
__global__ void __launch_bounds__(128, 4)
    mvdr_solve_w_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                        const int64_t *__restrict__ woff, const float2 *__restrict__ at32,
                        const float2 *__restrict__ atlo, const double2 *__restrict__ at64, float2 *__restrict__ c,
                        int32_t *__restrict__ info, int64_t slot0, int64_t slot1, double kappa_max, int refine,
                        int allow_f64, const int32_t *__restrict__ order, const float *__restrict__ dpre) {
    constexpr int GW = (WT <= 8) ? 8 : 16;
    constexpr int PPC = 128 / GW;
    __shared__ double2 scratch[PPC][GW][GW + 1];
    const int grp = threadIdx.x / GW;
    const int lane = threadIdx.x % GW;
    const unsigned mask = (GW == 8) ? (0xFFu << (threadIdx.x & 24)) : ((threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu);
    const int64_t slot = slot0 + (int64_t)blockIdx.x * PPC + grp;
    if (slot >= slot1) return;   // uniform over the group
    const int64_t g = order ? (int64_t)order[slot] : slot;
    const int64_t wo = woff[g];
    solve_pair_body<WT, GW>(mask, lane, R + roff[g], at32 + wo, atlo + wo, at64 + wo, c + wo, info + g, kappa_max,
                            refine, allow_f64, scratch[grp], dpre ? dpre + wo : nullptr);
}

// The pairs of window size WT: slots wstart[WT] .. wstart[WT + 1] - 1 of
// the W-grouped order (the identity when every pair has that size).
template <int WT>
bs_status launch_solve_w(const bs_plan *p, const double2 *R, float2 *c, int32_t *info, cudaStream_t st,
                         const float *dpre, int refine, int f64) {
    constexpr int PPC = 128 / ((WT <= 8) ? 8 : 16);
    const int64_t s0 = p->wstart[WT], s1 = p->wstart[WT + 1];
    if (s1 <= s0) return BS_OK;
    const int32_t *order = p->Wmin == p->Wmax ? nullptr : p->d_order_w;
    const unsigned blocks = (unsigned)((s1 - s0 + PPC - 1) / PPC);
    mvdr_solve_w_kernel<WT><<<blocks, 128, 0, st>>>(R, p->d_roff, p->d_woff, p->d_at32, p->d_atlo, p->d_at64, c,
                                                    info, s0, s1, p->cfg.kappa_max, refine, f64, order, dpre);
    return check_launch("solve (one window size) launch");
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

// Fork: the first nst - 1 side streams of the plan wait for `st`.
static bs_status fork_streams(const bs_plan *p, cudaStream_t st, int nst) {
    if (nst <= 1) return BS_OK;
    cudaError_t e = cudaEventRecord(p->ev_fork, st);
    for (int k = 0; k + 1 < nst && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->solve_st[k], p->ev_fork, 0);
    return e == cudaSuccess ? BS_OK : cuda_error(e, "solve fork");
}
// Join: `st` waits for everything issued to those side streams.
static bs_status join_streams(const bs_plan *p, cudaStream_t st, int nst) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k + 1 < nst && e == cudaSuccess; ++k) {
        e = cudaEventRecord(p->ev_join[k], p->solve_st[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_join[k], 0);
    }
    return e == cudaSuccess ? BS_OK : cuda_error(e, "solve join");
}
static int window_classes(const bs_plan *p) {
    int n = 0;
    for (int w = 1; w <= 16; ++w) n += p->wstart[w + 1] > p->wstart[w];
    return n;
}

bool cov_solve_chains_apply(const bs_plan *p) {
    return !(p->cfg.flags & BS_FLAG_PLAIN) && p->nsmall == p->pairs && window_classes(p) > 1 &&
           window_cov_uses_warp(p);
}

bs_status launch_cov_solve_chains(const bs_plan *p, const void *ztr, double2 *R, float2 *c, int32_t *info,
                                  cudaStream_t st) {
    const int refine = (p->cfg.flags & BS_FLAG_NO_REFINE) ? 0 : 1;
    const int f64 = (p->cfg.flags & BS_FLAG_NO_FP64) ? 0 : 1;
    const int ncls = window_classes(p);
    const int nst = ncls < 1 + bs_plan::kSolveStreams ? ncls : 1 + bs_plan::kSolveStreams;
    if (bs_status s = fork_streams(p, st, nst)) return s;
    int li = 0;
    // one chain per window size (covariance of its pairs, then their solve),
    // largest windows first, chain i on stream i mod nst
#define BS_CHAIN(n)                                                                                          \
    if (p->wstart[n + 1] > p->wstart[n]) {                                                                   \
        const int k_ = li++ % nst;                                                                           \
        const cudaStream_t s_ = k_ == 0 ? st : p->solve_st[k_ - 1];                                          \
        if (bs_status s = launch_window_cov_warp(p, ztr, nullptr, R, s_, p->wstart[n], p->wstart[n + 1],     \
                                                 p->d_order_w))                                              \
            return s;                                                                                        \
        if (bs_status s = launch_solve_w<n>(p, R, c, info, s_, nullptr, refine, f64)) return s;              \
    }
    BS_CHAIN(16) BS_CHAIN(15) BS_CHAIN(14) BS_CHAIN(13) BS_CHAIN(12) BS_CHAIN(11) BS_CHAIN(10) BS_CHAIN(9)
    BS_CHAIN(8) BS_CHAIN(7) BS_CHAIN(6) BS_CHAIN(5) BS_CHAIN(4) BS_CHAIN(3) BS_CHAIN(2) BS_CHAIN(1)
#undef BS_CHAIN
    return join_streams(p, st, nst);
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
    // windows of up to 16 beams: one launch per window size present, each of
    // a kernel compiled for that size alone.  The launches are independent
    // (disjoint pairs): with several, they are spread over `st` and the
    // plan's side streams (forked from `st` and joined back into it; under
    // graph capture, parallel branches), so that one launch's tail overlaps
    // the others' work.
    const int64_t nsmall = p->nsmall;   // pairs with W <= 16 come first
    const int nlaunch = (nsmall < G ? 1 : 0) + window_classes(p);
    const int nst = nlaunch < 1 + bs_plan::kSolveStreams ? nlaunch : 1 + bs_plan::kSolveStreams;
    if (bs_status s = fork_streams(p, st, nst)) return s;
    int li = 0;   // launches issued; launch i goes to stream i mod nst
    auto next_stream = [&]() -> cudaStream_t {
        const int k = li++ % (nst > 0 ? nst : 1);
        return k == 0 ? st : p->solve_st[k - 1];
    };
    // largest windows first: the longest launches start first on their streams
#define BS_SOLVE_W(n)                                                                                  \
    if (p->wstart[n + 1] > p->wstart[n])                                                               \
        if (bs_status s = launch_solve_w<n>(p, R, c, info, next_stream(), dpre, refine, f64)) return s;
    BS_SOLVE_W(16) BS_SOLVE_W(15) BS_SOLVE_W(14) BS_SOLVE_W(13) BS_SOLVE_W(12) BS_SOLVE_W(11)
    BS_SOLVE_W(10) BS_SOLVE_W(9) BS_SOLVE_W(8) BS_SOLVE_W(7) BS_SOLVE_W(6) BS_SOLVE_W(5) BS_SOLVE_W(4)
    BS_SOLVE_W(3) BS_SOLVE_W(2) BS_SOLVE_W(1)
#undef BS_SOLVE_W
    const int32_t *order = p->Wmin == p->Wmax ? nullptr : p->d_order_w;   // pairs grouped by W, smallest first
    if (nsmall < G) {
        const cudaStream_t ws = next_stream();
        constexpr size_t smem = WIDE_WARPS * sizeof(WideSmem);
        static PerDevice attr;
        if (bs_status s = attr.get([](int *) {
                return cuda_error(cudaFuncSetAttribute(mvdr_solve_wide_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "solve (wide) attribute");
            }))
            return s;
        const unsigned blocks = (unsigned)((G - nsmall + WIDE_WARPS - 1) / WIDE_WARPS);
        mvdr_solve_wide_kernel<<<blocks, WIDE_WARPS * 32, smem, ws>>>(
            R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, p->d_atlo, p->d_at64, c, info, nsmall, G, p->cfg.kappa_max,
            refine, f64, order, dpre);
        if (bs_status s = check_launch("solve (wide) launch")) return s;
    }
    return join_streams(p, st, nst);   // `st` waits for every side stream's launches
}

}  // namespace bs
