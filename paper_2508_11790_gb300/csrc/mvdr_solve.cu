// MVDR correlator per (target, subband) pair (Eq. BeamCorrMVDR):
//   c = R^-1 a~ / (a~^H R^-1 a~).
//
// Batched Cholesky with one half-warp (16 lanes) per pair, W <= 16: lane i
// holds row i of R in registers.
//   1. R = L L^H in FP32 (right-looking; column k broadcast by shuffles);
//   2. u = L^-1 a~, v = L^-H u (triangular solves, one shuffle per step;
//      the backward solve reads L transposed from shared memory);
//   3. one refinement step: r = a~ - R v with R and the products in FP64,
//      v += L^-H L^-1 r;
//   4. c = v / (a~^H v), the normaliser accumulated in FP64 (a~^H v is
//      a~^H R^-1 a~; dividing by it makes c^H a~ = 1 exactly up to rounding).
// A pair whose FP32 factorisation fails, or whose pivot ratio
// (max L_ii / min L_ii)^2 exceeds kappa_max, is solved again entirely in
// FP64 (info = -2).  Non-finite input: info = -1, c = NaN.  FP64 pivot k
// not positive: info = k + 1, c = NaN.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace bs {

constexpr int WMAX = 16;
constexpr int SOLVE_PAIRS_PER_CTA = 8;

__device__ __forceinline__ float2 conjmul(float2 l, float2 v) {   // conj(l) * v
    return make_float2(l.x * v.x + l.y * v.y, l.x * v.y - l.y * v.x);
}
__device__ __forceinline__ double2 dcmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dcmulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 dconjmul(double2 l, double2 v) {  // conj(l) * v
    return make_double2(l.x * v.x + l.y * v.y, l.x * v.y - l.y * v.x);
}
__device__ __forceinline__ float2 shfl2(unsigned mask, float2 v, int src) {
    return make_float2(__shfl_sync(mask, v.x, src, 16), __shfl_sync(mask, v.y, src, 16));
}
__device__ __forceinline__ double2 shfl2d(unsigned mask, double2 v, int src) {
    return make_double2(__shfl_sync(mask, v.x, src, 16), __shfl_sync(mask, v.y, src, 16));
}

// FP32 triangular solves with the factor held as rows (A, diag) and its
// transpose in Ls: returns v = L^-H L^-1 b and (optionally) |L^-1 b|^2.
__device__ __forceinline__ float2 chol_solve_f32(unsigned mask, int lane, int W, const float2 (&A)[WMAX],
                                                 float diag, const float2 (*Ls)[WMAX + 1], float2 b) {
    float2 acc = b, u = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < WMAX; ++j) {
        if (j < W) {
            const float2 mine = (lane == j) ? cscale(acc, 1.0f / diag) : make_float2(0.f, 0.f);
            const float2 uj = shfl2(mask, mine, j);
            if (lane == j) u = uj;
            if (lane > j) acc = csub(acc, cmul(A[j], uj));
        }
    }
    acc = u;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = WMAX - 1; j >= 0; --j) {
        if (j < W) {
            const float2 mine = (lane == j) ? cscale(acc, 1.0f / diag) : make_float2(0.f, 0.f);
            const float2 vj = shfl2(mask, mine, j);
            if (lane == j) v = vj;
            if (lane < j) acc = csub(acc, conjmul(Ls[j][lane], vj));
        }
    }
    return v;
}

__device__ __forceinline__ double hw_sum(unsigned mask, double x) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, 16);
    return x;
}
__device__ __forceinline__ float hw_sumf(unsigned mask, float x) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, 16);
    return x;
}

// Whole solve in FP64 for one pair (escalation path).  Returns 0 or pivot+1.
__device__ int solve_f64(unsigned mask, int lane, int W, const double2 *__restrict__ Rg,
                         double2 a, double2 (*Ld)[WMAX + 1], double2 &c_out) {
    double2 D[WMAX];
    const bool row = lane < W;
#pragma unroll
    for (int j = 0; j < WMAX; ++j) D[j] = (row && j < W) ? Rg[lane * W + j] : make_double2(0.0, 0.0);
    int fail = 0;
    double diag = 1.0;
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        if (k < W) {
            const double dkk = __shfl_sync(mask, D[k].x, k, 16);
            if (!(dkk > 0.0) && fail == 0) fail = k + 1;
            const double pk = sqrt(dkk > 0.0 ? dkk : 1.0);
            const double inv = 1.0 / pk;
            if (lane > k) D[k] = make_double2(D[k].x * inv, D[k].y * inv);
            if (lane == k) { D[k] = make_double2(pk, 0.0); diag = pk; }
#pragma unroll
            for (int j = k + 1; j < WMAX; ++j) {
                if (j < W) {
                    const double2 ljk = shfl2d(mask, D[k], j);
                    if (lane >= j) {
                        const double2 t = dcmulc(D[k], ljk);
                        D[j] = make_double2(D[j].x - t.x, D[j].y - t.y);
                    }
                }
            }
        }
    }
    if (fail) return fail;
#pragma unroll
    for (int j = 0; j < WMAX; ++j)
        if (row && j <= lane) Ld[lane][j] = D[j];
    __syncwarp(mask);
    double2 acc = a, u = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < WMAX; ++j) {
        if (j < W) {
            const double2 mine = (lane == j) ? make_double2(acc.x / diag, acc.y / diag) : make_double2(0.0, 0.0);
            const double2 uj = shfl2d(mask, mine, j);
            if (lane == j) u = uj;
            if (lane > j) {
                const double2 t = dcmul(D[j], uj);
                acc = make_double2(acc.x - t.x, acc.y - t.y);
            }
        }
    }
    acc = u;
    double2 v = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = WMAX - 1; j >= 0; --j) {
        if (j < W) {
            const double2 mine = (lane == j) ? make_double2(acc.x / diag, acc.y / diag) : make_double2(0.0, 0.0);
            const double2 vj = shfl2d(mask, mine, j);
            if (lane == j) v = vj;
            if (lane < j) {
                const double2 t = dconjmul(Ld[j][lane], vj);
                acc = make_double2(acc.x - t.x, acc.y - t.y);
            }
        }
    }
    // s = a^H v
    const double2 av = dconjmul(a, v);
    const double sr = hw_sum(mask, row ? av.x : 0.0), si = hw_sum(mask, row ? av.y : 0.0);
    const double den = sr * sr + si * si;
    // v / s = v conj(s) / |s|^2
    c_out = make_double2((v.x * sr + v.y * si) / den, (v.y * sr - v.x * si) / den);
    return 0;
}

__global__ void __launch_bounds__(SOLVE_PAIRS_PER_CTA * 16)
    mvdr_solve_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                      const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                      const float2 *__restrict__ at32, const double2 *__restrict__ at64,
                      float2 *__restrict__ c, int32_t *__restrict__ info, int64_t pairs,
                      double kappa_max, int refine, int allow_f64) {
    // per half-warp scratch for the transposed factor: FP32 (Ls) on the
    // normal path, FP64 (Ld) on the escalation path; a half-warp uses one.
    __shared__ double2 scratch[SOLVE_PAIRS_PER_CTA][WMAX][WMAX + 1];
    const int hw = threadIdx.x >> 4;
    float2(*Lsf)[WMAX + 1] = reinterpret_cast<float2(*)[WMAX + 1]>(&scratch[hw][0][0]);
    double2(*Ldd)[WMAX + 1] = scratch[hw];
    const int lane = threadIdx.x & 15;
    const unsigned mask = (threadIdx.x & 16) ? 0xFFFF0000u : 0x0000FFFFu;
    const int64_t g = (int64_t)blockIdx.x * SOLVE_PAIRS_PER_CTA + hw;
    if (g >= pairs) return;   // uniform over the half-warp
    const int W = Wg[g];
    const double2 *Rg = R + roff[g];
    const int64_t wo = woff[g];
    const bool row = lane < W;

    float2 A[WMAX];
    bool finite = true;
#pragma unroll
    for (int j = 0; j < WMAX; ++j) {
        const double2 r = (row && j < W) ? Rg[lane * W + j] : make_double2(0.0, 0.0);
        finite = finite && isfinite(r.x) && isfinite(r.y);
        A[j] = make_float2((float)r.x, (float)r.y);
    }
    const double2 a64 = row ? at64[wo + lane] : make_double2(0.0, 0.0);
    finite = finite && isfinite(a64.x) && isfinite(a64.y);
    if (!__all_sync(mask, finite)) {
        if (row) c[wo + lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) info[g] = -1;
        return;
    }

    // 1. FP32 Cholesky
    int fail = 0;
    float diag = 1.f, dmax = 0.f, dmin = INFINITY;
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        if (k < W) {
            const float dkk = __shfl_sync(mask, A[k].x, k, 16);
            if (!(dkk > 0.f) && fail == 0) fail = k + 1;
            const float pk = sqrtf(dkk > 0.f ? dkk : 1.f);
            const float inv = 1.f / pk;
            dmax = fmaxf(dmax, pk);
            dmin = fminf(dmin, pk);
            if (lane > k) A[k] = cscale(A[k], inv);
            if (lane == k) { A[k] = make_float2(pk, 0.f); diag = pk; }
#pragma unroll
            for (int j = k + 1; j < WMAX; ++j) {
                if (j < W) {
                    const float2 ljk = shfl2(mask, A[k], j);
                    if (lane >= j) A[j] = csub(A[j], cmulc(A[k], ljk));
                }
            }
        }
    }
    const double ratio = (double)dmax / (double)dmin;
    const bool escalate = allow_f64 && (fail != 0 || ratio * ratio > kappa_max);
    if (!escalate && fail == 0) {
#pragma unroll
        for (int j = 0; j < WMAX; ++j)
            if (row && j <= lane) Lsf[lane][j] = A[j];
        __syncwarp(mask);
        const float2 a32 = row ? at32[wo + lane] : make_float2(0.f, 0.f);
        // 2. solve in FP32
        float2 v = chol_solve_f32(mask, lane, W, A, diag, Lsf, a32);
        double2 vd = make_double2((double)v.x, (double)v.y);
        // 3. refinement with an FP64 residual
        if (refine) {
            double2 r = a64;
#pragma unroll
            for (int j = 0; j < WMAX; ++j) {
                if (j < W) {
                    const double2 vj = shfl2d(mask, vd, j);
                    if (row) {
                        const double2 t = dcmul(Rg[lane * W + j], vj);
                        r = make_double2(r.x - t.x, r.y - t.y);
                    }
                }
            }
            const float2 dv = chol_solve_f32(mask, lane, W, A, diag, Lsf,
                                             make_float2((float)r.x, (float)r.y));
            vd = make_double2(vd.x + (double)dv.x, vd.y + (double)dv.y);
        }
        // 4. c = v / (a~^H v)
        const double2 av = dconjmul(a64, vd);
        const double sr = hw_sum(mask, row ? av.x : 0.0), si = hw_sum(mask, row ? av.y : 0.0);
        const double den = sr * sr + si * si;
        if (row)
            c[wo + lane] = make_float2((float)((vd.x * sr + vd.y * si) / den),
                                       (float)((vd.y * sr - vd.x * si) / den));
        if (lane == 0) info[g] = 0;
        return;
    }
    if (!escalate) {   // FP32 failure and escalation disabled
        if (row) c[wo + lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) info[g] = fail;
        return;
    }
    double2 cd;
    const int f64fail = solve_f64(mask, lane, W, Rg, a64, Ldd, cd);
    if (f64fail) {
        if (row) c[wo + lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) info[g] = f64fail;
        return;
    }
    if (row) c[wo + lane] = make_float2((float)cd.x, (float)cd.y);
    if (lane == 0) info[g] = -2;
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

bs_status launch_mvdr_solve(const bs_plan *p, const double2 *R, float2 *c, int32_t *info, cudaStream_t st) {
    const int64_t G = p->pairs;
    if (p->Wmax > WMAX) return set_error(BS_EUNSUPPORTED, "W > 16");
    if (p->cfg.flags & BS_FLAG_PLAIN) {
        plain_solve_kernel<<<(unsigned)G, 32, 0, st>>>(R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, c, info);
        return check_launch("plain solve launch");
    }
    const unsigned blocks = (unsigned)((G + SOLVE_PAIRS_PER_CTA - 1) / SOLVE_PAIRS_PER_CTA);
    mvdr_solve_kernel<<<blocks, SOLVE_PAIRS_PER_CTA * 16, 0, st>>>(
        R, p->d_roff, p->d_Wg, p->d_woff, p->d_at32, p->d_at64, c, info, G, p->cfg.kappa_max,
        (p->cfg.flags & BS_FLAG_NO_REFINE) ? 0 : 1, (p->cfg.flags & BS_FLAG_NO_FP64) ? 0 : 1);
    return check_launch("solve launch");
}

}  // namespace bs
