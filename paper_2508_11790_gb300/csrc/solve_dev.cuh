// Half-warp batched Cholesky MVDR solve of one (target, subband) pair,
// shared by the stand-alone solve kernel and the fused persistent kernel.
//
// Eq. BeamCorrMVDR: c = R^-1 a~ / (a~^H R^-1 a~).  Lane i of the half-warp
// holds row i of R (W <= 16).
//   1. R = L L^H in FP32 (right-looking; column k broadcast by shuffles);
//   2. u = L^-1 a~, v = L^-H u (triangular solves, one shuffle per step;
//      the backward solve reads L transposed from shared memory);
//   3. one refinement step: r = a~ - R v formed with error-free FP32
//      transformations from the double-float (hi + lo) parts of R and a~
//      (about twice FP32 precision, at FP32 speed: FP64 is a small
//      fraction of FP32 throughput on this part), v += L^-H L^-1 r;
//   4. c = v / (a~^H v) (a~^H v is a~^H R^-1 a~; dividing by it makes
//      c^H a~ = 1 up to rounding).
// A pair whose FP32 factorisation fails, or whose pivot ratio
// (max L_ii / min L_ii)^2 exceeds kappa_max, is solved again entirely in
// FP64 (info = -2).  Non-finite input: info = -1, c = NaN.  FP64 pivot k
// not positive: info = k + 1, c = NaN.
//
// Optional diagonal preconditioner d (the learned seed): with D = diag(2^e),
// e_i the exponent of d_i rounded to the nearest power of two, the solve
// runs on D R D and D a and returns c = D y / (a^H D y) -- the same c in
// exact arithmetic, and every scaling is exact (powers of two), so only
// the conditioning that the Cholesky sees (and the escalation test) change.
#pragma once
#include <math.h>

#include "common.cuh"

namespace bs {

constexpr int WMAX = 16;        // half-warp solve: W <= 16
constexpr int WMAX_WIDE = 32;   // whole-warp solve: 16 < W <= 32

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
// GW: lanes of the group that solves one pair (16: a half-warp for W <= 16;
// 32: a whole warp for 16 < W <= 32).
template <int GW = 16>
__device__ __forceinline__ float2 shfl2(unsigned mask, float2 v, int src) {
    return make_float2(__shfl_sync(mask, v.x, src, GW), __shfl_sync(mask, v.y, src, GW));
}
template <int GW = 16>
__device__ __forceinline__ double2 shfl2d(unsigned mask, double2 v, int src) {
    return make_double2(__shfl_sync(mask, v.x, src, GW), __shfl_sync(mask, v.y, src, GW));
}

// FP32 triangular solves with the factor held as rows (A, diag) and its
// transpose in Ls: returns v = L^-H L^-1 b.  WT = window size.
template <int WT, int GW = 16>
__device__ __forceinline__ float2 chol_solve_f32(unsigned mask, int lane, const float2 (&A)[WT], float diag,
                                                 const float2 (*Ls)[GW + 1], float2 b) {
    const float rdiag = 1.0f / diag;
    float2 acc = b, u = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < WT; ++j) {
        const float2 mine = (lane == j) ? cscale(acc, rdiag) : make_float2(0.f, 0.f);
        const float2 uj = shfl2<GW>(mask, mine, j);
        if (lane == j) u = uj;
        if (lane > j) acc = csub(acc, cmul(A[j], uj));
    }
    acc = u;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = WT - 1; j >= 0; --j) {
        const float2 mine = (lane == j) ? cscale(acc, rdiag) : make_float2(0.f, 0.f);
        const float2 vj = shfl2<GW>(mask, mine, j);
        if (lane == j) v = vj;
        if (lane < j) acc = csub(acc, conjmul(Ls[j][lane], vj));
    }
    return v;
}

template <int GW = 16>
__device__ __forceinline__ double hw_sum(unsigned mask, double x) {
#pragma unroll
    for (int o = GW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, GW);
    return x;
}
template <int GW = 16>
__device__ __forceinline__ float hw_sumf(unsigned mask, float x) {
#pragma unroll
    for (int o = GW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, GW);
    return x;
}

// Whole solve in FP64 for one pair (escalation path), row `lane` of R given
// in D.  Returns 0 or pivot+1.
template <int GW = 16>
static __device__ __forceinline__ int solve_f64_rows(unsigned mask, int lane, int W, double2 (&D)[GW], double2 a,
                                     double2 (*Ld)[GW + 1], double2 &c_out) {
    const bool row = lane < W;
#pragma unroll
    for (int j = 0; j < GW; ++j)
        if (!(row && j < W)) D[j] = make_double2(0.0, 0.0);
    int fail = 0;
    double diag = 1.0;
#pragma unroll
    for (int k = 0; k < GW; ++k) {
        if (k < W) {
            const double dkk = __shfl_sync(mask, D[k].x, k, GW);
            if (!(dkk > 0.0) && fail == 0) fail = k + 1;
            const double inv = rsqrt(dkk > 0.0 ? dkk : 1.0);   // one sequence instead of sqrt and a division
            const double pk = (dkk > 0.0 ? dkk : 1.0) * inv;
            if (lane > k) D[k] = make_double2(D[k].x * inv, D[k].y * inv);
            if (lane == k) { D[k] = make_double2(pk, 0.0); diag = pk; }
#pragma unroll
            for (int j = k + 1; j < GW; ++j) {
                if (j < W) {
                    const double2 ljk = shfl2d<GW>(mask, D[k], j);
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
    for (int j = 0; j < GW; ++j)
        if (row && j <= lane) Ld[lane][j] = D[j];
    __syncwarp(mask);
    // one FP64 division per lane: GB300's FP64 pipe is narrow and a division
    // is a long sequence on it (two per step of each solve before)
    const double rdiag = 1.0 / diag;
    double2 acc = a, u = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < GW; ++j) {
        if (j < W) {
            const double2 mine = (lane == j) ? make_double2(acc.x * rdiag, acc.y * rdiag) : make_double2(0.0, 0.0);
            const double2 uj = shfl2d<GW>(mask, mine, j);
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
    for (int j = GW - 1; j >= 0; --j) {
        if (j < W) {
            const double2 mine = (lane == j) ? make_double2(acc.x * rdiag, acc.y * rdiag) : make_double2(0.0, 0.0);
            const double2 vj = shfl2d<GW>(mask, mine, j);
            if (lane == j) v = vj;
            if (lane < j) {
                const double2 t = dconjmul(Ld[j][lane], vj);
                acc = make_double2(acc.x - t.x, acc.y - t.y);
            }
        }
    }
    // s = a^H v
    const double2 av = dconjmul(a, v);
    const double sr = hw_sum<GW>(mask, row ? av.x : 0.0), si = hw_sum<GW>(mask, row ? av.y : 0.0);
    const double rden = 1.0 / (sr * sr + si * si);
    // v / s = v conj(s) / |s|^2
    c_out = make_double2((v.x * sr + v.y * si) * rden, (v.y * sr - v.x * si) * rden);
    return 0;
}

// Exponent of the power of two nearest to d in log scale, clamped to
// [-30, 30]; 0 for non-positive or non-finite d (no scaling).
__device__ __forceinline__ int precond_exp(float d) {
    if (!(d > 0.f) || !isfinite(d)) return 0;
    const unsigned b = __float_as_uint(d);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    if (e == -127) return -30;                       // subnormal: as small as allowed
    if ((b & 0x7FFFFFu) >= 0x3504F3u) e += 1;        // mantissa >= sqrt(2): round up
    return e < -30 ? -30 : (e > 30 ? 30 : e);
}
// 2^e as a float, -126 <= e <= 127
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// Not inlined: compiled once per translation unit for every window size.
// ex: the lane's preconditioner exponent (0 without one); row j scales by
// 2^(ex_lane + ex_j), exactly.
template <int GW = 16>
static __device__ __noinline__ int solve_f64(unsigned mask, int lane, int W, const double2 *__restrict__ Rg, double2 a,
                                double2 (*Ld)[GW + 1], double2 &c_out, int ex) {
    double2 D[GW];
    const bool row = lane < W;
#pragma unroll
    for (int j = 0; j < GW; ++j) {
        const int ej = __shfl_sync(mask, ex, j, GW);
        const double s = (double)pow2f(ex + ej);
        const double2 r = (row && j < W) ? Rg[lane * W + j] : make_double2(0.0, 0.0);
        D[j] = make_double2(r.x * s, r.y * s);
    }
    const double si = (double)pow2f(ex);
    const int f = solve_f64_rows<GW>(mask, lane, W, D, make_double2(a.x * si, a.y * si), Ld, c_out);
    c_out = make_double2(c_out.x * si, c_out.y * si);
    return f;
}

// Error-free transformations (FP32): a*b = p + e exactly (FMA), a + b = s + t.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = a + b;
    const float bb = s - a;
    t = (a - (s - bb)) + (b - bb);
}

// Compensated residual r = a - R v for one row (Dot2-style): R = Rh + Rl and
// a = ah + al are double-float, v is FP32; products of the high parts are
// split exactly into value + error and summed with two-sum, so r carries
// about twice the FP32 precision (the refinement then converges like one
// with an FP64 residual).
template <int WT, int GW, class Rows>
__device__ __forceinline__ float2 residual_df(unsigned mask, int lane, Rows rows, float2 ah, float2 al, float2 v) {
    float sr = ah.x, si = ah.y, cr = al.x, ci = al.y;
    const bool row = lane < WT;
#pragma unroll
    for (int j = 0; j < WT; ++j) {
        const float2 vj = shfl2<GW>(mask, v, j);
        const float4 r4 = row ? rows(j) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 Rh = make_float2(r4.x, r4.y), Rl = make_float2(r4.z, r4.w);
        float p1, e1, p2, e2, p3, e3, p4, e4, t;
        two_prod(Rh.x, vj.x, p1, e1);   // re += -(Rh.re v.re) + (Rh.im v.im)
        two_prod(Rh.y, vj.y, p2, e2);
        two_prod(Rh.x, vj.y, p3, e3);   // im += -(Rh.re v.im) - (Rh.im v.re)
        two_prod(Rh.y, vj.x, p4, e4);
        two_sum(sr, -p1, sr, t); cr += t - e1;
        two_sum(sr, p2, sr, t);  cr += t + e2;
        two_sum(si, -p3, si, t); ci += t - e3;
        two_sum(si, -p4, si, t); ci += t - e4;
        cr -= Rl.x * vj.x - Rl.y * vj.y;
        ci -= Rl.x * vj.y + Rl.y * vj.x;
    }
    return make_float2(sr + cr, si + ci);
}

// Split a double into FP32 parts hi + lo (hi: the double rounded half-up to
// 24 significant bits, lo: the rest rounded to FP32) with integer operations
// only: GB300's FP64 pipe is narrow, and the conversions this replaces
// ((float)d, d - (double)hi, (float)(...)) all ran on it.  Non-finite input
// and magnitudes at or above 2^128 give an infinite or NaN hi; magnitudes
// below 2^-126 give zero.
__device__ __forceinline__ float2 split_f64(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sign = hw & 0x80000000u;
    const int e11 = (int)((hw >> 20) & 0x7FFu);
    if (e11 == 0x7FF) return make_float2(__uint_as_float(sign | 0x7F800000u | (((hw & 0xFFFFFu) | lw) ? 0x400000u : 0u)), 0.f);
    const int e8 = e11 - 896;   // FP32 biased exponent
    if (e8 <= 0) return make_float2(0.f, 0.f);
    if (e8 >= 255) return make_float2(__uint_as_float(sign | 0x7F800000u), 0.f);
    const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const unsigned rest = lw & 0x1FFFFFFFu;   // 29 mantissa bits below hi
    const unsigned up = rest >> 28;
    const unsigned hb = (sign | ((unsigned)e8 << 23) | m23) + up;   // a carry moves into the exponent
    const int lo_int = (int)rest - (int)(up << 29);               // d - hi in units of 2^(e11 - 1075)
    const int el = e11 - 948;                                       // FP32 biased exponent of 2^(e11 - 1075)
    const float lo = (el >= 1) ? (float)lo_int * __uint_as_float((unsigned)el << 23) : 0.f;
    return make_float2(__uint_as_float(hb), sign ? -lo : lo);
}

// Solve one pair of window size WT with the calling half-warp (lanes 0..15
// of `mask`).  Rg: its W x W covariance in FP64 (row-major; global or shared
// memory), read as FP32 (hi, lo) parts; a32/alo: the windowed steering
// vector as hi / lo FP32 parts, a64 in FP64 (escalation).  scratch: [16][17]
// double2 per half-warp.  Writes c[0..W) and *info.  Not inlined, so each
// window size is compiled once per translation unit.
template <int WT, int GW = 16>
__device__ __forceinline__ void solve_pair_body(unsigned mask, int lane, const double2 *Rg,
                                                     const float2 *__restrict__ a32g,
                                                     const float2 *__restrict__ alog,
                                                     const double2 *__restrict__ a64g, float2 *__restrict__ c,
                                                     int32_t *__restrict__ info, double kappa_max, int refine,
                                                     int allow_f64, double2 (*scratch)[GW + 1],
                                                     const float *__restrict__ dg) {
    const int ex = (dg && lane < WT) ? precond_exp(dg[lane]) : 0;   // this row's scaling exponent
    int exj[WT];                                                     // every column's
#pragma unroll
    for (int j = 0; j < WT; ++j) exj[j] = __shfl_sync(mask, ex, j, GW);
    auto rows = [&](int j) -> float4 {
        const double2 r = Rg[lane * WT + j];
        const float2 x = split_f64(r.x), y = split_f64(r.y);
        const float s = pow2f(ex + exj[j]);   // exact: a power of two
        return make_float4(x.x * s, y.x * s, x.y * s, y.y * s);
    };
    float2(*Lsf)[GW + 1] = reinterpret_cast<float2(*)[GW + 1]>(&scratch[0][0]);
    constexpr int W = WT;
    const bool row = lane < W;

    // Up to kKeepRow entries the lane's split row stays in registers for the
    // refinement residual (else it is read and split again there).
    constexpr int kKeepRow = 10;
    constexpr int NK = (WT <= kKeepRow) ? WT : 1;
    float4 Rrow[NK];
    float2 A[WT];
    bool finite = true;
#pragma unroll
    for (int j = 0; j < WT; ++j) {
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row) r = rows(j);
        finite = finite && isfinite(r.x) && isfinite(r.y);
        A[j] = make_float2(r.x, r.y);
        if constexpr (WT <= kKeepRow) Rrow[j] = r;
    }
    const float sa = pow2f(ex);
    const float2 ah = row ? cscale(a32g[lane], sa) : make_float2(0.f, 0.f);
    const float2 al = row ? cscale(alog[lane], sa) : make_float2(0.f, 0.f);
    finite = finite && isfinite(ah.x) && isfinite(ah.y);
    if (!__all_sync(mask, finite)) {
        if (row) c[lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) *info = -1;
        return;
    }

    // 1. FP32 Cholesky
    int fail = 0;
    float diag = 1.f, dmax = 0.f, dmin = INFINITY;
#pragma unroll
    for (int k = 0; k < WT; ++k) {
        const float dkk = __shfl_sync(mask, A[k].x, k, GW);
        if (!(dkk > 0.f) && fail == 0) fail = k + 1;
        const float inv = rsqrtf(dkk > 0.f ? dkk : 1.f);   // the refinement step absorbs its last-bit error
        const float pk = (dkk > 0.f ? dkk : 1.f) * inv;
        dmax = fmaxf(dmax, pk);
        dmin = fminf(dmin, pk);
        if (lane > k) A[k] = cscale(A[k], inv);
        if (lane == k) { A[k] = make_float2(pk, 0.f); diag = pk; }
#pragma unroll
        for (int j = k + 1; j < WT; ++j) {
            const float2 ljk = shfl2<GW>(mask, A[k], j);
            if (lane >= j) A[j] = csub(A[j], cmulc(A[k], ljk));
        }
    }
    const float ratio = dmax / dmin;
    const bool escalate = allow_f64 && (fail != 0 || ratio * ratio > (float)kappa_max);
    if (!escalate && fail == 0) {
#pragma unroll
        for (int j = 0; j < WT; ++j)
            if (row && j <= lane) Lsf[lane][j] = A[j];
        __syncwarp(mask);
        // 2. solve in FP32
        float2 v = chol_solve_f32<WT, GW>(mask, lane, A, diag, Lsf, ah);
        // 3. refinement with a compensated (double-float) residual
        if (refine) {
            float2 r;
            if constexpr (WT <= kKeepRow) r = residual_df<WT, GW>(mask, lane, [&](int j) { return Rrow[j]; }, ah, al, v);
            else r = residual_df<WT, GW>(mask, lane, rows, ah, al, v);
            const float2 dv = chol_solve_f32<WT, GW>(mask, lane, A, diag, Lsf, r);
            v = cadd(v, dv);
        }
        // 4. c = v / (a~^H v)
        const float2 av = row ? conjmul(ah, v) : make_float2(0.f, 0.f);
        const float sr = hw_sumf<GW>(mask, av.x), si = hw_sumf<GW>(mask, av.y);
        const float inv = sa / (sr * sr + si * si);   // c = D y / (b^H y), b = D a
        if (row) c[lane] = make_float2((v.x * sr + v.y * si) * inv, (v.y * sr - v.x * si) * inv);
        if (lane == 0) *info = 0;
        return;
    }
    if (!escalate) {   // FP32 failure and escalation disabled
        if (row) c[lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) *info = fail;
        return;
    }
    // FP64 path
    double2(*Ldd)[GW + 1] = scratch;
    __syncwarp(mask);
    double2 cd;
    const double2 a64 = row ? a64g[lane] : make_double2(0.0, 0.0);
    const int f64fail = solve_f64<GW>(mask, lane, W, Rg, a64, Ldd, cd, ex);
    if (f64fail) {
        if (row) c[lane] = make_float2(nanf(""), nanf(""));
        if (lane == 0) *info = f64fail;
        return;
    }
    if (row) c[lane] = make_float2((float)cd.x, (float)cd.y);
    if (lane == 0) *info = -2;
}

// The same solve as a separate function per window size (the fused and
// whole-warp kernels call it: one copy of the body per W and translation
// unit, and their own registers stay free of it).
template <int WT, int GW = 16>
static __device__ __noinline__ void solve_pair_fixed(unsigned mask, int lane, const double2 *Rg,
                                                     const float2 *__restrict__ a32g,
                                                     const float2 *__restrict__ alog,
                                                     const double2 *__restrict__ a64g, float2 *__restrict__ c,
                                                     int32_t *__restrict__ info, double kappa_max, int refine,
                                                     int allow_f64, double2 (*scratch)[GW + 1],
                                                     const float *__restrict__ dg) {
    solve_pair_body<WT, GW>(mask, lane, Rg, a32g, alog, a64g, c, info, kappa_max, refine, allow_f64, scratch, dg);
}

// R stored as FP64 (global or shared memory); dispatches on W to the solve
// compiled for that window size.
__device__ __forceinline__ void solve_pair(unsigned mask, int lane, int W, const double2 *Rg,
                                           const float2 *__restrict__ a32g, const float2 *__restrict__ alog,
                                           const double2 *__restrict__ a64g, float2 *__restrict__ c,
                                           int32_t *__restrict__ info, double kappa_max, int refine,
                                           int allow_f64, double2 (*scratch)[WMAX + 1],
                                           const float *__restrict__ dg = nullptr) {
#define BS_SOLVE_CASE(n) \
    case n: solve_pair_fixed<n>(mask, lane, Rg, a32g, alog, a64g, c, info, kappa_max, refine, allow_f64, scratch, dg); break;
    switch (W) {
        BS_SOLVE_CASE(1) BS_SOLVE_CASE(2) BS_SOLVE_CASE(3) BS_SOLVE_CASE(4)
        BS_SOLVE_CASE(5) BS_SOLVE_CASE(6) BS_SOLVE_CASE(7) BS_SOLVE_CASE(8)
        BS_SOLVE_CASE(9) BS_SOLVE_CASE(10) BS_SOLVE_CASE(11) BS_SOLVE_CASE(12)
        BS_SOLVE_CASE(13) BS_SOLVE_CASE(14) BS_SOLVE_CASE(15) default: BS_SOLVE_CASE(16)
    }
#undef BS_SOLVE_CASE
}

}  // namespace bs
