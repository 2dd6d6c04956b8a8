// Device helpers shared by the kernels: complex arithmetic, in-register
// power-of-two DFTs and the Stockham pass used by both FFT stages.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bs {

// Complex sums as one packed FP32x2 instruction (sm_100 and later): the same
// round-to-nearest result per component as two scalar adds, in half the
// issue slots, which the FFT kernels (issue-bound) are short of.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

// x * exp(-2 pi i e / 16); e is a compile-time constant at every call site
// (fully unrolled loops), so the switch folds to a few instructions.
__device__ __forceinline__ float2 twiddle16(int e, float2 x) {
    constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
    constexpr float H = 0.70710678118654752f;   // sqrt(1/2)
    float c, s;
    switch (e & 15) {
        case 0: return x;
        case 4: return make_float2(x.y, -x.x);
        case 8: return make_float2(-x.x, -x.y);
        case 12: return make_float2(-x.y, x.x);
        case 2: return make_float2((x.x + x.y) * H, (x.y - x.x) * H);
        case 6: return make_float2((x.y - x.x) * H, -(x.x + x.y) * H);
        case 10: return make_float2(-(x.x + x.y) * H, (x.x - x.y) * H);
        case 14: return make_float2((x.x - x.y) * H, (x.x + x.y) * H);
        case 1: c = C1; s = S1; break;
        case 3: c = S1; s = C1; break;
        case 5: c = -S1; s = C1; break;
        case 7: c = -C1; s = S1; break;
        case 9: c = -C1; s = -S1; break;
        case 11: c = -S1; s = -C1; break;
        case 13: c = S1; s = -C1; break;
        default: c = C1; s = -S1; break;  // 15
    }
    // x * (c - i s)
    return make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
}

// Forward DFT of R points held in registers, natural order in and out
// (radix-2 decimation in frequency, recursion resolved at compile time).
template <int R>
struct RegDFT {
    static __device__ __forceinline__ void run(float2 *v) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            e[k] = cadd(v[k], v[k + R / 2]);
            o[k] = twiddle16(k * (16 / R), csub(v[k], v[k + R / 2]));
        }
        RegDFT<R / 2>::run(e);
        RegDFT<R / 2>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            v[2 * k] = e[k];
            v[2 * k + 1] = o[k];
        }
    }
};
template <>
struct RegDFT<1> {
    static __device__ __forceinline__ void run(float2 *) {}
};

// Radix schedule of an n-point FFT (n = 2^k, 2..4096): passes of radix 16
// first, then one smaller pass for the remaining factor.
template <int n>
struct Radix {
    static constexpr int npass = (n <= 16) ? 1 : (n <= 256) ? 2 : 3;
    static constexpr int r0 = (n <= 16) ? n : 16;
    static constexpr int r1 = (npass < 2) ? 1 : (npass == 2 ? n / 16 : 16);
    static constexpr int r2 = (npass < 3) ? 1 : n / 256;
    static_assert(n >= 2 && n <= 4096 && (n & (n - 1)) == 0, "n must be a power of two <= 4096");
};

// w[r] = tw[r * e] for r < R (R = 2, 4, 8, 16; r * e < table length).
// Only w^1, w^4, w^8 and w^12 come from the table; the other powers are
// products of at most three table entries, which keeps their error within
// a few FP32 ulps while cutting the table loads per butterfly from R-1 to
// at most 4 (the loads of a warp hit scattered table lines).
template <int R>
__device__ __forceinline__ void twiddle_powers(const float2 *__restrict__ tw, int e, float2 (&w)[R]) {
    w[0] = make_float2(1.f, 0.f);
    w[1] = __ldg(&tw[e]);
    if constexpr (R >= 4) {
        w[2] = cmul(w[1], w[1]);
        w[3] = cmul(w[2], w[1]);
    }
    if constexpr (R >= 8) {
        w[4] = __ldg(&tw[4 * e]);
#pragma unroll
        for (int r = 5; r < 8; ++r) w[r] = cmul(w[4], w[r - 4]);
    }
    if constexpr (R >= 16) {
        w[8] = __ldg(&tw[8 * e]);
        w[12] = __ldg(&tw[12 * e]);
#pragma unroll
        for (int r = 9; r < 12; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
        for (int r = 13; r < 16; ++r) w[r] = cmul(w[12], w[r - 12]);
    }
}

// One Stockham autosort pass (decimation in time) of an n-point FFT over a
// batch of `ncols` independent columns, processed by `nthr` threads:
//   butterfly j < n/R of column c reads a[j + r n/R] (r < R), multiplies
//   by w^(r * (j mod Ns)) with w = e^{-2 pi i/(Ns R)}, takes the R-point DFT
//   and writes b[(j/Ns) Ns R + (j mod Ns) + r Ns].
// Ns is the product of the radices of the earlier passes.  `load(c, idx)`
// and `store(c, idx, v)` address the source and destination; with
// kSyncMid the pass reads everything into registers, synchronises the CTA
// and then writes (in-place passes through shared memory).
// kColFast: butterfly id -> (column = id % ncols) else (column = id / (n/R)).
// tw[k] = e^{-2 pi i k / n}, k < n.
template <int n, int R, int Ns, int ncols, int nthr, bool kColFast, bool kSyncMid,
          class Load, class Store>
__device__ __forceinline__ void stockham_pass(int tid, const float2 *__restrict__ tw, Load load,
                                              Store store) {
    constexpr int nb = ncols * (n / R);
    static_assert(nb % nthr == 0, "butterflies must divide evenly over threads");
    constexpr int bpt = nb / nthr;
    float2 v[bpt][R];
#pragma unroll
    for (int b = 0; b < bpt; ++b) {
        const int id = tid + b * nthr;
        const int c = kColFast ? (id % ncols) : (id / (n / R));
        const int j = kColFast ? (id / ncols) : (id % (n / R));
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = load(c, j + r * (n / R));
        if (Ns > 1) {
            float2 w[R];
            twiddle_powers<R>(tw, (j % Ns) * (n / (Ns * R)), w);
#pragma unroll
            for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
        }
        RegDFT<R>::run(v[b]);
    }
    if (kSyncMid) __syncthreads();
#pragma unroll
    for (int b = 0; b < bpt; ++b) {
        const int id = tid + b * nthr;
        const int c = kColFast ? (id % ncols) : (id / (n / R));
        const int j = kColFast ? (id / ncols) : (id % (n / R));
        const int k = j % Ns;
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) store(c, base + r * Ns, v[b][r]);
    }
}

// Double-float values (h + l, |l| <= ulp(h)/2): GB300's FP64 pipe is
// narrow, so the covariance epilogues assemble R in FP32 pairs and convert
// only the final value of each entry to FP64.
struct DF {
    float h, l;
};
__device__ __forceinline__ DF df_norm(float h, float l) {   // |l| small against h
    const float s = h + l;
    return DF{s, l - (s - h)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
    return df_norm(s, e);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_norm(p, e);
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.h + (double)a.l; }
// host side: a double as a double-float (for kernel parameters)
inline DF df_from_double(double v) {
    const float h = (float)v;
    return DF{h, (float)(v - (double)h)};
}

// Padded shared-memory row index: one spare slot every 16 rows spreads the
// radix-16 strided accesses over the banks.
__device__ __forceinline__ int padrow(int t) { return t + (t >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 16; }

}  // namespace bs
