// Tensor-core beamspace kernel for N = 1024 elements and M = 2048 beams
// (Eq. VerDFT, Eq. BeamTransform, Eq. OverallWindow, Eq. ApplyWindow).
//
// Same result as the other beamspace kernels: every (record, bin) vector
// zero-padded to M points, its M-point DFT scaled by 1/sqrt(M), and the W_t
// beams start_g + w (mod M) of every target written to the packed window
// arrays.  With n = 16 n1 + n2 (n1 < 64, n2 < 16) and beams m = k + 128 m2
// (k < 128, m2 < 16):
//
//   X[k + 128 m2] = sum_n2 W_16^(n2 m2) W_M^(n2 k) Y[k][n2],
//   Y[k][n2]      = sum_n1 W_128^(n1 k) x[16 n1 + n2].
//
// Y is a complex (128 x 64) x (64 x 16 per vector) matrix product and runs
// on the tensor cores: tcgen05.mma, FP16 operands, FP32 accumulators in
// tensor memory, four vectors (N = 64 columns) per product.  FP32 accuracy
// comes from splitting both operands into FP16 high and low parts and
// summing hi*hi + hi*lo + lo*hi (the dropped lo*lo term is 2^-22 of the
// product); every vector is scaled by the power of two that brings its
// largest component into [2^13, 2^14), so both parts of the data stay in
// FP16's normal range whatever the input scale.  The DFT matrix (its real
// and imaginary parts, high and low) is the A
// operand and lives in tensor memory for the whole kernel; the vectors are
// the B operand, staged in shared memory in the canonical K-major layout.
//
// The twiddles W_M^(n2 k) and the 16-point DFTs along n2 run on the CUDA
// cores: epilogue thread k reads row k of the accumulators (its tensor-memory
// lane) for two vectors at once and keeps them as structure-of-arrays pairs,
// so that every butterfly of the 16-point DFT is one packed FP32x2
// instruction for both vectors.  The beams go to shared memory, and all
// threads then store the windows.
//
// One CTA per SM, 13 warps: warps 0-7 are two epilogue groups (warp w reads
// tensor-memory lanes 32 (w mod 4) .. + 31 of the tiles of parity w / 4,
// one vector pair at a time, and stores the pair's windows), warps 8-11 scale and split one vector each
// of the tile after next (each vector arrives by one bulk copy, issued a
// tile ahead) and write the per-target gather entries of the current tile,
// and warp 12 issues the products.  The roles hand work over through
// mbarriers only (stage written, accumulator read, products done, entries
// written, windows stored), and an epilogue group meets only itself at a
// named barrier, so one group's stores overlap the other's arithmetic and
// the MMA warp's waits on the tensor pipe stall nobody else.
// Three accumulators and two B stages let the tensor cores work on the
// next tiles while the CUDA cores finish the current ones.  Every wait on an
// mbarrier is bounded; a wait that gives up sets bit 0 of the plan's error
// word and the CTA stops after freeing its tensor memory.
#include "beamspace_dev.cuh"
#include "internal.h"
#include "tma.cuh"

#include <algorithm>

namespace bs {

namespace {

constexpr int kTcThreads = 416;   // 8 epilogue warps, 4 producer warps, 1 MMA warp
constexpr int kTcVec = 4;     // vectors per tile
constexpr int kTcN = 64;      // MMA N: 4 vectors x 16 columns n2
// shared memory (bytes)
constexpr int kSmB = 0;                          // 2 stages x {Xre_hi, Xre_lo, Xim_hi, Xim_lo}, 8 KB each
constexpr int kSmBStage = 32768;
constexpr int kSmBMat = 8192;
constexpr int kSmBeam = 2 * kSmBStage;           // 2 vector pairs x {re, im} x 2048 beams x float2
constexpr int kSmBeamPair = 2 * 2048 * 8;
constexpr int kSmTab = kSmBeam + 2 * kSmBeamPair;  // [2 tiles][2 pairs][kTabT] TabEnt
constexpr int kSmTw = kSmTab + 4 * kTabT * 8;     // [16 n2][128 k] W_M^(n2 k) (row 0 unused)
constexpr int kSmRaw = kSmTw + 16 * 128 * 8;     // [4 vectors][1024] float2: the producers' bulk-copied inputs
constexpr int kSmMisc = kSmRaw + 4 * 8192;
constexpr int kSmGlist = kSmMisc + 256;             // [sumW] gather entry list (dynamic size)
constexpr int kSmTotalMax = kSmGlist + 4 * kTabT * 32;
static_assert(kSmTotalMax <= 227 * 1024, "shared memory");
// tensor memory columns: three accumulators {Re Y [64], Im Y [64]}, then
// the A operand: ReD hi, ReD lo, ImD hi, ImD lo (32 columns of two FP16
// values each per row)
constexpr uint32_t kTmCols = 512;
constexpr int kTcAcc = 3;
constexpr uint32_t kTmA = 128 * kTcAcc;

// Gather entry of a target for one vector pair: window-array offset of the
// pair's even vector, and start | (W << 11) | (stores << 17), where stores
// (0..2) counts the vectors of the pair that have a window row (training
// rows stop at K).
struct __align__(8) TabEnt {
    int base;
    int swn;
};

struct TcArgs {
    const float2 *y;       // the launch's vectors, [nvec][1024]
    const float2 *tw;      // W_2048^e, e < 2048
    const int32_t *glist;  // [sumW]: (t << 8) | w, target-major
    int sumW;
    float store_scale;     // training windows in 16-bit precision: x store_scale
    int *err;
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, LBO = 128 bytes between core matrices
// adjacent in K, SBO = 1024 bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46);
}

// D (tensor memory) (+)= A (tensor memory) x B (shared memory), kind::f16.
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive 32-bit columns of this warp's lanes, two ranges, then wait.
__device__ __forceinline__ void tmem_ld2x32(uint32_t a0, uint32_t a1, float (&r)[32], float (&s)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, "
        "%45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
          "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]),
          "=f"(r[16]), "=f"(r[17]), "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]),
          "=f"(r[24]), "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]), "=f"(r[30]), "=f"(r[31]),
          "=f"(s[0]), "=f"(s[1]), "=f"(s[2]), "=f"(s[3]), "=f"(s[4]), "=f"(s[5]), "=f"(s[6]), "=f"(s[7]),
          "=f"(s[8]), "=f"(s[9]), "=f"(s[10]), "=f"(s[11]), "=f"(s[12]), "=f"(s[13]), "=f"(s[14]), "=f"(s[15]),
          "=f"(s[16]), "=f"(s[17]), "=f"(s[18]), "=f"(s[19]), "=f"(s[20]), "=f"(s[21]), "=f"(s[22]), "=f"(s[23]),
          "=f"(s[24]), "=f"(s[25]), "=f"(s[26]), "=f"(s[27]), "=f"(s[28]), "=f"(s[29]), "=f"(s[30]), "=f"(s[31])
        : "r"(a0), "r"(a1)
        : "memory");
}

// 32 consecutive 32-bit columns of this warp's lanes from registers, then wait.
__device__ __forceinline__ void tmem_st32(uint32_t a, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(a),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]),
        "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]),
        "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Barrier of the four epilogue warps of vector pair g (named barriers 3, 4).
__device__ __forceinline__ void group_bar(int g) {
    if (g == 0)
        asm volatile("bar.sync 3, 128;" ::: "memory");
    else
        asm volatile("bar.sync 4, 128;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t half2_bits(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// x with the low 13 mantissa bits cleared: exactly representable in FP16
// when its exponent is in FP16's normal range.
__device__ __forceinline__ float trunc_f16(float x) { return __int_as_float(__float_as_int(x) & 0xFFFFE000); }

// ------------------------------------------- 16-point DFT on vector pairs

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pmul(float2 a, float c) { return __fmul2_rn(a, make_float2(c, c)); }
__device__ __forceinline__ float2 pfma(float2 a, float c, float2 b) { return __ffma2_rn(a, make_float2(c, c), b); }

// (dr + i di) W_16^e for e = 1, 2, 3, 5, 6, 7 on structure-of-arrays pairs
// (dr, di hold the real and the imaginary parts of two values); e is a
// compile-time constant at every call site.
__device__ __forceinline__ void rot16(int e, float2 dr, float2 di, float2 &orr, float2 &oi) {
    constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
    constexpr float H = 0.70710678118654752f;   // sqrt(1/2)
    if (e == 2) {   // W^2 = H - i H
        orr = pmul(padd(dr, di), H);
        oi = pmul(psub(di, dr), H);
        return;
    }
    if (e == 6) {   // W^6 = -H - i H
        orr = pmul(psub(di, dr), H);
        oi = pmul(padd(dr, di), -H);
        return;
    }
    // W^e = c - i s, angle 2 pi e / 16
    const float c = (e == 1) ? C1 : (e == 3) ? S1 : (e == 5) ? -S1 : -C1;
    const float s = (e == 1) ? S1 : (e == 3) ? C1 : (e == 5) ? C1 : S1;
    orr = pfma(di, s, pmul(dr, c));
    oi = pfma(dr, -s, pmul(di, c));
}

// Forward DFT of R points (R | 16) held as structure-of-arrays pairs,
// natural order in and out (radix-2 decimation in frequency, recursion
// resolved at compile time): every butterfly is one packed instruction per
// part for both values of a pair.
template <int R>
struct SoaDFT {
    static __device__ __forceinline__ void run(float2 *re, float2 *im) {
        float2 er[R / 2], ei[R / 2], orr[R / 2], oi[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            er[k] = padd(re[k], re[k + R / 2]);
            ei[k] = padd(im[k], im[k + R / 2]);
            const int e = k * (16 / R);
            if (e == 0) {
                orr[k] = psub(re[k], re[k + R / 2]);
                oi[k] = psub(im[k], im[k + R / 2]);
            } else if (e == 4) {   // times -i
                orr[k] = psub(im[k], im[k + R / 2]);
                oi[k] = psub(re[k + R / 2], re[k]);
            } else {
                rot16(e, psub(re[k], re[k + R / 2]), psub(im[k], im[k + R / 2]), orr[k], oi[k]);
            }
        }
        SoaDFT<R / 2>::run(er, ei);
        SoaDFT<R / 2>::run(orr, oi);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            re[2 * k] = er[k];
            im[2 * k] = ei[k];
            re[2 * k + 1] = orr[k];
            im[2 * k + 1] = oi[k];
        }
    }
};
template <>
struct SoaDFT<1> {
    static __device__ __forceinline__ void run(float2 *, float2 *) {}
};

// ------------------------------------------------------------ producer side

// One producer warp per vector of the tile.  The vector arrives by one
// 8 KB bulk copy into the warp's own shared-memory slot; lane n2 = lane mod
// 16 then reads the 32 values n1 = 32 (lane / 16) + j of its column.
struct PrepRegs {
    float2 x[32];
};

__device__ __forceinline__ void prep_fetch(float2 *raw, uint64_t *bar, const float2 *y, int64_t vec, int lane) {
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, 8192);
        bulk_load(raw, y + vec * 1024, 8192, bar);
    }
}

__device__ __forceinline__ void prep_read(PrepRegs &r, const float2 *raw, int lane) {
    const float2 *src = raw + 16 * (32 * (lane >> 4)) + (lane & 15);
#pragma unroll
    for (int j = 0; j < 32; ++j) r.x[j] = src[16 * j];
}

// Scale the vector by 2^(13 - e) (its largest component in [2^e, 2^(e+1))),
// split it into FP16 high and low parts and store the four B matrices of
// the stage (Xre hi, Xre lo, Xim hi, Xim lo: rows c = 16 v + n2, K = n1,
// core matrices of 8 rows x 8 K).  vsc[v] receives the factor that undoes
// the scale, times `post`.
__device__ __forceinline__ void prep_store(const PrepRegs &r, uint32_t stage, float *vsc, int v, int lane,
                                           float post) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) m = fmaxf(m, fmaxf(fabsf(r.x[j].x), fabsf(r.x[j].y)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    int e = (m > 0.f) ? ((__float_as_int(m) >> 23) & 255) - 127 : 0;
    e = max(-100, min(e, 100));
    const float s = __int_as_float((127 + 13 - e) << 23);
    if (lane == 0) vsc[v] = __int_as_float((127 - 13 + e) << 23) * post;
    const int c = 16 * v + (lane & 15);
    const uint32_t row = stage + (uint32_t)((c >> 3) * 1024 + (c & 7) * 16);
#pragma unroll
    for (int blk = 0; blk < 4; ++blk) {
        const uint32_t at = row + (uint32_t)((4 * (lane >> 4) + blk) * 128);
        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const float2 a0 = __fmul2_rn(r.x[8 * blk + 2 * qq], make_float2(s, s));
            const float2 a1 = __fmul2_rn(r.x[8 * blk + 2 * qq + 1], make_float2(s, s));
            const float2 h0 = make_float2(trunc_f16(a0.x), trunc_f16(a0.y));
            const float2 h1 = make_float2(trunc_f16(a1.x), trunc_f16(a1.y));
            const float2 l0 = __fadd2_rn(a0, make_float2(-h0.x, -h0.y));
            const float2 l1 = __fadd2_rn(a1, make_float2(-h1.x, -h1.y));
            rh[qq] = half2_bits(h0.x, h1.x);
            ih[qq] = half2_bits(h0.y, h1.y);
            rl[qq] = half2_bits(l0.x, l1.x);
            il[qq] = half2_bits(l0.y, l1.y);
        }
        st_shared_v4(at, rh[0], rh[1], rh[2], rh[3]);
        st_shared_v4(at + kSmBMat, rl[0], rl[1], rl[2], rl[3]);
        st_shared_v4(at + 2 * kSmBMat, ih[0], ih[1], ih[2], ih[3]);
        st_shared_v4(at + 3 * kSmBMat, il[0], il[1], il[2], il[3]);
    }
    fence_proxy_async();   // the tensor cores read the stage through the async proxy
}

// Gather entries of the tile's two vector pairs (both vectors of a pair are
// neighbouring bins of one subband and one record), written by the producer
// warps: the per-pair fields of the tile's subband are fetched one tile
// ahead (the loads overlap the producer's other work) and written out when
// the tile comes up.  Producer thread tp handles entries tp + 128 j
// (T <= 256).
constexpr int kTabPerThread = 2 * kTabT / 128;
struct TabFetch {
    long long off[kTabPerThread];   // ztr_off or zte_off of the pair (whichever the tile's record uses)
    int sw[kTabPerThread], K[kTabPerThread];   // start | (W << 16), training vectors
};

__device__ __forceinline__ void tile_subband(const GatherArgs &ga, int64_t vec0, int p, int &sb, bool &train,
                                             int &v0) {
    const int64_t v = ga.vbase + vec0 + 2 * p;
    const int pr = (int)(v >> ga.log2F);
    const int qb = (int)(v & ((1 << ga.log2F) - 1));
    const int i = qb & ((1 << ga.log2B) - 1);
    sb = qb >> ga.log2B;
    train = pr < ga.P_train;
    v0 = train ? (pr << ga.log2B) + i : ((pr - ga.P_train) << ga.log2B) + i;
}

__device__ __forceinline__ void tab_fetch(const GatherArgs &ga, int64_t vec0, TabFetch &f, int tp) {
#pragma unroll
    for (int j = 0; j < kTabPerThread; ++j) {
        const int idx = tp + 128 * j;
        if (idx < 2 * ga.T) {
            const int p = idx >= ga.T ? 1 : 0;
            int sb, v0;
            bool train;
            tile_subband(ga, vec0, p, sb, train, v0);
            const long long *gs = reinterpret_cast<const long long *>(ga.gsub + 2 * ((int64_t)sb * ga.T + (idx - p * ga.T)));
            f.off[j] = __ldg(gs + (train ? 0 : 1));
            const int4 mk = __ldg(reinterpret_cast<const int4 *>(gs + 2));
            f.sw[j] = mk.x;
            f.K[j] = mk.z;
        }
    }
}

__device__ __forceinline__ void tab_write(const GatherArgs &ga, int64_t vec0, const TabFetch &f, TabEnt *tab,
                                          int tp) {
#pragma unroll
    for (int j = 0; j < kTabPerThread; ++j) {
        const int idx = tp + 128 * j;
        if (idx < 2 * ga.T) {
            const int p = idx >= ga.T ? 1 : 0;
            int sb, v0;
            bool train;
            tile_subband(ga, vec0, p, sb, train, v0);
            const int W = f.sw[j] >> 16;
            const int nst = train ? max(0, min(2, f.K[j] - v0)) : 2;
            TabEnt te;
            te.base = (int)(f.off[j] + (long long)v0 * W);
            te.swn = (f.sw[j] & 0xFFFF) | (W << 11) | (nst << 17);
            tab[p * kTabT + (idx - p * ga.T)] = te;
        }
    }
}

// ------------------------------------------------------------ epilogue side

// Row k of the DFT matrix D[k][n1] = W_128^(n1 k) into tensor memory (this
// warp's lanes): ReD and ImD, each as FP16 high and low parts, two n1 per
// 32-bit column.
__device__ __noinline__ void write_dft_rows(uint32_t tmem, const float2 *__restrict__ tw, int q, int k) {
    const uint32_t lanebits = (uint32_t)(32 * q) << 16;
#pragma unroll 1
    for (int mat = 0; mat < 4; ++mat) {
        uint32_t w[32];
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
            float v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float2 d = __ldg(&tw[16 * ((k * (2 * cc + u)) & 127)]);
                const float val = (mat < 2) ? d.x : d.y;
                const float hi = __half2float(__float2half_rn(val));
                v[u] = (mat & 1) ? val - hi : hi;
            }
            w[cc] = half2_bits(v[0], v[1]);
        }
        tmem_st32(tmem + lanebits + kTmA + 32 * mat, w);
    }
}

// Row k of the accumulators for one vector pair: twiddles W_M^(n2 k), the
// 16-point DFT along n2, beams k + 128 m2 to the pair's shared buffers (real
// parts, then imaginary parts; each entry holds the two vectors).
__device__ __forceinline__ void epilogue(uint32_t tacc, const float2 *tw, float2 *beam, int k, uint64_t *freed) {
    float re[32], im[32];
    tmem_ld2x32(tacc, tacc + 64, re, im);
    if (freed) {
        tc_fence_before();
        mbar_arrive(freed);   // the accumulator may be overwritten
    }
    float2 R[16], I[16];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
        R[n2] = make_float2(re[n2], re[16 + n2]);
        I[n2] = make_float2(im[n2], im[16 + n2]);
    }
#pragma unroll
    for (int n2 = 1; n2 < 16; ++n2) {
        const float2 t = tw[n2 * 128 + k];
        const float c = t.x, s = t.y;
        const float2 a = R[n2], b = I[n2];
        R[n2] = make_float2(a.x * c - b.x * s, a.y * c - b.y * s);
        I[n2] = make_float2(a.x * s + b.x * c, a.y * s + b.y * c);
    }
    SoaDFT<16>::run(R, I);
#pragma unroll
    for (int m2 = 0; m2 < 16; ++m2) {
        beam[k + 128 * m2] = R[m2];
        beam[2048 + k + 128 * m2] = I[m2];
    }
}

// The 48 products of one tile (N = 64 columns, K = 64 in four slices of 16):
//   Re Y = ReD Xre - ImD Xim,  Im Y = ImD Xre + ReD Xim,
// each as hi*hi + hi*lo + lo*hi (the minus through the instruction's
// negate-A bit); then one commit to `bar`.
__device__ __forceinline__ void issue_tile(uint32_t tmem, int acc, uint32_t stage, uint64_t *bar) {
    constexpr uint32_t idesc = (1u << 4)                                  // D: FP32
                               | ((uint32_t)(kTcN >> 3) << 17)            // N
                               | ((uint32_t)(128 >> 4) << 24);            // M; A, B: FP16, K-major
    constexpr uint32_t kNegA = 1u << 13;
    // A: 0 ReD hi, 1 ReD lo, 2 ImD hi, 3 ImD lo; B: 0 Xre hi, 1 Xre lo, 2 Xim hi, 3 Xim lo
    constexpr int kA[2][6] = {{0, 0, 1, 2, 2, 3}, {2, 2, 3, 0, 0, 1}};
    constexpr int kB[2][6] = {{0, 1, 0, 2, 3, 2}, {0, 1, 0, 2, 3, 2}};
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        const uint32_t d = tmem + 128 * acc + 64 * part;
#pragma unroll
        for (int t = 0; t < 6; ++t)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                mma_ts(d, tmem + kTmA + 32 * kA[part][t] + 8 * j,
                       smem_desc(stage + kSmBMat * kB[part][t] + 256 * j),
                       (part == 0 && t >= 3) ? (idesc | kNegA) : idesc, t | j);
    }
    mma_commit(bar);
}

// Window stores of vector pair p of a tile by its epilogue group (thread
// gt of 128): every (target, w) entry of the list (t << 8) | w reads beam
// start + w of both vectors of the pair from the group's beam buffer and
// stores the rows that exist.  Two entries per iteration keep two load
// chains in flight; TRAIN selects the window array (training rows in the
// plan precision, test rows in FP32).
template <int PREC, bool TRAIN>
__device__ __forceinline__ void gather_entry(const GatherArgs &ga, float2 sc, const TabEnt *tab, const float2 *beams,
                                             int pk) {
    const TabEnt te = tab[pk >> 8];
    const int n = te.swn >> 17;
    if (n == 0) return;
    const int w = pk & 255;
    const float2 *bp = beams + (((te.swn & 2047) + w) & 2047);
    const float2 re = __fmul2_rn(bp[0], sc), im = __fmul2_rn(bp[2048], sc);
    const int i0 = te.base + w;
    const int W = (te.swn >> 11) & 63;
    if (TRAIN) {
        store_train<PREC>(ga.ztr, i0, make_float2(re.x, im.x), 1.f);
        if (n > 1) store_train<PREC>(ga.ztr, i0 + W, make_float2(re.y, im.y), 1.f);
    } else {
        ga.zte[i0] = make_float2(re.x, im.x);
        ga.zte[i0 + W] = make_float2(re.y, im.y);
    }
}

template <int PREC, bool TRAIN>
__device__ __forceinline__ void gather_loop(const GatherArgs &ga, int sumW, const int *glist, float2 sc,
                                            const TabEnt *tab, const float2 *beams, int gt) {
    for (int e = gt; e < sumW; e += 256) {
        const int e1 = e + 128;
        const int pk0 = glist[e];
        const int pk1 = e1 < sumW ? glist[e1] : -1;
        gather_entry<PREC, TRAIN>(ga, sc, tab, beams, pk0);
        if (pk1 >= 0) gather_entry<PREC, TRAIN>(ga, sc, tab, beams, pk1);
    }
}

template <int PREC>
__device__ __forceinline__ void gather_pair(const TcArgs &a, const GatherArgs &ga, bool train, const int *glist,
                                            const TabEnt *tab, const float2 *beams, const float *vsc, int p, int gt) {
    const float ss = (train && PREC != BS_PREC_FP32) ? a.store_scale : 1.f;
    const float2 sc = make_float2(vsc[2 * p] * ss, vsc[2 * p + 1] * ss);
    if (train)
        gather_loop<PREC, true>(ga, a.sumW, glist, sc, tab + p * kTabT, beams, gt);
    else
        gather_loop<PREC, false>(ga, a.sumW, glist, sc, tab + p * kTabT, beams, gt);
}

// --------------------------------------------------------------------- kernel

template <int PREC>
__global__ void __launch_bounds__(kTcThreads, 1) beamspace_tc_kernel(TcArgs a, GatherArgs ga) {
    extern __shared__ __align__(1024) unsigned char smtc[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // mbarriers: done[c] (products into accumulator c complete; one
    // commit), full[b] (stage b written; 128 producer threads), freed[c]
    // (accumulator c read; the 128 threads of an epilogue group), tabfull[b]
    // (gather entries of a tile of parity b written; 128 producers),
    // tabfree[b] (that tile's windows stored; 128 epilogue threads),
    // rawbar[v] (producer v's input copy landed).  Tile i uses accumulator
    // i mod 3, stage and entry buffer i mod 2.
    uint64_t *done = reinterpret_cast<uint64_t *>(smtc + kSmMisc);
    uint64_t *full = done + 3;
    uint64_t *freed = done + 5;
    uint64_t *tabfull = done + 8;
    uint64_t *tabfree = done + 10;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smtc + kSmMisc + 96);
    int *gflag = reinterpret_cast<int *>(smtc + kSmMisc + 100);          // [2]: a group's wait gave up
    float *vsc = reinterpret_cast<float *>(smtc + kSmMisc + 112);       // [4 tiles][4 vectors]
    uint64_t *rawbar = reinterpret_cast<uint64_t *>(smtc + kSmMisc + 176);   // [4]
    TabEnt *tabs = reinterpret_cast<TabEnt *>(smtc + kSmTab);           // [2 tiles][2 pairs][kTabT]
    float2 *beams = reinterpret_cast<float2 *>(smtc + kSmBeam);         // [2 pairs][re, im][2048]
    auto train_of = [&](int64_t vec0) { return (int)((ga.vbase + vec0) >> ga.log2F) < ga.P_train; };
    const uint32_t sbase = smem_u32(smtc);
    const int64_t ntiles = ga.nvec / kTcVec;
    const int nt = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // >= 1 (grid <= ntiles)
    auto vec0_of = [&](int i) { return ((int64_t)blockIdx.x + (int64_t)i * gridDim.x) * kTcVec; };
    constexpr float post = 0.022097086912079608f;   // 1/sqrt(2048)

    if (tid == 0) {
        for (int j = 0; j < kTcAcc; ++j) {
            mbar_init(&done[j], 1);
            mbar_init(&freed[j], 128);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&full[j], 128);
            mbar_init(&tabfull[j], 128);
            mbar_init(&tabfree[j], 128);
            gflag[j] = 0;
        }
        for (int j = 0; j < 4; ++j) mbar_init(&rawbar[j], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, kTmCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    int *glist = reinterpret_cast<int *>(smtc + kSmGlist);
    for (int e = tid; e < a.sumW; e += kTcThreads) glist[e] = __ldg(&a.glist[e]);

    if (warp < 8) {
        // ---- epilogue group g = warp / 4 takes the tiles i = g mod 2 (their
        // accumulator is g): for vector pair 0, then pair 1, accumulator rows
        // k into the group's beam buffer and then that pair's window stores.
        // The two groups work on different tiles, so one group's stores
        // overlap the other's arithmetic.
        const int q = warp & 3, k = 32 * q + lane, g = warp >> 2, gt = tid & 127;
        float2 *tws = reinterpret_cast<float2 *>(smtc + kSmTw);
        if (warp < 4) {
            write_dft_rows(tmem, a.tw, q, k);
            for (int n2 = 1; n2 < 16; ++n2) tws[n2 * 128 + k] = __ldg(&a.tw[(n2 * k) & 2047]);
        }
        tc_fence_before();
        __syncthreads();   // A rows in tensor memory, twiddles and entry list in shared memory
        float2 *pb = beams + g * (kSmBeamPair / 8);
        for (int i = g; i < nt; i += 2) {
            const unsigned ph = (unsigned)(i >> 1) & 1u;
            const int c = i % kTcAcc;
            bool ok = mbar_wait_bounded(&done[c], (unsigned)(i / kTcAcc) & 1u);
            for (int p = 0; p < 2; ++p) {
                if (ok) {
                    tc_fence_after();
                    epilogue(tmem + ((uint32_t)(32 * q) << 16) + 128 * c + 32 * p, tws, pb, k,
                             p == 1 ? &freed[c] : nullptr);
                } else {
                    gflag[g] = 1;
                }
                group_bar(g);   // beams of pair p ready
                if (gflag[g]) break;
                if (p == 0 && !mbar_wait_bounded(&tabfull[g], ph)) gflag[g] = 1;
                else
                    gather_pair<PREC>(a, ga, train_of(vec0_of(i)), glist, tabs + g * 2 * kTabT, pb,
                                      vsc + 4 * (i & 3), p, gt);
                group_bar(g);   // beams free
                if (gflag[g]) break;
            }
            if (gflag[g]) break;
            mbar_arrive(&tabfree[g]);
        }
        if (gflag[g] && gt == 0) atomicOr(a.err, 1);
    } else if (warp < 12) {
        // ---- producer warps: vector v = warp - 8 of the tile after next, and
        // the gather entries of the current tile
        const int v = warp - 8, tp = tid - 256;
        float2 *raw = reinterpret_cast<float2 *>(smtc + kSmRaw) + v * 1024;
        uint64_t *rbar = rawbar + v;
        PrepRegs pr;
        TabFetch tf;
        __syncthreads();
        tab_fetch(ga, vec0_of(0), tf, tp);
        bool ok = true;
        for (int i = 0; i < 2 && i < nt && ok; ++i) {   // tiles 0 and 1 into the two stages
            prep_fetch(raw, rbar, a.y, vec0_of(i) + v, lane);
            ok = mbar_wait_bounded(rbar, (unsigned)i & 1u);
            if (!ok) break;
            prep_read(pr, raw, lane);
            prep_store(pr, sbase + kSmB + i * kSmBStage, vsc + 4 * i, v, lane, post);
            mbar_arrive(&full[i]);
            __syncwarp();   // every lane has read the slot before it is refilled
        }
        if (ok && nt > 2) prep_fetch(raw, rbar, a.y, vec0_of(2) + v, lane);
        for (int i = 0; i < nt && ok; ++i) {
            const int b = i & 1;
            // entries of tile i into buffer b once tile i - 2's windows are stored
            if (i >= 2) ok = mbar_wait_bounded(&tabfree[b], (unsigned)((i >> 1) - 1) & 1u);
            if (!ok) break;
            tab_write(ga, vec0_of(i), tf, tabs + b * 2 * kTabT, tp);
            mbar_arrive(&tabfull[b]);
            if (i + 1 < nt) tab_fetch(ga, vec0_of(i + 1), tf, tp);
            if (i + 2 < nt) {   // tile i + 2 into stage b once the products of tile i are done
                ok = mbar_wait_bounded(rbar, (unsigned)i & 1u);
                if (!ok) break;
                prep_read(pr, raw, lane);
                fence_proxy_async();   // the reads complete before the slot is refilled by the async proxy
                __syncwarp();
                if (i + 3 < nt) prep_fetch(raw, rbar, a.y, vec0_of(i + 3) + v, lane);
                ok = mbar_wait_bounded(&done[i % kTcAcc], (unsigned)(i / kTcAcc) & 1u);
                if (!ok) break;
                prep_store(pr, sbase + kSmB + b * kSmBStage, vsc + 4 * ((i + 2) & 3), v, lane, post);
                mbar_arrive(&full[b]);
            }
        }
        if (!ok && lane == 0) atomicOr(a.err, 1);
    } else {
        // ---- MMA warp: products of tile i into accumulator i mod 3 once stage
        // i mod 2 is written and (from tile 3 on) the accumulator has been read
        __syncthreads();
        for (int i = 0; i < nt; ++i) {
            const int b = i & 1, c = i % kTcAcc;
            bool ok = mbar_wait_bounded(&full[b], (unsigned)(i >> 1) & 1u);
            if (ok && i >= kTcAcc) ok = mbar_wait_bounded(&freed[c], (unsigned)(i / kTcAcc - 1) & 1u);
            if (!ok) {   // the other warps then give up on their waits
                if (lane == 0) atomicOr(a.err, 1);
                break;
            }
            tc_fence_after();
            if (lane == 0) issue_tile(tmem, c, sbase + kSmB + b * kSmBStage, &done[c]);
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmCols);
    }
}

template <int PREC>
bs_status launch_tc_p(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st) {
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            return cuda_error(cudaFuncSetAttribute(beamspace_tc_kernel<PREC>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmTotalMax),
                              "beamspace (tensor cores) attribute");
        }))
        return s;
    const int64_t ntiles = ga.nvec / kTcVec;
    if (ntiles == 0) return BS_OK;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)p->num_sms);
    TcArgs a;
    a.y = xc;
    a.tw = p->d_twM;
    a.glist = p->d_glist;
    a.sumW = p->sumW;
    a.store_scale = ga.store_scale;
    a.err = p->d_err;
    const size_t smem = (size_t)kSmGlist + 4 * (size_t)((p->sumW + 3) & ~3);
    beamspace_tc_kernel<PREC><<<grid, kTcThreads, smem, st>>>(a, ga);
    return check_launch("beamspace (tensor cores) launch");
}

}  // namespace

bool beamspace_tc_applies(const bs_plan *p) {
    return p->cfg.N == 1024 && p->cfg.M == 2048 && !p->planar && (p->B % 2) == 0 && (p->Fs % kTcVec) == 0 &&
           p->cfg.T <= kTabT && p->Wmax <= 32 && p->ztr_elems < (1LL << 31) - 64 && p->zte_elems < (1LL << 31) - 64 &&
           !(p->cfg.flags & (BS_FLAG_NO_TMA | BS_FLAG_STAGED_FFT | BS_FLAG_SIMT_FFT));
}

bs_status launch_beamspace_tc(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                              bool *used) {
    *used = false;
    if (!beamspace_tc_applies(p)) return BS_OK;
    *used = true;
    switch (p->cfg.precision) {
        case BS_PREC_FP32: return launch_tc_p<BS_PREC_FP32>(p, xc, ga, st);
        case BS_PREC_FP16: return launch_tc_p<BS_PREC_FP16>(p, xc, ga, st);
        default: return launch_tc_p<BS_PREC_BF16>(p, xc, ga, st);
    }
}

}  // namespace bs
