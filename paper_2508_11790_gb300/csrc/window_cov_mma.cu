// Loaded window covariance from 16-bit windows on the tensor cores
// (Eq. EmpiricalCov on the windowed vectors, plus loading), FP32 accumulate.
//
// With real rows m = 2w + c (c = 0: real part, 1: imaginary part of window
// entry w) the K training vectors of a pair form a real 2W x K matrix A, and
//   D = A A^T,   R_ij = (D[2i][2j] + D[2i+1][2j+1]
//                        + j (D[2i+1][2j] - D[2i][2j+1])) / K.
// One warp per pair computes the lower part of D with mma.sync m16n8k16
// (FP16 or BF16 inputs, FP32 accumulators): per 16 vectors, two
// ldmatrix.x4.trans per 16-row tile of A and per 16 columns of A^T, and one
// MMA per (16 x 8) output tile on or below the diagonal.
//
// Windows stream through a per-warp ring of shared-memory stages of 64
// vectors (cp.async).  For 2W <= 24 the stage rows are 48 bytes apart
// (ldmatrix's 8 row reads then start in 8 different 16-byte bank groups)
// and the ring has 4 stages, so three chunks are in flight while one is
// consumed; wider windows use 80-byte rows and 2 stages in the same 12 KB.
// A window stream of one pair is latency-bound per warp: the bytes in flight
// per SM set its bandwidth.  The accumulators are folded into double-float
// every 128 vectors, and R is assembled in FP64.  The per-pair body is
// compiled once per tile class ceil(2W / 8) = 1 .. 4, so tile counts, ring
// stride and depth are constants and only the accumulators of tiles on or
// below the diagonal exist; full 64-vector stages run an unrolled k loop.
//
// The covariance is HBM-bound (2 W flop per byte for 16-bit windows): the
// tensor cores remove the FP32 multiply-add work that otherwise bounds the
// kernel, leaving the window stream.
#include "common.cuh"
#include "internal.h"

namespace bs {

constexpr int MMA_CH = 64;                 // vectors per stage
constexpr int MMA_WARPS = 4;               // warps (= pairs) per CTA
constexpr int MMA_WARP_HALVES = 6144;      // per-warp ring: 4 x 64 x 24 or 2 x 64 x 40 16-bit elements (12 KB)
// dynamic shared memory: the rings plus 64 bytes, because ldmatrix of the
// columns 16..31 of a 24-element row reads into the next row (those columns
// only feed rows and columns of D beyond 2W, which are not used)
constexpr size_t MMA_SMEM = (size_t)MMA_WARPS * MMA_WARP_HALVES * 2 + 64;

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_mma() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_mma() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], const void *row_addr) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(row_addr));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

template <int PREC>
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    if constexpr (PREC == BS_PREC_FP16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

__device__ __forceinline__ void df_fold(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}


// One pair (the calling warp) of window size W with NNT = ceil(2W / 8)
// 8-column tiles of A^T: the tile counts, the ring's row stride and depth
// and the accumulators that exist are compile-time per class.
template <int PREC, int NNT>
__device__ __forceinline__ void cov_pair(uint16_t *ring, int lane, int64_t g, int W, int K, const void *z,
                                         const int64_t *__restrict__ ztr_off, const int64_t *__restrict__ roff,
                                         const float *__restrict__ delta_pair, DF delta, DF inv_sc2,
                                         double2 *__restrict__ R) {
    constexpr int nnt = NNT;                    // 8-column tiles of A^T
    constexpr int nmt = (NNT + 1) / 2;          // 16-row tiles of A
    constexpr int RS = (NNT <= 3) ? 24 : 40;    // stage row stride (16-bit elements): 2W <= 24 or <= 32
    constexpr int nst = (NNT <= 3) ? 4 : 2;     // stages in the ring
    auto srow = [&](int b, int v) { return ring + (b * MMA_CH + v) * RS; };
    const uint32_t *zg = reinterpret_cast<const uint32_t *>(z) + ztr_off[g];   // one 32-bit word per complex

    // zero the ring (padding columns must read as 0)
    for (int q = lane; q < MMA_WARP_HALVES / 2; q += 32) reinterpret_cast<uint32_t *>(ring)[q] = 0u;
    __syncwarp();

    // lane -> (window entry w = lane % 16, vector parity lane / 16): no division
    const int lw = lane & 15, lv = lane >> 4;
    auto issue = [&](int k0, int buf) {   // commits one group, empty past the end
        const int n = min(MMA_CH, K - k0);
        if (lw < W) {
            const uint32_t *src = zg + (int64_t)(k0 + lv) * W + lw;
            for (int v = lv; v < n; v += 2, src += 2 * W) cp_async4(srow(buf, v) + 2 * lw, src);
        }
        cp_async_commit_mma();
    };

    float acc[2][4][4];
    float hi[2][4][4], lo[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[a][b][e] = hi[a][b][e] = lo[a][b][e] = 0.f;

    const int mi = lane >> 3, rr = lane & 7;   // ldmatrix: matrix index and row of this lane's address
    const int nch = (K + MMA_CH - 1) / MMA_CH;
    for (int c = 0; c < nst - 1; ++c) issue(c * MMA_CH, c);
    for (int c = 0; c < nch; ++c) {
        const int k0 = c * MMA_CH, buf = c % nst;
        const int n = min(MMA_CH, K - k0);
        issue(k0 + (nst - 1) * MMA_CH, (c + nst - 1) % nst);   // stage consumed at c - 1
        if (nst == 4) cp_async_wait_mma<3>();
        else cp_async_wait_mma<1>();
        __syncwarp();
        if (n < MMA_CH) {   // last chunk: vectors n .. up to the next multiple of 16 must be zero
            const int top = (n + 15) & ~15;
            for (int q = lane; q < (top - n) * RS / 2; q += 32)
                reinterpret_cast<uint32_t *>(srow(buf, n))[q] = 0u;
            __syncwarp();
        }
        auto kstep = [&](int kk) {
            // A^T fragments (B operand) for column tiles 0..nnt-1, two tiles per ldmatrix.x4
            unsigned bfr[4][2];
#pragma unroll
            for (int tp = 0; tp < 2; ++tp) {
                if (2 * tp < nnt) {
                    // matrices: (cols 16tp, k), (16tp, k+8), (16tp+8, k), (16tp+8, k+8)
                    const int col = 16 * tp + ((mi >> 1) << 3);
                    const int krow = kk + ((mi & 1) << 3) + rr;
                    unsigned r[4];
                    ldsm_x4_trans(r, srow(buf, krow) + col);
                    bfr[2 * tp][0] = r[0];
                    bfr[2 * tp][1] = r[1];
                    bfr[2 * tp + 1][0] = r[2];
                    bfr[2 * tp + 1][1] = r[3];
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt < nmt) {
                    // matrices: (rows 16mt, k), (16mt+8, k), (16mt, k+8), (16mt+8, k+8)
                    const int row = 16 * mt + ((mi & 1) << 3);
                    const int krow = kk + ((mi >> 1) << 3) + rr;
                    unsigned afr[4];
                    ldsm_x4_trans(afr, srow(buf, krow) + row);
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        if (nt < nnt && 16 * mt + 15 >= 8 * nt) mma16816<PREC>(acc[mt][nt], afr, bfr[nt][0], bfr[nt][1]);
                }
            }
        };
        if (n == MMA_CH) {
#pragma unroll
            for (int kk = 0; kk < MMA_CH; kk += 16) kstep(kk);
        } else {
            for (int kk = 0; kk < n; kk += 16) kstep(kk);
        }
        // fold the FP32 accumulators (at most 128 vectors each) into double-float
        if (c % 2 == 1 || c == nch - 1) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (a < nmt && b < nnt && 16 * a + 15 >= 8 * b) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            df_fold(hi[a][b][e], lo[a][b][e], acc[a][b][e]);
                            acc[a][b][e] = 0.f;
                        }
                    }
        }
        __syncwarp();   // this stage is reloaded by the next iteration's issue
    }
    cp_async_wait_mma<0>();   // the empty trailing groups
    __syncwarp();

    // D (double-float) into the warp's ring, then R from its 2x2 real blocks
    float2 *Dm = reinterpret_cast<float2 *>(ring);   // [32][32] pairs = 8 KB <= 12 KB
    const int gr = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
            if (mt < nmt && nt < nnt && 16 * mt + 15 >= 8 * nt) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = 16 * mt + gr + ((e >> 1) << 3);
                    const int col = 8 * nt + 2 * tg + (e & 1);
                    Dm[row * 32 + col] = make_float2(hi[mt][nt][e], lo[mt][nt][e]);
                }
            }
    __syncwarp();
    // sc = inv_sc2 / K in double-float (K < 2^24 is exact in FP32)
    const float Kf = (float)K;
    const float q = inv_sc2.h / Kf;
    const float rem = fmaf(-q, Kf, inv_sc2.h);
    const DF sc = df_norm(q, (rem + inv_sc2.l) / Kf);
    const DF dl = delta_pair ? DF{delta_pair[g], 0.f} : delta;
    auto D = [&](int r, int c) {
        const float2 v = Dm[r * 32 + c];
        return DF{v.x, v.y};
    };
    double2 *Rg = R + roff[g];
    const int E = W * (W + 1) / 2;
    for (int e = lane; e < E; e += 32) {
        int i = 0, r2 = e;
        while (r2 > i) { r2 -= i + 1; ++i; }
        const int j = r2;
        DF re = df_mul(df_add(D(2 * i, 2 * j), D(2 * i + 1, 2 * j + 1)), sc);
        if (i == j) {
            Rg[i * W + i] = make_double2(df_to_double(df_add(re, dl)), 0.0);
        } else {
            const DF nd = D(2 * i, 2 * j + 1);
            const DF im = df_mul(df_add(D(2 * i + 1, 2 * j), DF{-nd.h, -nd.l}), sc);
            const double rd = df_to_double(re), id = df_to_double(im);
            Rg[i * W + j] = make_double2(rd, id);
            Rg[j * W + i] = make_double2(rd, __longlong_as_double(__double_as_longlong(id) ^ (1ll << 63)));
        }
    }
}

// One warp per pair; the pair's tile class is a warp-uniform switch (a
// kernel compiled for one class alone was slower: with the shared memory
// setting the occupancy, the smaller register budget only cost overlap).
template <int PREC>
__global__ void __launch_bounds__(MMA_WARPS * 32)
    window_cov_mma_kernel(const void *__restrict__ z, const int64_t *__restrict__ ztr_off,
                          const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                          const int64_t *__restrict__ roff, const float *__restrict__ delta_pair, DF delta,
                          DF inv_sc2, double2 *__restrict__ R, int64_t pairs) {
    extern __shared__ __align__(16) uint16_t mma_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * MMA_WARPS + warp;
    if (g >= pairs) return;   // uniform per warp; no CTA-wide barrier below
    uint16_t *ring = mma_smem + warp * MMA_WARP_HALVES;
    const int W = Wg[g], K = Kg[g];
    switch ((2 * W + 7) >> 3) {   // warp-uniform
        case 1: cov_pair<PREC, 1>(ring, lane, g, W, K, z, ztr_off, roff, delta_pair, delta, inv_sc2, R); break;
        case 2: cov_pair<PREC, 2>(ring, lane, g, W, K, z, ztr_off, roff, delta_pair, delta, inv_sc2, R); break;
        case 3: cov_pair<PREC, 3>(ring, lane, g, W, K, z, ztr_off, roff, delta_pair, delta, inv_sc2, R); break;
        default: cov_pair<PREC, 4>(ring, lane, g, W, K, z, ztr_off, roff, delta_pair, delta, inv_sc2, R); break;
    }
}

bs_status launch_window_cov_mma(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                                cudaStream_t st) {
    const int64_t G = p->pairs;
    const unsigned blocks = (unsigned)((G + MMA_WARPS - 1) / MMA_WARPS);
    static PerDevice attr;
    if (bs_status s = attr.get([](int *) {
            cudaError_t e = cudaFuncSetAttribute(window_cov_mma_kernel<BS_PREC_FP16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MMA_SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(window_cov_mma_kernel<BS_PREC_BF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MMA_SMEM);
            return cuda_error(e, "covariance (tensor core) attribute");
        }))
        return s;
    const DF sc = df_from_double(1.0 / ((double)p->cfg.store_scale * (double)p->cfg.store_scale));
    const DF dl = df_from_double(p->cfg.delta);
    if (p->cfg.precision == BS_PREC_FP16)
        window_cov_mma_kernel<BS_PREC_FP16><<<blocks, MMA_WARPS * 32, MMA_SMEM, st>>>(
            ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, dl, sc, R, G);
    else
        window_cov_mma_kernel<BS_PREC_BF16><<<blocks, MMA_WARPS * 32, MMA_SMEM, st>>>(
            ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, dl, sc, R, G);
    return check_launch("covariance (tensor core) launch");
}

}  // namespace bs
