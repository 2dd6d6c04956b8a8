// Loaded window covariance (Eq. EmpiricalCov on the windowed vectors of
// Eq. ApplyWindow, plus diagonal loading):
//   R_g = (1/K_g) sum_{v < K_g} z_v z_v^H + delta_g I,  stored in FP64.
//
// Accuracy: with a strong interferer the entries of R_g span many orders of
// magnitude and the MVDR weights are sensitive to unstructured relative
// errors of about kappa(R) * eps in R.  Products are therefore summed in
// FP32 over blocks of at most 16 vectors only, and the block sums are
// combined in double-float (hi + lo FP32 pair, error-free two-sum), which
// keeps R accurate far beyond FP32 at little extra cost.
#include "common.cuh"
#include "internal.h"

namespace bs {

constexpr int COV_THREADS = 128;
constexpr int WMAX_COV = 16;             // largest window
constexpr int COV_STAGE_ELEMS = 1024;  // window elements per staging buffer (8 KB in FP32)

// (hi, lo) += b with Knuth's two-sum; the pair keeps ~48 bits.
__device__ __forceinline__ void df_add(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}

// cp.async (global -> shared, bypassing registers) of one 8-byte or 4-byte
// element; completion is tracked per thread with commit/wait groups.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int PREC>
__device__ __forceinline__ float2 widen(const void *stage, int q, float inv_sc) {
    if constexpr (PREC == BS_PREC_FP32) {
        return reinterpret_cast<const float2 *>(stage)[q];
    } else if constexpr (PREC == BS_PREC_FP16) {
        const float2 f = __half22float2(reinterpret_cast<const __half2 *>(stage)[q]);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    } else {
        const float2 f = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(stage)[q]);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    }
}

// One CTA per pair.  The K x W windows stream through two shared-memory
// stages (cp.async, the next chunk loads while the current one is used).
// The lower triangle is cut into 3x3 tiles; thread (tile, slice) keeps its
// tile in registers and, per vector, loads 6 window entries for 9 complex
// multiply-adds.  FP32 sums cover at most 16 vectors and are folded into
// double-float accumulators; the slices are reduced in double-float.
template <int PREC>
__global__ void __launch_bounds__(COV_THREADS)
    window_cov_kernel(const void *__restrict__ z, const int64_t *__restrict__ ztr_off,
                      const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                      const int64_t *__restrict__ roff, const float *__restrict__ delta_pair,
                      DF delta, float inv_sc, double2 *__restrict__ R) {
    constexpr int ES = (PREC == BS_PREC_FP32) ? 8 : 4;          // bytes per stored element
    __shared__ __align__(16) unsigned char stage[2][COV_STAGE_ELEMS * ES];
    __shared__ float red[4][9][COV_THREADS];
    const int64_t g = blockIdx.x;
    const int tid = threadIdx.x;
    const int W = Wg[g], K = Kg[g];
    const int nb3 = (W + 2) / 3;
    const int nblk = nb3 * (nb3 + 1) / 2;
    const int H = COV_THREADS / nblk;
    const int tile = tid % nblk, h = tid / nblk;
    const bool active = h < H;
    int bi = 0, rem = tile;
    while (rem > bi) { rem -= bi + 1; ++bi; }
    const int i0 = 3 * bi, j0 = 3 * rem;
    const int kc = COV_STAGE_ELEMS / W;                            // vectors per chunk
    const unsigned char *zg = reinterpret_cast<const unsigned char *>(z) + ztr_off[g] * ES;

    auto issue = [&](int k0, int buf) {
        const int n = min(kc, K - k0);
        for (int q = tid; q < n * W; q += COV_THREADS)
            cp_async<ES>(&stage[buf][q * ES], zg + ((int64_t)k0 * W + q) * ES);
        cp_async_commit();
    };

    float ar[3][3], ai[3][3], hr[3][3], lr[3][3], hi[3][3], li[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) ar[r][q] = ai[r][q] = hr[r][q] = lr[r][q] = hi[r][q] = li[r][q] = 0.f;
    int cnt = 0;

    issue(0, 0);
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += kc, buf ^= 1) {
        const int n = min(kc, K - k0);
        if (k0 + kc < K) {
            issue(k0 + kc, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
            for (int v = h; v < n; v += H) {
                const int o = v * W;
                float2 zi[3], zj[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    zi[r] = (i0 + r < W) ? widen<PREC>(stage[buf], o + i0 + r, inv_sc) : make_float2(0.f, 0.f);
                    zj[r] = (j0 + r < W) ? widen<PREC>(stage[buf], o + j0 + r, inv_sc) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {   // z_i conj(z_j)
                        ar[r][q] = fmaf(zi[r].x, zj[q].x, fmaf(zi[r].y, zj[q].y, ar[r][q]));
                        ai[r][q] = fmaf(zi[r].y, zj[q].x, fmaf(-zi[r].x, zj[q].y, ai[r][q]));
                    }
                if (++cnt == 16) {
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            df_add(hr[r][q], lr[r][q], ar[r][q]);
                            df_add(hi[r][q], li[r][q], ai[r][q]);
                            ar[r][q] = ai[r][q] = 0.f;
                        }
                    cnt = 0;
                }
            }
        }
        __syncthreads();   // this stage is reloaded two chunks later
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            df_add(hr[r][q], lr[r][q], ar[r][q]);
            df_add(hi[r][q], li[r][q], ai[r][q]);
            red[0][3 * r + q][tid] = hr[r][q];
            red[1][3 * r + q][tid] = lr[r][q];
            red[2][3 * r + q][tid] = hi[r][q];
            red[3][3 * r + q][tid] = li[r][q];
        }
    __syncthreads();

    // 1/K, the loading and R in double-float; FP64 only for the stored values
    const float Kf = (float)K;
    const float qk = 1.f / Kf;
    const DF invK = df_norm(qk, fmaf(-qk, Kf, 1.f) / Kf);
    const DF dl = delta_pair ? DF{delta_pair[g], 0.f} : delta;
    double2 *Rg = R + roff[g];
    const int E = W * (W + 1) / 2;
    for (int e = tid; e < E; e += COV_THREADS) {
        int i = 0, r2 = e;
        while (r2 > i) { r2 -= i + 1; ++i; }
        const int j = r2;
        const int b = (i / 3) * (i / 3 + 1) / 2 + j / 3;
        const int ee = 3 * (i % 3) + (j % 3);
        float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
        for (int hh = 0; hh < H; ++hh) {
            const int o = hh * nblk + b;
            df_add(sh, sl, red[0][ee][o]);
            sl += red[1][ee][o];
            df_add(th, tl, red[2][ee][o]);
            tl += red[3][ee][o];
        }
        const DF re = df_mul(df_norm(sh, sl), invK);
        if (i == j) {
            Rg[i * W + i] = make_double2(df_to_double(df_add(re, dl)), 0.0);
        } else {
            const double rd = df_to_double(re), id = df_to_double(df_mul(df_norm(th, tl), invK));
            Rg[i * W + j] = make_double2(rd, id);
            Rg[j * W + i] = make_double2(rd, __longlong_as_double(__double_as_longlong(id) ^ (1ll << 63)));
        }
    }
}

// Short window streams (K <= 128): one warp per pair, four pairs per CTA.
// The warp stages chunks of 64 vectors of its pair with coalesced loads;
// lane l owns entries e = l + 32 k (k < ceil(E / 32) <= 5) of the lower
// triangle (E = W (W + 1) / 2 <= 136, a per-pair switch on the count) and
// sums z_i conj(z_j) over the vectors itself, in FP32 over
// COVW_FOLD vectors folded into double-float, so no reduction across
// threads is needed; R is assembled as in window_cov_kernel.  With one CTA
// per pair, a short stream left each thread at most a vector or two and
// the CTA-wide reduction and barriers dominated.
constexpr int COVW_WARPS = 4;
constexpr int COVW_CH = 64;    // vectors per staged chunk
// FP32 partial sums cover COVW_FOLD vectors before they are folded into
// double-float.  With 16 (the CTA kernel's bound) the worst MVDR weight
// error of the short-stream workloads was 2.1e-4 (K = 18, W = 9) and 1.9e-3
// (K = 6..120, W = 3..15); with 4 it is 5.7e-5 and 5.1e-4 (the CTA kernel,
// which spreads a short stream over many thread slices so that its FP32
// sums hold a product or two: 2.0e-5 and 1.1e-3).
constexpr int COVW_FOLD = 4;

// One pair (the calling warp) with EPL = ceil(W (W + 1) / 64) entries per
// lane; lanes past the last entry accumulate entry (0, 0) and store nothing,
// so the vector loop has no per-entry predicate.
template <int PREC, int EPL>
__device__ __forceinline__ void cov_warp_pair(unsigned char *sb, int lane, int64_t g, int W, int K,
                                              const unsigned char *zg, const int64_t *__restrict__ roff,
                                              const float *__restrict__ delta_pair, DF delta, float inv_sc,
                                              double2 *__restrict__ R) {
    constexpr int ES = (PREC == BS_PREC_FP32) ? 8 : 4;   // bytes per stored element
    const int E = W * (W + 1) / 2;
    int ii[EPL], jj[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        int i = 0, r = lane + 32 * k;
        if (r < E) {
            while (r > i) { r -= i + 1; ++i; }
        } else {
            r = 0;
        }
        ii[k] = i;
        jj[k] = r;
    }
    float ar[EPL], ai[EPL], hr[EPL], lr[EPL], hi[EPL], li[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) ar[k] = ai[k] = hr[k] = lr[k] = hi[k] = li[k] = 0.f;
    auto fold = [&]() {
#pragma unroll
        for (int k = 0; k < EPL; ++k) {
            df_add(hr[k], lr[k], ar[k]);
            df_add(hi[k], li[k], ai[k]);
            ar[k] = ai[k] = 0.f;
        }
    };
    int cnt = 0;
    for (int k0 = 0; k0 < K; k0 += COVW_CH) {
        const int n = min(COVW_CH, K - k0);
        if constexpr (ES == 8) {
            const float2 *src = reinterpret_cast<const float2 *>(zg) + (int64_t)k0 * W;
            float2 *dst = reinterpret_cast<float2 *>(sb);
            for (int q = lane; q < n * W; q += 32) dst[q] = __ldg(src + q);
        } else {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(zg) + (int64_t)k0 * W;
            uint32_t *dst = reinterpret_cast<uint32_t *>(sb);
            for (int q = lane; q < n * W; q += 32) dst[q] = __ldg(src + q);
        }
        __syncwarp();
        for (int v = 0, o = 0; v < n; ++v, o += W) {
#pragma unroll
            for (int k = 0; k < EPL; ++k) {   // z_i conj(z_j)
                const float2 zi = widen<PREC>(sb, o + ii[k], inv_sc), zj = widen<PREC>(sb, o + jj[k], inv_sc);
                ar[k] = fmaf(zi.x, zj.x, fmaf(zi.y, zj.y, ar[k]));
                ai[k] = fmaf(zi.y, zj.x, fmaf(-zi.x, zj.y, ai[k]));
            }
            if (++cnt == COVW_FOLD) {
                fold();
                cnt = 0;
            }
        }
        __syncwarp();   // the chunk is overwritten by the next one
    }
    fold();

    // 1/K, the loading and R in double-float; FP64 only for the stored values
    const float Kf = (float)K;
    const float qk = 1.f / Kf;
    const DF invK = df_norm(qk, fmaf(-qk, Kf, 1.f) / Kf);
    const DF dl = delta_pair ? DF{delta_pair[g], 0.f} : delta;
    double2 *Rg = R + roff[g];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        if (lane + 32 * k >= E) continue;
        const int i = ii[k], j = jj[k];
        const DF re = df_mul(df_norm(hr[k], lr[k]), invK);
        if (i == j) {
            Rg[i * W + i] = make_double2(df_to_double(df_add(re, dl)), 0.0);
        } else {
            const double rd = df_to_double(re), id = df_to_double(df_mul(df_norm(hi[k], li[k]), invK));
            Rg[i * W + j] = make_double2(rd, id);
            Rg[j * W + i] = make_double2(rd, __longlong_as_double(__double_as_longlong(id) ^ (1ll << 63)));
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(COVW_WARPS * 32)
    window_cov_warp_kernel(const void *__restrict__ z, const int64_t *__restrict__ ztr_off,
                           const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                           const int64_t *__restrict__ roff, const float *__restrict__ delta_pair, DF delta,
                           float inv_sc, double2 *__restrict__ R, int64_t slot0, int64_t slot1,
                           const int32_t *__restrict__ order) {
    constexpr int ES = (PREC == BS_PREC_FP32) ? 8 : 4;   // bytes per stored element
    __shared__ __align__(16) unsigned char stage[COVW_WARPS][COVW_CH * WMAX_COV * ES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slot = slot0 + (int64_t)blockIdx.x * COVW_WARPS + warp;
    if (slot >= slot1) return;   // uniform per warp; no CTA barrier below
    const int64_t g = order ? (int64_t)order[slot] : slot;   // pairs [slot0, slot1) of `order`, or in pair order
    const int W = Wg[g], K = Kg[g];
    unsigned char *sb = stage[warp];
    const unsigned char *zg = reinterpret_cast<const unsigned char *>(z) + ztr_off[g] * ES;
    switch ((W * (W + 1) / 2 + 31) >> 5) {   // warp-uniform
        case 1: cov_warp_pair<PREC, 1>(sb, lane, g, W, K, zg, roff, delta_pair, delta, inv_sc, R); break;
        case 2: cov_warp_pair<PREC, 2>(sb, lane, g, W, K, zg, roff, delta_pair, delta, inv_sc, R); break;
        case 3: cov_warp_pair<PREC, 3>(sb, lane, g, W, K, zg, roff, delta_pair, delta, inv_sc, R); break;
        case 4: cov_warp_pair<PREC, 4>(sb, lane, g, W, K, zg, roff, delta_pair, delta, inv_sc, R); break;
        default: cov_warp_pair<PREC, 5>(sb, lane, g, W, K, zg, roff, delta_pair, delta, inv_sc, R); break;
    }
}

// Plain FP32 per-pair covariance: one CTA per pair, one thread per matrix
// entry, one FP32 sum over all K vectors read straight from memory.
__global__ void plain_cov_kernel(const float2 *__restrict__ z, const int64_t *__restrict__ ztr_off,
                                 const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                                 const int64_t *__restrict__ roff, const float *__restrict__ delta_pair,
                                 float delta, double2 *__restrict__ R) {
    const int64_t g = blockIdx.x;
    const int W = Wg[g], K = Kg[g];
    const int side = blockDim.x == 256 ? 16 : 32;   // thread (i, j) per entry
    const int i = threadIdx.x / side, j = threadIdx.x % side;
    if (i >= W || j >= W) return;
    const float2 *zg = z + ztr_off[g];
    float ar = 0.f, ai = 0.f;
    for (int v = 0; v < K; ++v) {
        const float2 a = zg[v * W + i], b = zg[v * W + j];
        ar += a.x * b.x + a.y * b.y;
        ai += a.y * b.x - a.x * b.y;
    }
    const float invK = 1.0f / (float)K;
    ar *= invK;
    ai *= invK;
    if (i == j) ar += delta_pair ? delta_pair[g] : delta;
    R[roff[g] + i * W + j] = make_double2((double)ar, (double)ai);
}

bool window_cov_uses_warp(const bs_plan *p) {
    if (p->cfg.flags & BS_FLAG_PLAIN) return false;
    const bool wide = p->Wmax > WMAX_COV;
    const int tv = p->tune_cov;
    const bool mma_ok = !wide && p->cfg.precision != BS_PREC_FP32;
    if (mma_ok && (tv == 2 || (tv < 0 && !(p->cfg.flags & BS_FLAG_SIMT_COV)))) return false;
    const bool warp_ok = !wide && p->Kmax <= 128;
    return warp_ok && (tv == 1 || (tv < 0 && p->pairs >= 4 * (int64_t)p->num_sms));
}

bs_status launch_window_cov_warp(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                                 cudaStream_t st, int64_t slot0, int64_t slot1, const int32_t *order) {
    if (slot1 <= slot0) return BS_OK;
    const unsigned blocks = (unsigned)((slot1 - slot0 + COVW_WARPS - 1) / COVW_WARPS);
    const DF dl = df_from_double(p->cfg.delta);
    const float inv_sc = 1.0f / p->cfg.store_scale;
    switch (p->cfg.precision) {
        case BS_PREC_FP32:
            window_cov_warp_kernel<BS_PREC_FP32><<<blocks, COVW_WARPS * 32, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, dl, 1.0f, R, slot0, slot1, order);
            break;
        case BS_PREC_FP16:
            window_cov_warp_kernel<BS_PREC_FP16><<<blocks, COVW_WARPS * 32, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, dl, inv_sc, R, slot0, slot1, order);
            break;
        default:
            window_cov_warp_kernel<BS_PREC_BF16><<<blocks, COVW_WARPS * 32, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, dl, inv_sc, R, slot0, slot1, order);
            break;
    }
    return check_launch("covariance (warp per pair) launch");
}

bs_status launch_window_cov(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                            cudaStream_t st) {
    const unsigned G = (unsigned)p->pairs;
    if (p->cfg.flags & BS_FLAG_PLAIN) {
        if (p->cfg.precision != BS_PREC_FP32)
            return set_error(BS_EINVAL, "the plain path is FP32 only");
        plain_cov_kernel<<<G, p->Wmax <= 16 ? 256 : 1024, 0, st>>>((const float2 *)ztr, p->d_ztr_off, p->d_Wg,
                                                                   p->d_Kg, p->d_roff, delta, (float)p->cfg.delta, R);
        return check_launch("plain covariance launch");
    }
    // windows above 16 beams: the CTA-per-pair kernel (its 3 x 3 tiles cover
    // any W; 16-bit windows are widened to FP32 as they are staged)
    const bool wide = p->Wmax > WMAX_COV;
    if (wide && p->Wmax > 32) return set_error(BS_EUNSUPPORTED, "W > 32");
    const int tv = p->tune_cov;   // a variant chosen by bs_autotune_pass, where it applies
    const bool mma_ok = !wide && p->cfg.precision != BS_PREC_FP32;
    if (mma_ok && (tv == 2 || (tv < 0 && !(p->cfg.flags & BS_FLAG_SIMT_COV))))
        return launch_window_cov_mma(p, ztr, delta, R, st);
    const float inv_sc = 1.0f / p->cfg.store_scale;
    // warp per pair: short streams over enough pairs to fill the GPU by warps
    if (window_cov_uses_warp(p)) return launch_window_cov_warp(p, ztr, delta, R, st, 0, p->pairs, nullptr);
    switch (p->cfg.precision) {
        case BS_PREC_FP32:
            window_cov_kernel<BS_PREC_FP32><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, df_from_double(p->cfg.delta), 1.0f, R);
            break;
        case BS_PREC_FP16:
            window_cov_kernel<BS_PREC_FP16><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, df_from_double(p->cfg.delta), inv_sc, R);
            break;
        default:
            window_cov_kernel<BS_PREC_BF16><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, df_from_double(p->cfg.delta), inv_sc, R);
            break;
    }
    return check_launch("covariance launch");
}

}  // namespace bs
