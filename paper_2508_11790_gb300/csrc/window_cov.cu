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
//
// One CTA per pair.  The lower triangle (i >= j) has E = W(W+1)/2 entries;
// thread (e, h) accumulates entry e over the vectors v = h (mod H),
// H = blockDim / E.  Vectors are staged through shared memory in chunks of
// 16*H so every thread adds exactly one block of <= 16 products per chunk.
#include "common.cuh"
#include "internal.h"

namespace bs {

constexpr int COV_THREADS = 256;
constexpr int COV_SMEM_ELEMS = 2048;   // float2 staging elements (16 KB)

// (hi, lo) += b with Knuth's two-sum; the pair keeps ~48 bits.
__device__ __forceinline__ void df_add(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}

template <int PREC>
__device__ __forceinline__ float2 load_window(const void *z, int64_t idx, float inv_sc) {
    if constexpr (PREC == BS_PREC_FP32) {
        return __ldcs(reinterpret_cast<const float2 *>(z) + idx);
    } else if constexpr (PREC == BS_PREC_FP16) {
        const __half2 h = reinterpret_cast<const __half2 *>(z)[idx];
        const float2 f = __half22float2(h);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    } else {
        const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162 *>(z)[idx];
        const float2 f = __bfloat1622float2(h);
        return make_float2(f.x * inv_sc, f.y * inv_sc);
    }
}

template <int PREC>
__global__ void __launch_bounds__(COV_THREADS)
    window_cov_kernel(const void *__restrict__ z, const int64_t *__restrict__ ztr_off,
                      const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                      const int64_t *__restrict__ roff, const float *__restrict__ delta_pair,
                      double delta, float inv_sc, double2 *__restrict__ R) {
    __shared__ float2 zs[COV_SMEM_ELEMS];
    __shared__ float red[4][COV_THREADS];
    const int64_t g = blockIdx.x;
    const int tid = threadIdx.x;
    const int W = Wg[g], K = Kg[g];
    const int E = W * (W + 1) / 2;
    int H = COV_THREADS / E;
    int kc = 16 * H;
    if (kc * W > COV_SMEM_ELEMS) kc = COV_SMEM_ELEMS / W;
    const int64_t zb = ztr_off[g];

    // this thread's entry (i, j), i >= j, and slice h
    const int e = tid % E, h = tid / E;
    const bool active = h < H;
    int i = 0, j = 0;
    {
        int rem = e;
        while (rem > i) { rem -= i + 1; ++i; }
        j = rem;
    }
    float hr = 0.f, lr = 0.f, hi_ = 0.f, li = 0.f;

    for (int k0 = 0; k0 < K; k0 += kc) {
        const int n = min(kc, K - k0);
        __syncthreads();
        for (int q = tid; q < n * W; q += COV_THREADS)
            zs[q] = load_window<PREC>(z, zb + (int64_t)k0 * W + q, inv_sc);
        __syncthreads();
        if (active) {
            float ar = 0.f, ai = 0.f;
            for (int v = h; v < n; v += H) {
                const float2 a = zs[v * W + i], b = zs[v * W + j];
                ar = fmaf(a.x, b.x, fmaf(a.y, b.y, ar));
                ai = fmaf(a.y, b.x, fmaf(-a.x, b.y, ai));
            }
            df_add(hr, lr, ar);
            df_add(hi_, li, ai);
        }
    }
    red[0][tid] = hr;
    red[1][tid] = lr;
    red[2][tid] = hi_;
    red[3][tid] = li;
    __syncthreads();
    if (tid < E) {
        double sr = 0.0, si = 0.0;
        for (int hh = 0; hh < H; ++hh) {
            const int o = hh * E + tid;
            sr += (double)red[0][o] + (double)red[1][o];
            si += (double)red[2][o] + (double)red[3][o];
        }
        const double d = delta_pair ? (double)delta_pair[g] : delta;
        const double invK = 1.0 / (double)K;
        double2 *Rg = R + roff[g];
        sr *= invK;
        si *= invK;
        if (i == j) {
            Rg[i * W + i] = make_double2(sr + d, 0.0);
        } else {
            Rg[i * W + j] = make_double2(sr, si);
            Rg[j * W + i] = make_double2(sr, -si);
        }
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
    const int i = threadIdx.x / 16, j = threadIdx.x % 16;
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

bs_status launch_window_cov(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                            cudaStream_t st) {
    const unsigned G = (unsigned)p->pairs;
    if (p->cfg.flags & BS_FLAG_PLAIN) {
        if (p->cfg.precision != BS_PREC_FP32)
            return set_error(BS_EINVAL, "the plain path is FP32 only");
        plain_cov_kernel<<<G, 256, 0, st>>>((const float2 *)ztr, p->d_ztr_off, p->d_Wg, p->d_Kg,
                                            p->d_roff, delta, (float)p->cfg.delta, R);
        return check_launch("plain covariance launch");
    }
    const float inv_sc = 1.0f / p->cfg.store_scale;
    switch (p->cfg.precision) {
        case BS_PREC_FP32:
            window_cov_kernel<BS_PREC_FP32><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, p->cfg.delta, 1.0f, R);
            break;
        case BS_PREC_FP16:
            window_cov_kernel<BS_PREC_FP16><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, p->cfg.delta, inv_sc, R);
            break;
        default:
            window_cov_kernel<BS_PREC_BF16><<<G, COV_THREADS, 0, st>>>(
                ztr, p->d_ztr_off, p->d_Wg, p->d_Kg, p->d_roff, delta, p->cfg.delta, inv_sc, R);
            break;
    }
    return check_launch("covariance launch");
}

}  // namespace bs
