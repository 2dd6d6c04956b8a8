// Learned diagonal loading: window features, output SINR, labels, and the
// forward / backward / Adam kernels of a 3-layer MLP (hidden width H) that
// maps the features of a window to [log10 delta, log10 d_1..d_W].
//
// Features of a window with unloaded sample covariance R (K training
// vectors, Eq. EmpiricalCov) and windowed steering vector a (Sec. III-C),
// tau = tr(R) / W:
//   diag(R)/tau (W) | Re R_ij/tau, i > j row-major | Im R_ij/tau, same order |
//   Re a/|a| (W) | Im a/|a| (W) | log10 tau | log10(K/W)      (W^2 + 2W + 2).
// Weights are kept in FP32 (master, Adam) with a BF16 copy that the forward
// and backward products read; all products accumulate in FP32.
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace bs {

// ----------------------------------------------------------------- features
__global__ void features_kernel(const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                                const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg,
                                const int64_t *__restrict__ woff, const double2 *__restrict__ at64,
                                int64_t pairs, int nfeat, float *__restrict__ X) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    const int W = Wg[g];
    const double2 *Rg = R + roff[g];
    const double2 *a = at64 + woff[g];
    float *x = X + g * nfeat;
    double tr = 0.0;
    for (int i = 0; i < W; ++i) tr += Rg[i * W + i].x;
    const double tau = tr / W;
    const double itau = 1.0 / tau;
    int o = 0;
    for (int i = 0; i < W; ++i) x[o++] = (float)(Rg[i * W + i].x * itau);
    for (int i = 1; i < W; ++i)
        for (int j = 0; j < i; ++j) x[o++] = (float)(Rg[i * W + j].x * itau);
    for (int i = 1; i < W; ++i)
        for (int j = 0; j < i; ++j) x[o++] = (float)(Rg[i * W + j].y * itau);
    double na = 0.0;
    for (int i = 0; i < W; ++i) na += a[i].x * a[i].x + a[i].y * a[i].y;
    const double ina = 1.0 / sqrt(na);
    for (int i = 0; i < W; ++i) x[o++] = (float)(a[i].x * ina);
    for (int i = 0; i < W; ++i) x[o++] = (float)(a[i].y * ina);
    x[o++] = (float)log10(tau);
    x[o++] = (float)log10((double)Kg[g] / (double)W);
}

// ----------------------------------------------------------------- SINR judge
// sinr[g] = |c^H a|^2 / (c^H R_ref c) (FP64), c and a of pair g.
__global__ void sinr_kernel(const float2 *__restrict__ c, const double2 *__restrict__ Rref,
                            const int64_t *__restrict__ roff, const int32_t *__restrict__ Wg,
                            const int64_t *__restrict__ woff, const double2 *__restrict__ at64, int64_t pairs,
                            double *__restrict__ sinr) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    const int W = Wg[g];
    const float2 *cg = c + woff[g];
    const double2 *a = at64 + woff[g];
    const double2 *Rg = Rref + roff[g];
    double nr = 0.0, ni = 0.0, den = 0.0;
    for (int i = 0; i < W; ++i) {
        const double cr = cg[i].x, ci = cg[i].y;
        nr += cr * a[i].x + ci * a[i].y;   // conj(c) a
        ni += cr * a[i].y - ci * a[i].x;
        double tr = 0.0, ti = 0.0;          // (R c)_i
        for (int j = 0; j < W; ++j) {
            const double2 r = Rg[i * W + j];
            const double xr = cg[j].x, xi = cg[j].y;
            tr += r.x * xr - r.y * xi;
            ti += r.x * xi + r.y * xr;
        }
        den += cr * tr + ci * ti;           // Re(conj(c_i) (R c)_i)
    }
    sinr[g] = (nr * nr + ni * ni) / den;
}

// ----------------------------------------------------------------- labels
// For each pair: argmax over the loading grid of sinr[k][g] (first maximum),
// targets [log10 delta*, -0.5 log10(R_ii + delta*)].
__global__ void labels_kernel(const double *__restrict__ sinr, int ngrid, const double *__restrict__ grid,
                              const double2 *__restrict__ R, const int64_t *__restrict__ roff,
                              const int32_t *__restrict__ Wg, int64_t pairs, int nout, float *__restrict__ T,
                              float *__restrict__ best_delta) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    int kb = 0;
    double sb = sinr[g];
    for (int k = 1; k < ngrid; ++k) {
        const double s = sinr[(int64_t)k * pairs + g];
        if (s > sb) { sb = s; kb = k; }
    }
    const double d = grid[kb];
    if (best_delta) best_delta[g] = (float)d;
    float *t = T + g * nout;
    t[0] = (float)log10(d);
    const int W = Wg[g];
    const double2 *Rg = R + roff[g];
    for (int i = 0; i < W && i + 1 < nout; ++i) t[1 + i] = (float)(-0.5 * log10(Rg[i * W + i].x + d));
}

// ----------------------------------------------------------------- GEMM
// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) (ReLU), with
//   A(m, k) = A[m * sam + k * sak],  B(k, n) = B[k * sbk + n * sbn].
// 64 x 64 tiles, k steps of 16, 256 threads with 4 x 4 outputs each; B is
// FP32 or BF16 (widened on the way into shared memory); FP32 accumulation.
template <class TB, bool kBias, bool kRelu>
__global__ void __launch_bounds__(256)
    gemm_kernel(const float *__restrict__ A, int64_t sam, int64_t sak, const TB *__restrict__ B, int64_t sbk,
                int64_t sbn, const float *__restrict__ bias, float *__restrict__ C, int64_t ldc, int M, int N,
                int K, float *__restrict__ Cpre) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e / 64, i = e % 64;
            const int m = m0 + i, k = k0 + kk;
            As[kk][i] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : 0.f;
            const int n = n0 + i;
            float bv = 0.f;
            if (n < N && k < K) {
                if constexpr (sizeof(TB) == 2)
                    bv = __bfloat162float(B[(int64_t)k * sbk + (int64_t)n * sbn]);
                else
                    bv = B[(int64_t)k * sbk + (int64_t)n * sbn];
            }
            Bs[kk][i] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                a[r] = As[kk][tm + r];
                b[r] = Bs[kk][tn + r];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int m = m0 + tm + r, n = n0 + tn + q;
            if (m < M && n < N) {
                float v = acc[r][q];
                if constexpr (kBias) v += bias[n];
                if (Cpre) Cpre[(int64_t)m * ldc + n] = v;
                if constexpr (kRelu) v = fmaxf(v, 0.f);
                C[(int64_t)m * ldc + n] = v;
            }
        }
}

template <class TB, bool kBias, bool kRelu>
static void gemm(const float *A, int64_t sam, int64_t sak, const TB *B, int64_t sbk, int64_t sbn,
                 const float *bias, float *C, int64_t ldc, int M, int N, int K, float *Cpre, cudaStream_t st) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TB, kBias, kRelu><<<grid, 256, 0, st>>>(A, sam, sak, B, sbk, sbn, bias, C, ldc, M, N, K, Cpre);
}

// ----------------------------------------------------------------- elementwise
__global__ void relu_bwd_kernel(float *__restrict__ d, const float *__restrict__ z, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(z[i] > 0.f)) d[i] = 0.f;
}

// db[j] = sum_i dz[i][j]: 32 columns x 8 row groups per CTA, then atomics.
__global__ void colsum_kernel(const float *__restrict__ dz, int M, int N, float *__restrict__ db) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * 256 + threadIdx.y;
    if (j >= N) return;
    float s = 0.f;
    for (int i = r0; i < M && i < (int)(blockIdx.y + 1) * 256; i += 8) s += dz[(int64_t)i * N + j];
    atomicAdd(&db[j], s);
}

// dY = 2 (Y - T) / (M N); loss += sum (Y - T)^2 / (M N)
__global__ void mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, int64_t n, float scale,
                                float *__restrict__ dY, double *__restrict__ loss) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float e2 = 0.f;
    if (i < n) {
        const float e = Y[i] - T[i];
        dY[i] = 2.f * e * scale;
        e2 = e * e * scale;
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xFFFFFFFFu, e2, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, (double)e2);
}

// Adam (bias-corrected), FP32 master parameters, BF16 copy refreshed.
__global__ void adam_kernel(float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

__global__ void gather_rows_kernel(const float *__restrict__ src, const int64_t *__restrict__ idx, int64_t rows,
                                   int cols, float *__restrict__ dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e / cols;
    const int c = (int)(e - r * cols);
    dst[e] = src[idx[r] * cols + c];
}

// delta_g = 10^y[g][0], clipped to [lo, hi]; non-finite -> fallback.
__global__ void loading_from_mlp_kernel(const float *__restrict__ Y, int nout, int64_t pairs, float lo, float hi,
                                        float fallback, float *__restrict__ delta) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= pairs) return;
    const float y = Y[g * nout];
    float d = exp10f(y);
    if (!isfinite(y) || !isfinite(d)) d = fallback;
    delta[g] = fminf(fmaxf(d, lo), hi);
}

// d[g][i] = 10^Y[g][1 + i] for the W entries of pair g (the preconditioner
// outputs); a non-finite output gives 1 (no scaling of that entry).
__global__ void precond_from_mlp_kernel(const float *__restrict__ Y, int nout, int64_t pairs, int W,
                                        float *__restrict__ d) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= pairs * W) return;
    const int64_t g = e / W;
    const int i = (int)(e % W);
    const float y = Y[g * nout + 1 + i];
    const float v = exp10f(y);
    d[e] = (isfinite(y) && isfinite(v) && v > 0.f) ? v : 1.0f;
}

static unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace bs

using bs::set_error;

// ---------------------------------------------------------------- C entry points
extern "C" {

int64_t bs_mlp_param_count(int32_t n_in, int32_t n_hidden, int32_t n_out) {
    return (int64_t)n_hidden * n_in + n_hidden + (int64_t)n_hidden * n_hidden + n_hidden +
           (int64_t)n_out * n_hidden + n_out;
}

bs_status bs_features(const bs_plan *p, const bs_cf64 *R_unloaded, float *X, bs_stream stream) {
    if (!p || !R_unloaded || !X) return set_error(BS_EINVAL, "NULL argument");
    for (int t = 1; t < p->cfg.T; ++t)
        if (p->Wt[t] != p->Wt[0]) return set_error(BS_EINVAL, "features need one window size for all targets");
    const int W = p->Wt[0];
    const int nfeat = W * W + 2 * W + 2;
    bs::features_kernel<<<bs::blocks_for(p->pairs, 128), 128, 0, (cudaStream_t)stream>>>(
        (const double2 *)R_unloaded, p->d_roff, p->d_Wg, p->d_Kg, p->d_woff, p->d_at64, p->pairs, nfeat, X);
    return bs::check_launch("features launch");
}

bs_status bs_output_sinr(const bs_plan *p, const bs_cf32 *c, const bs_cf64 *R_ref, double *sinr, bs_stream stream) {
    if (!p || !c || !R_ref || !sinr) return set_error(BS_EINVAL, "NULL argument");
    bs::sinr_kernel<<<bs::blocks_for(p->pairs, 128), 128, 0, (cudaStream_t)stream>>>(
        (const float2 *)c, (const double2 *)R_ref, p->d_roff, p->d_Wg, p->d_woff, p->d_at64, p->pairs, sinr);
    return bs::check_launch("sinr launch");
}

bs_status bs_loading_labels(const bs_plan *p, const double *sinr, int32_t ngrid, const double *grid,
                            const bs_cf64 *R_unloaded, int32_t nout, float *T, float *best_delta, bs_stream stream) {
    if (!p || !sinr || !grid || !R_unloaded || !T || ngrid < 1 || nout < 1) return set_error(BS_EINVAL, "bad argument");
    bs::labels_kernel<<<bs::blocks_for(p->pairs, 128), 128, 0, (cudaStream_t)stream>>>(
        sinr, ngrid, grid, (const double2 *)R_unloaded, p->d_roff, p->d_Wg, p->pairs, nout, T, best_delta);
    return bs::check_launch("labels launch");
}

// Parameter layout (FP32 master and BF16 copy alike):
// W1 [H][n_in] | b1 [H] | W2 [H][H] | b2 [H] | W3 [n_out][H] | b3 [n_out]
static bs_status mlp_check(const bs_mlp *m) {
    if (!m || !m->master || !m->weights_bf16) return set_error(BS_EINVAL, "NULL MLP");
    if (m->n_in < 1 || m->n_hidden < 1 || m->n_out < 1) return set_error(BS_EINVAL, "bad MLP sizes");
    return BS_OK;
}

bs_status bs_mlp_forward(const bs_mlp *m, const float *X, int64_t batch, float *Y, const bs_mlp_work *w,
                         bs_stream stream) {
    if (bs_status s = mlp_check(m)) return s;
    if (!X || !Y || !w || !w->z1 || !w->h1 || !w->z2 || !w->h2) return set_error(BS_EINVAL, "NULL buffer");
    if (batch < 0 || batch > w->capacity) return set_error(BS_EINVAL, "batch exceeds the work buffers");
    if (batch == 0) return BS_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    const int I = m->n_in, H = m->n_hidden, O = m->n_out, B = (int)batch;
    const __nv_bfloat16 *wb = (const __nv_bfloat16 *)m->weights_bf16;
    const float *b1 = m->master + (int64_t)H * I, *b2 = b1 + H + (int64_t)H * H, *b3 = b2 + H + (int64_t)O * H;
    const __nv_bfloat16 *W1 = wb, *W2 = wb + (int64_t)H * I + H, *W3 = W2 + (int64_t)H * H + H;
    // Z1 = X W1^T + b1, H1 = relu(Z1)   (B(k, n) = W1[n][k])
    bs::gemm<__nv_bfloat16, true, true>(X, I, 1, W1, 1, I, b1, w->h1, H, B, H, I, w->z1, st);
    bs::gemm<__nv_bfloat16, true, true>(w->h1, H, 1, W2, 1, H, b2, w->h2, H, B, H, H, w->z2, st);
    bs::gemm<__nv_bfloat16, true, false>(w->h2, H, 1, W3, 1, H, b3, Y, O, B, O, H, nullptr, st);
    return bs::check_launch("MLP forward");
}

bs_status bs_mlp_train_step(bs_mlp *m, const float *X, const float *T, int64_t batch, const bs_mlp_work *w,
                            float lr, double *loss, bs_stream stream) {
    if (bs_status s = bs_mlp_forward(m, X, batch, w->y, w, stream)) return s;
    if (!T || !m->grad || !m->adam_m || !m->adam_v || !w->dy || !w->dh1 || !w->dh2)
        return set_error(BS_EINVAL, "NULL buffer");
    if (batch == 0) return BS_OK;
    const cudaStream_t st = (cudaStream_t)stream;
    const int I = m->n_in, H = m->n_hidden, O = m->n_out, B = (int)batch;
    const int64_t P = bs_mlp_param_count(I, H, O);
    const __nv_bfloat16 *wb = (const __nv_bfloat16 *)m->weights_bf16;
    const __nv_bfloat16 *W2 = wb + (int64_t)H * I + H, *W3 = W2 + (int64_t)H * H + H;
    float *gW1 = m->grad, *gb1 = gW1 + (int64_t)H * I, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H;
    float *gW3 = gb2 + H, *gb3 = gW3 + (int64_t)O * H;
    cudaError_t e = cudaMemsetAsync(m->grad, 0, P * sizeof(float), st);
    if (e != cudaSuccess) return bs::cuda_error(e, "gradient reset");
    // dY
    bs::mse_grad_kernel<<<bs::blocks_for((int64_t)B * O), 256, 0, st>>>(w->y, T, (int64_t)B * O,
                                                                          1.0f / (float)((int64_t)B * O), w->dy, loss);
    // layer 3: gW3 = dY^T H2 [O][H], gb3 = colsum dY, dH2 = dY W3 [B][H]
    bs::gemm<float, false, false>(w->dy, 1, O, w->h2, H, 1, nullptr, gW3, H, O, H, B, nullptr, st);
    bs::colsum_kernel<<<dim3((O + 31) / 32, (B + 255) / 256), dim3(32, 8), 0, st>>>(w->dy, B, O, gb3);
    bs::gemm<__nv_bfloat16, false, false>(w->dy, O, 1, W3, H, 1, nullptr, w->dh2, H, B, H, O, nullptr, st);
    bs::relu_bwd_kernel<<<bs::blocks_for((int64_t)B * H), 256, 0, st>>>(w->dh2, w->z2, (int64_t)B * H);
    // layer 2
    bs::gemm<float, false, false>(w->dh2, 1, H, w->h1, H, 1, nullptr, gW2, H, H, H, B, nullptr, st);
    bs::colsum_kernel<<<dim3((H + 31) / 32, (B + 255) / 256), dim3(32, 8), 0, st>>>(w->dh2, B, H, gb2);
    bs::gemm<__nv_bfloat16, false, false>(w->dh2, H, 1, W2, H, 1, nullptr, w->dh1, H, B, H, H, nullptr, st);
    bs::relu_bwd_kernel<<<bs::blocks_for((int64_t)B * H), 256, 0, st>>>(w->dh1, w->z1, (int64_t)B * H);
    // layer 1
    bs::gemm<float, false, false>(w->dh1, 1, H, X, I, 1, nullptr, gW1, I, H, I, B, nullptr, st);
    bs::colsum_kernel<<<dim3((H + 31) / 32, (B + 255) / 256), dim3(32, 8), 0, st>>>(w->dh1, B, H, gb1);
    if (bs_status s = bs::check_launch("MLP backward")) return s;
    if (lr > 0.f) {
        m->step += 1;
        const float bc1 = 1.f - powf(0.9f, (float)m->step), bc2 = 1.f - powf(0.999f, (float)m->step);
        bs::adam_kernel<<<bs::blocks_for(P), 256, 0, st>>>(m->master, (__nv_bfloat16 *)m->weights_bf16, m->grad,
                                                          m->adam_m, m->adam_v, P, lr, 0.9f, 0.999f, 1e-8f, bc1, bc2);
        return bs::check_launch("Adam");
    }
    return BS_OK;
}

bs_status bs_mlp_sync_bf16(const bs_mlp *m, bs_stream stream) {
    if (bs_status s = mlp_check(m)) return s;
    const int64_t P = bs_mlp_param_count(m->n_in, m->n_hidden, m->n_out);
    bs::to_bf16_kernel<<<bs::blocks_for(P), 256, 0, (cudaStream_t)stream>>>(
        m->master, (__nv_bfloat16 *)m->weights_bf16, P);
    return bs::check_launch("BF16 copy");
}

bs_status bs_gather_rows(const float *src, const int64_t *idx, int64_t rows, int32_t cols, float *dst,
                         bs_stream stream) {
    if (!src || !idx || !dst || rows < 0 || cols < 1) return set_error(BS_EINVAL, "bad argument");
    if (rows == 0) return BS_OK;
    bs::gather_rows_kernel<<<bs::blocks_for(rows * cols), 256, 0, (cudaStream_t)stream>>>(src, idx, rows, cols, dst);
    return bs::check_launch("gather");
}

bs_status bs_precond_from_mlp(const float *Y, int32_t nout, int64_t pairs, int32_t W, float *d, bs_stream stream) {
    if (!Y || !d || W < 1 || nout < 1 + W || pairs < 0) return set_error(BS_EINVAL, "bad argument");
    if (pairs == 0) return BS_OK;
    bs::precond_from_mlp_kernel<<<bs::blocks_for(pairs * W), 256, 0, (cudaStream_t)stream>>>(Y, nout, pairs, W, d);
    return bs::check_launch("preconditioner from MLP");
}

bs_status bs_loading_from_mlp(const float *Y, int32_t nout, int64_t pairs, float lo, float hi, float fallback,
                              float *delta, bs_stream stream) {
    if (!Y || !delta || nout < 1 || pairs < 0 || !(lo > 0.f) || !(hi >= lo)) return set_error(BS_EINVAL, "bad argument");
    if (pairs == 0) return BS_OK;
    bs::loading_from_mlp_kernel<<<bs::blocks_for(pairs), 256, 0, (cudaStream_t)stream>>>(Y, nout, pairs, lo, hi,
                                                                                         fallback, delta);
    return bs::check_launch("loading from MLP");
}

}  // extern "C"
