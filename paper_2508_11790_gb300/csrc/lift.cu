// Lifted correlator (Sec. III-C, Eq. AntennaEqCorr), its antenna-space
// application and its beam pattern (Eq. Cosine Sim).
//
// * lift: c_hat_g = D^H S_g^T c_g, i.e. c_hat_g[n] = M^-1/2 sum_w c_g[w]
//   e^{+j 2 pi m_w n / M} with m_w = start_g + w.  With z = e^{+j 2 pi n/M}
//   this is M^-1/2 z^start (sum_w c_g[w] z^w), the sum by Horner's rule:
//   two conjugated entries of the plan's M-point twiddle table per output
//   (indices n and start n mod M) and no transcendental.  Thread per
//   (pair, n).
// * apply_lifted: out[g][v'] = c_hat_g^H y_v', y_v' the channelised
//   antenna-domain vector of test vector v' of pair g's subband.  For one
//   subband this is the complex product C^H Y of the [T][N] lifted weights
//   and the [Vte][N] test vectors; a CTA computes a 32 x 32 tile of it with
//   32-element slices of both staged in shared memory.  FP32 SIMT: the path
//   keeps the accuracy of the FP32 test windows it stands in for.
// * beam_pattern: |c_hat_g^H a(Omega)| / (||c_hat_g|| sqrt(N)) for a grid of
//   direction sines u_k at pair g's squinted frequency, Omega = pi u_k f/f_d.
//   A CTA per pair holds c_hat_g in shared memory; a warp per direction sums
//   conj(c_hat[n]) e^{j Omega n} over its lanes' elements with a complex
//   rotation per 32 elements (one sincospi per lane and per direction).
#include "common.cuh"
#include "internal.h"

namespace bs {

__global__ void __launch_bounds__(256)
    lift_kernel(const float2 *__restrict__ c, const int64_t *__restrict__ woff, const int32_t *__restrict__ Wg,
                const int32_t *__restrict__ start, const float2 *__restrict__ twM, int M, int N, float scale,
                float2 *__restrict__ c_hat) {
    const int64_t g = blockIdx.x;
    const int n = blockIdx.y * blockDim.x + threadIdx.x;
    __shared__ float2 cw[32];
    const int W = Wg[g];
    if (threadIdx.x < W) cw[threadIdx.x] = c[woff[g] + threadIdx.x];
    __syncthreads();
    if (n >= N) return;
    const float2 tz = __ldg(&twM[n & (M - 1)]);
    const float2 ts = __ldg(&twM[(start[g] * n) & (M - 1)]);
    const float2 z = make_float2(tz.x, -tz.y), zs = make_float2(ts.x, -ts.y);   // e^{+j 2 pi n / M}, its start-th power
    float2 acc = cw[W - 1];
    for (int w = W - 2; w >= 0; --w) acc = cadd(cmul(acc, z), cw[w]);
    acc = cmul(acc, zs);
    c_hat[g * N + n] = make_float2(acc.x * scale, acc.y * scale);
}

constexpr int AL_T = 32;   // targets per tile
constexpr int AL_V = 32;   // test vectors per tile
constexpr int AL_K = 32;   // elements per shared-memory slice

// grid (ceil(T/32), ceil(Vte/32), L); 256 threads as 16 x 16, 2 x 2 outputs each
__global__ void __launch_bounds__(256)
    apply_lifted_kernel(const float2 *__restrict__ xc, const float2 *__restrict__ c_hat, float2 *__restrict__ out,
                        int N, int F, int B, int L, int T, int P_train, int Vte) {
    __shared__ float2 Cs[AL_T][AL_K + 1];
    __shared__ float2 Ys[AL_V][AL_K + 1];
    const int s = blockIdx.z;
    const int t0 = blockIdx.x * AL_T, v0 = blockIdx.y * AL_V;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < N; k0 += AL_K) {
        // stage: row r of each tile, lanes along the elements (coalesced)
        for (int e = threadIdx.x; e < AL_T * AL_K; e += 256) {
            const int r = e / AL_K, k = e % AL_K;
            const int t = t0 + r, v = v0 + r, n = k0 + k;
            float2 cv = make_float2(0.f, 0.f), yv = make_float2(0.f, 0.f);
            if (t < T && n < N) cv = __ldg(&c_hat[((int64_t)t * L + s) * N + n]);
            if (v < Vte && n < N) {
                const int p = P_train + v / B, q = s * B + v % B;
                yv = __ldcs(&xc[((int64_t)p * F + q) * N + n]);
            }
            Cs[r][k] = cv;
            Ys[r][k] = yv;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < AL_K; ++k) {
            const float2 c0 = Cs[2 * ty][k], c1 = Cs[2 * ty + 1][k];
            const float2 y0 = Ys[2 * tx][k], y1 = Ys[2 * tx + 1][k];
            const float2 cc[2] = {c0, c1}, yy[2] = {y0, y1};
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {   // conj(c) * y
                    acc[a][b].x = fmaf(cc[a].x, yy[b].x, fmaf(cc[a].y, yy[b].y, acc[a][b].x));
                    acc[a][b].y = fmaf(cc[a].x, yy[b].y, fmaf(-cc[a].y, yy[b].x, acc[a][b].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int t = t0 + 2 * ty + a, v = v0 + 2 * tx + b;
            if (t < T && v < Vte) out[((int64_t)t * L + s) * Vte + v] = acc[a][b];
        }
}

// one CTA per pair, a warp per direction
__global__ void __launch_bounds__(256)
    beam_pattern_kernel(const float2 *__restrict__ c_hat, const double *__restrict__ u, int n_dirs, int N, int L,
                        int Ls, int s0, double fc, double fs, double fd, float *__restrict__ pattern) {
    extern __shared__ float2 ch[];   // [N] c_hat, then [n_dirs] Omega / pi as FP32 (hi, lo)
    float2 *omt = ch + N;
    __shared__ float part[8];
    const int64_t g = blockIdx.x;
    const int s = s0 + (int)(g % Ls);   // subband of pair g among the L (plans of a shard: s0 + local)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float nrm = 0.f;
    for (int n = threadIdx.x; n < N; n += 256) {
        const float2 v = c_hat[g * N + n];
        ch[n] = v;
        nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
    }
    for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xFFFFFFFFu, nrm, o);
    if (lane == 0) part[warp] = nrm;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < 8; ++w) tot += part[w];
    const float inv = 1.f / (sqrtf(tot) * sqrtf((float)N));
    // subband centre frequency (Eq. SubChannelFreq): fc + ((l - 1/2) / L) fs,
    // l = s - L/2 + 1, in this order; Omega / pi = u f / f_d per direction,
    // formed once per CTA in FP64 and kept as an FP32 (hi, lo) pair (the FP64
    // pipe is narrow, so the per-lane work below is FP32 only)
    const double f = fc + (((double)(s - L / 2 + 1) - 0.5) / (double)L) * fs;
    const double ratio = f / fd;
    for (int k = threadIdx.x; k < n_dirs; k += 256) {
        const double om = u[k] * ratio;
        const float hi = (float)om;
        omt[k] = make_float2(hi, (float)(om - (double)hi));
    }
    __syncthreads();
    constexpr int DPW = 4;   // directions per warp pass: each shared load feeds four sums
    for (int k0 = warp * DPW; k0 < n_dirs; k0 += 8 * DPW) {
        // Omega / pi = u f / fd; e^{j Omega n} with n = lane + 32 i.  The two
        // phases (in units of pi) are reduced to [-1, 1] in FP64 before the
        // FP32 sincospi, so their error does not grow with n.
        float er[DPW], ei[DPW], c32[DPW], s32[DPW], re[DPW], im[DPW];
#pragma unroll
        for (int d = 0; d < DPW; ++d) {
            const float2 om = (k0 + d < n_dirs) ? omt[k0 + d] : make_float2(0.f, 0.f);
            // x0 = om * lane: exact product of the high part (fmaf), reduced
            // modulo 2 before the low-order terms are added
            const float p = om.x * (float)lane;
            const float e = fmaf(om.x, (float)lane, -p) + om.y * (float)lane;
            const float x0 = (p - 2.f * rintf(0.5f * p)) + e;
            const float q = om.x * 32.f;   // exact
            const float x32 = (q - 2.f * rintf(0.5f * q)) + om.y * 32.f;
            sincospif(x0, &ei[d], &er[d]);
            sincospif(x32, &s32[d], &c32[d]);
            re[d] = im[d] = 0.f;
        }
        for (int n = lane; n < N; n += 32) {
            const float2 a = ch[n];
#pragma unroll
            for (int d = 0; d < DPW; ++d) {   // conj(a) * e, then e *= e^{j 32 Omega}
                re[d] = fmaf(a.x, er[d], fmaf(a.y, ei[d], re[d]));
                im[d] = fmaf(a.x, ei[d], fmaf(-a.y, er[d], im[d]));
                const float nr = er[d] * c32[d] - ei[d] * s32[d];
                ei[d] = fmaf(er[d], s32[d], ei[d] * c32[d]);
                er[d] = nr;
            }
        }
#pragma unroll
        for (int d = 0; d < DPW; ++d) {
            for (int o = 16; o; o >>= 1) {
                re[d] += __shfl_xor_sync(0xFFFFFFFFu, re[d], o);
                im[d] += __shfl_xor_sync(0xFFFFFFFFu, im[d], o);
            }
            if (lane == 0 && k0 + d < n_dirs) pattern[g * n_dirs + k0 + d] = sqrtf(re[d] * re[d] + im[d] * im[d]) * inv;
        }
    }
}

bs_status launch_lift(const bs_plan *p, const float2 *c, float2 *c_hat, cudaStream_t st) {
    const int N = p->cfg.N;
    if (p->pairs == 0) return BS_OK;
    if (p->Wmax > 32) return set_error(BS_EUNSUPPORTED, "W > 32");
    dim3 grid((unsigned)p->pairs, (N + 255) / 256);
    lift_kernel<<<grid, 256, 0, st>>>(c, p->d_woff, p->d_Wg, p->d_start, p->d_twM, p->cfg.M, N,
                                      1.0f / sqrtf((float)p->cfg.M), c_hat);
    return check_launch("lift launch");
}

bs_status launch_apply_lifted(const bs_plan *p, const float2 *xc, const float2 *c_hat, float2 *out,
                              cudaStream_t st) {
    const int T = p->cfg.T, L = p->Ls, Vte = p->Vte;   // the plan's subbands, Fs bins per record of xc
    if (Vte == 0 || p->pairs == 0) return BS_OK;
    if (L > 65535) return set_error(BS_EUNSUPPORTED, "apply_lifted: at most 65535 subbands");
    dim3 grid((T + AL_T - 1) / AL_T, (Vte + AL_V - 1) / AL_V, L);
    apply_lifted_kernel<<<grid, 256, 0, st>>>(xc, c_hat, out, p->cfg.N, p->Fs, p->B, L, T, p->cfg.P_train, Vte);
    return check_launch("apply_lifted launch");
}

bs_status launch_beam_pattern(const bs_plan *p, const float2 *c_hat, int n_dirs, const double *u, float *pattern,
                              cudaStream_t st) {
    if (n_dirs == 0 || p->pairs == 0) return BS_OK;
    const size_t smem = ((size_t)p->cfg.N + n_dirs) * sizeof(float2);
    if (smem > 200 * 1024) return set_error(BS_EUNSUPPORTED, "beam pattern: N + n_dirs must be <= 25600");
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(beam_pattern_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "beam pattern attribute");
    }
    beam_pattern_kernel<<<(unsigned)p->pairs, 256, smem, st>>>(c_hat, u, n_dirs, p->cfg.N, p->cfg.L, p->Ls, p->s0,
                                                              p->cfg.fc, p->cfg.fs, p->cfg.fd, pattern);
    return check_launch("beam pattern launch");
}

}  // namespace bs
