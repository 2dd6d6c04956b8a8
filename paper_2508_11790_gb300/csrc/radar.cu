// Processing after the beamformer (Sec. II, Fig. 1: synthesis of the
// wideband output and standard range-Doppler processing; Sec. IV: detection
// 10 dB above the noise floor).
//
// * gather: the beamformed output of pair (t, s) at test vector r B + i is
//   bin q = s B + i of record r, FFT bin k = (q - F/2) mod F.  The matched
//   filter multiplies it by conj(P[k]) (P: the transmitted pulse's
//   orthonormal spectrum).  The synthesis IFFT runs as a forward FFT of the
//   conjugate, IFFT(Z) = conj(FFT(conj Z)) (orthonormal), so the gather
//   writes conj(Y conj(P)) = conj(Y) P.
// * rows: the library's one-shot row FFT (F points, F-point twiddle table).
// * doppler: map[t][d][tau] = |sum_r rp[t][r][tau] e^{-j 2 pi d r / P_te}|^2
//   with rp = conj(row FFT output); thread per (t, tau), all d.
// * cfar (Sec. IV-B: a one-dimensional CFAR across the velocity bins): one
//   CTA per target, a thread per range cell tau: the floor of cell (d, tau)
//   is the mean of the other P_te - 1 velocity bins of range cell tau (the
//   cell under test left out), a detection is a cell above its floor x
//   10^(thr/10) (FP32); the CTA counts the detections and reduces the
//   strongest one (smallest index on ties) to the target's peak cell.
#include "common.cuh"
#include "internal.h"

namespace bs {

__global__ void rd_gather_kernel(const float2 *__restrict__ out, const float2 *__restrict__ pulse,
                                 float2 *__restrict__ w, int T, int L, int B, int P_te) {
    const int F = L * B;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (t, r, q)
    const int64_t total = (int64_t)T * P_te * F;
    if (e >= total) return;
    const int q = (int)(e % F);
    const int64_t tr = e / F;
    const int r = (int)(tr % P_te), t = (int)(tr / P_te);
    const int s = q / B, i = q % B;
    const int k = (q - F / 2 + F) % F;
    const float2 y = out[((int64_t)t * L + s) * ((int64_t)P_te * B) + (int64_t)r * B + i];
    const float2 pk = pulse[k];
    // conj(y) * pk
    w[tr * F + k] = make_float2(y.x * pk.x + y.y * pk.y, y.x * pk.y - y.y * pk.x);
}

__global__ void rd_doppler_kernel(const float2 *__restrict__ fr, float *__restrict__ map, int T, int P_te, int F) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (t, tau)
    if (e >= (int64_t)T * F) return;
    const int tau = (int)(e % F), t = (int)(e / F);
    const float2 *col = fr + (int64_t)t * P_te * F + tau;
    for (int d = 0; d < P_te; ++d) {
        float re = 0.f, im = 0.f;
        for (int r = 0; r < P_te; ++r) {
            const float2 v = col[(int64_t)r * F];       // rp = conj(v)
            float sn, cs;
            sincospif(-2.f * (float)((d * r) % P_te) / (float)P_te, &sn, &cs);
            // conj(v) * (cs + j sn)
            re = fmaf(v.x, cs, fmaf(v.y, sn, re));
            im = fmaf(v.x, sn, fmaf(-v.y, cs, im));
        }
        map[((int64_t)t * P_te + d) * F + tau] = re * re + im * im;
    }
}

__global__ void __launch_bounds__(256) rd_cfar_kernel(const float *__restrict__ map, int P_te, int F, float ratio,
                                                      float *__restrict__ floor_out, int32_t *__restrict__ count,
                                                      uint8_t *__restrict__ mask, int32_t *__restrict__ peak) {
    const int t = blockIdx.x;
    const int64_t cells = (int64_t)P_te * F;
    const float *m = map + (int64_t)t * cells;
    __shared__ float best_v[256];
    __shared__ int best_i[256];
    __shared__ int cnt_s;
    if (threadIdx.x == 0) cnt_s = 0;
    __syncthreads();
    const float inv = 1.0f / (float)(P_te - 1);
    float bv = -1.0f;   // map cells are >= 0
    int bi = -1, mine = 0;
    for (int tau = threadIdx.x; tau < F; tau += 256) {
        for (int d = 0; d < P_te; ++d) {
            float sum = 0.f;   // the other velocity bins of range cell tau, in order
            for (int e = 0; e < P_te; ++e)
                if (e != d) sum += m[(int64_t)e * F + tau];
            const float fl = sum * inv;
            const int64_t c = (int64_t)d * F + tau;
            const float v = m[c];
            const bool hit = v > fl * ratio;
            floor_out[(int64_t)t * cells + c] = fl;
            if (mask) mask[(int64_t)t * cells + c] = hit ? 1 : 0;
            mine += hit;
            if (hit && (v > bv || (v == bv && (int)c < bi))) {
                bv = v;
                bi = (int)c;
            }
        }
    }
    best_v[threadIdx.x] = bv;
    best_i[threadIdx.x] = bi;
    atomicAdd(&cnt_s, mine);
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            const float v2 = best_v[threadIdx.x + o];
            const int i2 = best_i[threadIdx.x + o];
            const float v1 = best_v[threadIdx.x];
            const int i1 = best_i[threadIdx.x];
            if (i2 >= 0 && (i1 < 0 || v2 > v1 || (v2 == v1 && i2 < i1))) {
                best_v[threadIdx.x] = v2;
                best_i[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        count[t] = cnt_s;
        if (peak) peak[t] = best_i[0];
    }
}

bs_status launch_range_doppler(const bs_plan *p, const float2 *out, const float2 *pulse, float2 *work, float *map,
                               cudaStream_t st) {
    const int T = p->cfg.T, L = p->cfg.L, B = p->B, P_te = p->cfg.P_test, F = p->cfg.F;
    if (P_te == 0 || T == 0) return BS_OK;
    const int64_t rows = (int64_t)T * P_te;
    const int64_t n1 = rows * F;
    float2 *w1 = work, *w2 = work + n1;
    rd_gather_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(out, pulse, w1, T, L, B, P_te);
    if (bs_status s = check_launch("range-Doppler gather launch")) return s;
    if (bs_status s = launch_fft_rows(p, w1, rows, w2, st)) return s;
    const int64_t n2 = (int64_t)T * F;
    rd_doppler_kernel<<<(unsigned)((n2 + 127) / 128), 128, 0, st>>>(w2, map, T, P_te, F);
    return check_launch("Doppler launch");
}

bs_status launch_cfar(const bs_plan *p, const float *map, float threshold_db, float *floor, int32_t *count,
                      uint8_t *mask, int32_t *peak, cudaStream_t st) {
    const int T = p->cfg.T;
    if (T == 0 || p->cfg.P_test == 0) return BS_OK;
    const float ratio = powf(10.f, threshold_db / 10.f);
    rd_cfar_kernel<<<T, 256, 0, st>>>(map, p->cfg.P_test, p->cfg.F, ratio, floor, count, mask, peak);
    return check_launch("CFAR launch");
}

}  // namespace bs
