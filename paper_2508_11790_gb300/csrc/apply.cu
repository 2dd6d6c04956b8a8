// Beamformer output (Sec. II-B, applied per pair to the windowed test
// vectors): out[g][v'] = c_g^H z_test[g][v'] = sum_w conj(c_g[w]) z[v'][w].
//
// One thread per output: each reads its W_g contiguous window entries;
// neighbouring threads read neighbouring windows, so the loads of a warp
// cover one contiguous span.  Memory bound (8 W + 8 bytes per output).
#include "common.cuh"
#include "internal.h"

namespace bs {

__global__ void __launch_bounds__(256)
    apply_kernel(const float2 *__restrict__ z, const int64_t *__restrict__ zte_off,
                 const int32_t *__restrict__ Wg, const int64_t *__restrict__ woff,
                 const float2 *__restrict__ c, float2 *__restrict__ out, int64_t total, int Vte) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t g = idx / Vte;
    const int v = (int)(idx - g * Vte);
    const int W = __ldg(&Wg[g]);
    const float2 *zv = z + __ldg(&zte_off[g]) + (int64_t)v * W;
    const float2 *cg = c + __ldg(&woff[g]);
    float re = 0.f, im = 0.f;
    for (int w = 0; w < W; ++w) {
        const float2 a = __ldcs(&zv[w]);
        const float2 b = __ldg(&cg[w]);
        // conj(b) * a
        re = fmaf(b.x, a.x, fmaf(b.y, a.y, re));
        im = fmaf(b.x, a.y, fmaf(-b.y, a.x, im));
    }
    out[idx] = make_float2(re, im);
}

bs_status launch_apply(const bs_plan *p, const float2 *zte, const float2 *c, float2 *out, cudaStream_t st) {
    const int64_t total = p->pairs * p->Vte;
    if (total == 0) return BS_OK;
    const int64_t blocks = (total + 255) / 256;
    apply_kernel<<<(unsigned)blocks, 256, 0, st>>>(zte, p->d_zte_off, p->d_Wg, p->d_woff, c, out, total, p->Vte);
    return check_launch("apply launch");
}

}  // namespace bs
