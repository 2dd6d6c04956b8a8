// Window-gather arguments and helpers shared by the beamspace kernels
// (Eq. OverallWindow, Eq. ApplyWindow): which beams of a transformed
// (record, bin) vector land where in the packed training / test windows.
#pragma once
#include "common.cuh"
#include "bs.h"

struct bs_plan;

namespace bs {

// Vectors per CTA of the beamspace kernels: vpb = 4096 / M clamped to
// [1, 16] (34.8 KB of padded shared memory at M = 2048).
template <int M>
struct BsCfg {
    static constexpr int vpb = (4096 / M > 16) ? 16 : ((4096 / M < 1) ? 1 : 4096 / M);
    static constexpr int nthr = (vpb * M / 16 < 256) ? vpb * M / 16 : 256;
    static constexpr int pl = padded_len(M);
    static constexpr size_t smem = (size_t)vpb * pl * sizeof(float2);
    static constexpr int minb = (smem <= 40 * 1024) ? 4 : ((smem <= 72 * 1024) ? 3 : 1);
};

struct GatherArgs {
    int64_t nvec;           // vectors of this launch (a whole number of records)
    int64_t vbase;          // index of its first vector in the cube (multiple of F)
    int log2F, log2B, L, P_train, T;
    int uniform;            // B % vpb == 0: the vectors of a CTA share (record, subband)
    const int32_t *gather;  // [vpb * sumW] (t << 10) | (c << 5) | w
    const longlong2 *gsub;  // [L][T][2]: {ztr_off, zte_off}, {start | W << 16, K}
    int ngather;
    const int32_t *Wg, *Kg, *start;
    const int64_t *ztr_off, *zte_off;
    void *ztr;              // training windows (plan precision)
    float2 *zte;            // test windows
    float store_scale;
};

template <int PREC>
__device__ __forceinline__ void store_train(void *z, int64_t idx, float2 v, float sc) {
    if constexpr (PREC == BS_PREC_FP32) {
        reinterpret_cast<float2 *>(z)[idx] = v;
    } else if constexpr (PREC == BS_PREC_FP16) {
        reinterpret_cast<__half2 *>(z)[idx] = __floats2half2_rn(v.x * sc, v.y * sc);
    } else {
        reinterpret_cast<__nv_bfloat162 *>(z)[idx] = __floats2bfloat162_rn(v.x * sc, v.y * sc);
    }
}

constexpr int kTabT = 256;   // targets whose gather entries are staged in shared memory

// Gather entry of one target for the current vector or group (16 bytes: one
// shared-memory load): window-array base, start | (W << 16), output count.
struct __align__(16) GatherEnt {
    long long base;
    int sw;
    int n;
};

// Gather entry of target t for a CTA at subband s whose first vector is v0:
// base element offset in the window array, start | (W << 16), output count.
__device__ __forceinline__ void fill_target_entry(const GatherArgs &ga, int t, int s, int v0, int nv,
                                                  bool train, long long *base, int *sw, int *nout,
                                                  int slot = -1) {
    const int i = slot < 0 ? t : slot;
    const int64_t g = (int64_t)t * ga.L + s;
    const int W = __ldg(&ga.Wg[g]);
    const int st = __ldg(&ga.start[g]);
    int n = nv * W;
    long long b;
    if (train) {
        const int K = __ldg(&ga.Kg[g]);
        n = (v0 >= K) ? 0 : min(n, (K - v0) * W);
        b = __ldg(&ga.ztr_off[g]) + (long long)v0 * W;
    } else {
        b = __ldg(&ga.zte_off[g]) + (long long)v0 * W;
    }
    base[i] = b;
    sw[i] = st | (W << 16);
    nout[i] = n;
}

// Persistent bulk-copy variant (beamspace_tma.cu); *used = false when the
// plan does not qualify (M outside 512 .. 4096, odd N, unaligned input,
// groups of vpb vectors crossing a subband, or BS_FLAG_NO_TMA).
bs_status launch_beamspace_tma(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                               bool *used);
// Warp-per-transform variant (beamspace_warp.cu) for M = 1024, 2048, 4096
// and N <= 1024; *used = false for other plans, more than kTabT targets,
// BS_FLAG_STAGED_FFT or BS_FLAG_NO_TMA.
bs_status launch_beamspace_warp(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                                bool *used);
// Tensor-core variant (beamspace_tc.cu) for N = 1024, M = 2048, B even,
// F (per shard) a multiple of 4 and at most kTabT targets; *used = false
// otherwise, or with BS_FLAG_SIMT_FFT, BS_FLAG_STAGED_FFT or BS_FLAG_NO_TMA.
bs_status launch_beamspace_tc(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                              bool *used);
// Planar arrays (beamspace2d.cu): 2-D transform and Wx x Wz window gather.
bs_status launch_beamspace2d(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st);

}  // namespace bs
