// Warp-per-transform beamspace kernel for M = 1024 r (r = 1, 2, 4) and
// N <= 1024 (Eq. VerDFT, Eq. BeamTransform, Eq. OverallWindow,
// Eq. ApplyWindow).
//
// Same result as the other beamspace kernels (every (record, bin) vector
// zero-padded to M points, M-point DFT scaled by 1/sqrt(M), the W_t beams
// start_g + w (mod M) of every target written to the packed window arrays),
// with the transform split so that one warp owns it and no CTA barrier is
// needed.  With n = 32 n1 + n2 (n < 1024) and beams m = r k1 + c + 32 r m2:
//
//   X[m] = sum_n2 W_32^(n2 m2) W_M^(n2 (r k1 + c)) sum_n1 x[32 n1 + n2] W_(32 r)^(c n1) W_32^(n1 k1)
//
// so residue c = m mod r of the beams is two 32-point DFTs: lane n2 takes
// the 32 inputs of its column straight from HBM (one 256-byte coalesced
// load per n1), multiplies them by W_(32 r)^(c n1) (a row of a shared table,
// read as a broadcast), runs a 32-point DFT in registers and the twiddles
// W_M^(n2 (r k1 + c)) (a shared table), and writes row k1 of a padded
// 32 x 33 transpose buffer; lane k1 then reads its row, runs the second
// 32-point DFT and writes the 32 beams back to the same row.  All
// warps run one code path (c is a run-time value): a code copy per residue
// doubled the instruction-cache misses.  The r residues of one vector are r
// warps of a CTA, which meet at a named barrier and split the window gather
// between them, consecutive lanes taking consecutive entries of a target's
// window so that the stores are contiguous.  The next vector's inputs are
// loaded into the freed registers before the gather, so the loads overlap it.
//
// Shared memory per CTA: the twiddle tables (r x 8.25 KB), eight 32 x 33
// transpose buffers (66 KB) and, per vector in flight, the T per-target
// gather entries of 16 bytes: two CTAs of 256 threads per SM.
#include "beamspace_dev.cuh"
#include "internal.h"

#include <algorithm>

namespace bs {

namespace {

constexpr int kRow = 33;                // padded row of the 32 x 32 transpose
constexpr int kBuf = 32 * kRow;         // float2 per warp
// Distance between the buffers of one vector's residues: 8 float2 (16
// banks) more than a buffer, so that the gather's reads of beams 2k and
// 2k + 1 (residues 0 and 1 at the same offset) fall in different banks.
constexpr int kBufS = kBuf + 8;
constexpr int kWarpGatherRegs = 12;     // gather entries per lane held in registers
constexpr int kBatch = 4;               // gather entries whose loads are issued together

// cos(2 pi j / 128), j = 0 .. 32
__host__ __device__ constexpr float cos128(int j) {
    switch (j) {
        case 0: return 1.0f;
        case 1: return 0.99879545620517241f;
        case 2: return 0.99518472667219693f;
        case 3: return 0.98917650996478101f;
        case 4: return 0.98078528040323043f;
        case 5: return 0.97003125319454397f;
        case 6: return 0.95694033573220882f;
        case 7: return 0.94154406518302081f;
        case 8: return 0.92387953251128674f;
        case 9: return 0.90398929312344334f;
        case 10: return 0.88192126434835505f;
        case 11: return 0.85772861000027212f;
        case 12: return 0.83146961230254524f;
        case 13: return 0.80320753148064494f;
        case 14: return 0.77301045336273699f;
        case 15: return 0.74095112535495911f;
        case 16: return 0.70710678118654757f;
        case 17: return 0.67155895484701833f;
        case 18: return 0.63439328416364549f;
        case 19: return 0.59569930449243347f;
        case 20: return 0.55557023301960229f;
        case 21: return 0.51410274419322166f;
        case 22: return 0.47139673682599781f;
        case 23: return 0.42755509343028220f;
        case 24: return 0.38268343236508984f;
        case 25: return 0.33688985339222005f;
        case 26: return 0.29028467725446233f;
        case 27: return 0.24298017990326398f;
        case 28: return 0.19509032201612833f;
        case 29: return 0.14673047445536175f;
        case 30: return 0.09801714032956077f;
        case 31: return 0.049067674327418126f;
        default: return 0.0f;
    }
}

// x * exp(-2 pi i e / D) for D | 128; e is a compile-time constant at every
// call site (fully unrolled loops), so the branches fold away.
template <int D>
__device__ __forceinline__ float2 twiddle_d(int e, float2 x) {
    static_assert(128 % D == 0, "D must divide 128");
    const int k = (e * (128 / D)) & 127;
    const int q = k >> 5, j = k & 31;
    float2 y = x;
    if (j != 0) {
        const float c = cos128(j), s = cos128(32 - j);   // angle 2 pi j / 128
        y = make_float2(x.x * c + x.y * s, x.y * c - x.x * s);
    }
    switch (q) {   // times (-i)^q
        case 0: return y;
        case 1: return make_float2(y.y, -y.x);
        case 2: return make_float2(-y.x, -y.y);
        default: return make_float2(-y.y, y.x);
    }
}

// 32-point forward DFT in registers, natural order in and out: one radix-2
// decimation-in-frequency stage, then two 16-point DFTs.
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    float2 e[16], o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        e[k] = cadd(v[k], v[k + 16]);
        o[k] = twiddle_d<32>(k, csub(v[k], v[k + 16]));
    }
    RegDFT<16>::run(e);
    RegDFT<16>::run(o);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[2 * k] = e[k];
        v[2 * k + 1] = o[k];
    }
}

// barrier of the R warps of one vector slot (named barrier 1 + slot; the
// identifiers are immediates so that the kernel reserves only the ones it uses)
template <int R>
__device__ __forceinline__ void group_sync(int slot) {
    if constexpr (R == 1) {
        __syncwarp();
    } else {
        switch (slot) {
            case 0: asm volatile("bar.sync 1, %0;" ::"n"(32 * R) : "memory"); break;
            case 1: asm volatile("bar.sync 2, %0;" ::"n"(32 * R) : "memory"); break;
            case 2: asm volatile("bar.sync 3, %0;" ::"n"(32 * R) : "memory"); break;
            default: asm volatile("bar.sync 4, %0;" ::"n"(32 * R) : "memory"); break;
        }
    }
}

struct WarpArgs {
    const float2 *y;
    int N;
    float scale, sc_tr;
    int prec;
    const int32_t *glist;   // [sumW]: (t << 8) | w, target-major
    int sumW;
};

// One warp: residue CC of the beams of vectors vec, vec + vstride, ...
// (kFull: N = 1024, no tail predicates).
template <int R, bool kFull, int PREC>
__device__ __forceinline__ void warp_units(const WarpArgs &wa, const GatherArgs &ga, const float2 *tw,
                                           const float2 *ptw, float2 *grp, GatherEnt *tab,
                                           const int (&gent)[kWarpGatherRegs], int slot, int CC, int64_t vec,
                                           int64_t vstride) {
    constexpr int M = 1024 * R;
    constexpr int log2r = (R == 1) ? 0 : (R == 2 ? 1 : 2);
    const int lane = threadIdx.x & 31;
    float2 *buf = grp + CC * kBufS;
    const float2 *twc = tw + CC * 1024;
    const float2 *ptc = ptw + CC * 32;
    // the inter-stage twiddles of this lane, W_M^(n2 (R k1 + CC)), are a
    // geometric sequence in k1 with ratio rho = W_M^(n2 R): read every 8th
    // from the table and step 7 times by rho (at most 7 roundings)
    const float2 rho0 = tw[32 + lane];   // W_M^(n2 R) (the table's residue-0 row k1 = 1)
    float2 a[32];
    auto load = [&](int64_t v) {   // column n2 = lane of vector v
        const float2 *src = wa.y + v * wa.N + lane;
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            if constexpr (kFull) a[n1] = __ldcg(src + 32 * n1);
            else a[n1] = (32 * n1 + lane < wa.N) ? __ldcg(src + 32 * n1) : make_float2(0.f, 0.f);
        }
    };
    auto put = [&](long long idx, float2 val, bool train) {
        if (!train) {
            ga.zte[idx] = cscale(val, wa.scale);
        } else if constexpr (PREC == BS_PREC_FP32) {
            store_train<BS_PREC_FP32>(ga.ztr, idx, cscale(val, wa.sc_tr), 1.f);
        } else {
            store_train<PREC>(ga.ztr, idx, val, wa.sc_tr);
        }
    };
    if (vec < ga.nvec) load(vec);
    for (; vec < ga.nvec; vec += vstride) {
        // pass 1: residue CC of a (32 R)-point DFT along n1, then the twiddles
        if constexpr (R == 2) {   // W_64^(n1) for residue 1: compile-time constants
            if (CC == 1) {
#pragma unroll
                for (int n1 = 1; n1 < 32; ++n1) a[n1] = twiddle_d<64>(n1, a[n1]);
            }
        } else if (R > 1 && CC != 0) {   // W_(32 R)^(CC n1): one broadcast table row
#pragma unroll
            for (int n1 = 1; n1 < 32; ++n1) a[n1] = cmul(a[n1], ptc[n1]);
        }
        dft32(a);
#pragma unroll
        for (int k8 = 0; k8 < 32; k8 += 8) {
            float2 t = twc[k8 * 32 + lane];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i) t = cmul(t, rho0);
                buf[(k8 + i) * kRow + lane] = cmul(a[k8 + i], t);
            }
        }
        // this vector's per-target entries, split over the R warps
        const int64_t v = ga.vbase + vec;
        const int p = (int)(v >> ga.log2F);
        const int q = (int)(v & ((1 << ga.log2F) - 1));
        const int sb = q >> ga.log2B;
        const int i = q & ((1 << ga.log2B) - 1);
        const bool train = p < ga.P_train;
        const int v0 = train ? (p << ga.log2B) + i : ((p - ga.P_train) << ga.log2B) + i;
        for (int t = CC * 32 + lane; t < ga.T; t += 32 * R) {
            const longlong2 *gs = ga.gsub + 2 * ((int64_t)sb * ga.T + t);
            const longlong2 o = __ldg(gs), m = __ldg(gs + 1);
            const int W = (int)(m.x >> 16);
            const int n = (train && v0 >= (int)m.y) ? 0 : W;
            tab[t] = GatherEnt{(train ? o.x : o.y) + (long long)v0 * W, (int)m.x, n};
        }
        __syncwarp();
        // pass 2: row k1 = lane, 32-point DFT along n2; beams back to the row
#pragma unroll
        for (int n2 = 0; n2 < 32; ++n2) a[n2] = buf[lane * kRow + n2];
        dft32(a);
#pragma unroll
        for (int m2 = 0; m2 < 32; ++m2) buf[lane * kRow + m2] = a[m2];

        if (vec + vstride < ga.nvec) load(vec + vstride);   // overlaps the gather
        group_sync<R>(slot);   // all residues' beams and the entries are in place

        // entries in batches of kBatch: every shared-memory read of a batch
        // is issued before its stores (a dependent chain per entry otherwise);
        // a missing entry (-1) reads target 0's entry and stores nothing
        auto batch = [&](const int *pk) {
            float2 val[kBatch];
            long long gi[kBatch];
            bool ok[kBatch];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int packed = pk[j];
                const int t = packed < 0 ? 0 : packed >> 8, w = packed & 255;
                const GatherEnt te = tab[t];
                ok[j] = packed >= 0 && w < te.n;
                const int m = ((te.sw & 0xFFFF) + w) & (M - 1);
                const int kk = m >> log2r;
                // entries that store nothing (training vectors past the
                // target's K) skip the shared-memory read
                val[j] = ok[j] ? grp[(m & (R - 1)) * kBufS + (kk & 31) * kRow + (kk >> 5)] : make_float2(0.f, 0.f);
                gi[j] = te.base + w;
            }
#pragma unroll
            for (int j = 0; j < kBatch; ++j)
                if (ok[j]) put(gi[j], val[j], train);
        };
#pragma unroll
        for (int j = 0; j < kWarpGatherRegs; j += kBatch) batch(gent + j);
        for (int e = (kWarpGatherRegs * R + CC) * 32 + lane; e < wa.sumW; e += kBatch * 32 * R) {
            int pk[kBatch];
#pragma unroll
            for (int j = 0; j < kBatch; ++j) {
                const int ej = e + j * 32 * R;
                pk[j] = ej < wa.sumW ? __ldg(&wa.glist[ej]) : -1;
            }
            batch(pk);
        }
        group_sync<R>(slot);   // buffers and entries free for the next vector
    }
}

template <int R, bool kFull, int PREC>
__global__ void __launch_bounds__(256, 2)
    beamspace_warp_kernel(WarpArgs wa, GatherArgs ga, const float2 *__restrict__ twM) {
    constexpr int M = 1024 * R, vpc = 8 / R;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *tw = reinterpret_cast<float2 *>(smraw);    // [R][32 k1][32 n2]
    float2 *ptw = tw + R * 1024;                       // [R][32 n1]
    float2 *bufs = ptw + R * 32;                       // [8 warps][kBufS]
    GatherEnt *tabs = reinterpret_cast<GatherEnt *>(bufs + 8 * kBufS);   // [vpc][T]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = warp / R, cc = warp % R;
    for (int e = tid; e < R * 1024; e += 256) {
        const int c = e >> 10, k1 = (e >> 5) & 31, n2 = e & 31;
        tw[e] = __ldg(&twM[(n2 * (R * k1 + c)) & (M - 1)]);
    }
    for (int e = tid; e < R * 32; e += 256) ptw[e] = __ldg(&twM[(32 * (e >> 5) * (e & 31)) & (M - 1)]);
    int gent[kWarpGatherRegs];   // entries (j R + cc) 32 + lane of the list
#pragma unroll
    for (int j = 0; j < kWarpGatherRegs; ++j) {
        const int e = (j * R + cc) * 32 + lane;
        gent[j] = (e < wa.sumW) ? __ldg(&wa.glist[e]) : -1;
    }
    __syncthreads();
    float2 *grp = bufs + slot * R * kBufS;
    GatherEnt *tab = tabs + slot * ga.T;
    const int64_t vec = (int64_t)blockIdx.x * vpc + slot;
    const int64_t vstride = (int64_t)gridDim.x * vpc;
    warp_units<R, kFull, PREC>(wa, ga, tw, ptw, grp, tab, gent, slot, cc, vec, vstride);
}

template <int R, bool kFull, int PREC>
bs_status launch_warp_t(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st) {
    constexpr int vpc = 8 / R;
    const size_t fixed = (size_t)R * 1056 * sizeof(float2) + 8 * (size_t)kBufS * sizeof(float2);
    const size_t smem = fixed + (size_t)vpc * ga.T * sizeof(GatherEnt);
    const size_t smem_max = fixed + (size_t)vpc * kTabT * sizeof(GatherEnt);
    static PerDevice occ;
    int blocks_per_sm = 1;
    if (bs_status s = occ.get(
            [&](int *v) {
                cudaError_t e = cudaFuncSetAttribute(beamspace_warp_kernel<R, kFull, PREC>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
                if (e != cudaSuccess) return cuda_error(e, "beamspace (warp) attribute");
                int nb = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, beamspace_warp_kernel<R, kFull, PREC>, 256,
                                                                  smem_max);
                if (e != cudaSuccess) return cuda_error(e, "beamspace (warp) occupancy");
                *v = std::max(nb, 1);
                return BS_OK;
            },
            &blocks_per_sm))
        return s;
    const int64_t groups = (ga.nvec + vpc - 1) / vpc;
    if (groups == 0) return BS_OK;
    const int grid = (int)std::min<int64_t>(groups, (int64_t)p->num_sms * blocks_per_sm);
    WarpArgs wa;
    wa.y = xc;
    wa.N = p->cfg.N;
    wa.scale = 1.0f / sqrtf((float)(1024 * R));
    wa.prec = p->cfg.precision;
    wa.sc_tr = (wa.prec == BS_PREC_FP32) ? wa.scale : wa.scale * ga.store_scale;
    wa.glist = p->d_glist;
    wa.sumW = p->sumW;
    beamspace_warp_kernel<R, kFull, PREC><<<grid, 256, smem, st>>>(wa, ga, p->d_twM);
    return check_launch("beamspace (warp) launch");
}

template <int PREC>
bs_status launch_warp_p(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st) {
    const int M = p->cfg.M;
    const bool full = p->cfg.N == 1024;
    if (M == 1024) return full ? launch_warp_t<1, true, PREC>(p, xc, ga, st) : launch_warp_t<1, false, PREC>(p, xc, ga, st);
    if (M == 2048) return full ? launch_warp_t<2, true, PREC>(p, xc, ga, st) : launch_warp_t<2, false, PREC>(p, xc, ga, st);
    return full ? launch_warp_t<4, true, PREC>(p, xc, ga, st) : launch_warp_t<4, false, PREC>(p, xc, ga, st);
}

}  // namespace

bs_status launch_beamspace_warp(const bs_plan *p, const float2 *xc, const GatherArgs &ga, cudaStream_t st,
                                bool *used) {
    *used = false;
    const int M = p->cfg.M;
    if ((p->cfg.flags & (BS_FLAG_NO_TMA | BS_FLAG_STAGED_FFT)) || p->cfg.N > 1024 || ga.T > kTabT ||
        (M != 1024 && M != 2048 && M != 4096))
        return BS_OK;
    *used = true;
    switch (p->cfg.precision) {
        case BS_PREC_FP32: return launch_warp_p<BS_PREC_FP32>(p, xc, ga, st);
        case BS_PREC_FP16: return launch_warp_p<BS_PREC_FP16>(p, xc, ga, st);
        default: return launch_warp_p<BS_PREC_BF16>(p, xc, ga, st);
    }
}

}  // namespace bs
