// Allocation-free variant of the fused covariance + MVDR solve.
//
// Who needs it: callers that must not allocate device memory once they are
// running, for example a real-time radar processing loop whose memory is
// fixed at start-up (a device allocation can stall the whole device), or a
// host application that owns every device buffer and forbids libraries to
// allocate.  Such callers cannot create a bs_plan either (plan creation
// allocates its tables), so this entry point takes every per-pair table from
// the caller and keeps its own scratch in a fixed array in device memory.
//
// Scratch: g_nalloc_scratch below holds the work-queue head and the pair
// order of the queue (pairs sorted by decreasing W^2 K).  It has room for
// kNallocMaxPairs pairs; larger requests are refused.  The array exists on
// every GPU that loads this library, for the life of the process.  All
// calls share it: two calls whose kernels overlap on the GPU (different
// streams, or different host threads on one device) race on it and must not
// be issued.  Each call rewrites the parts it uses (head and order list) in
// its first kernel, so stale contents from an earlier call do no harm.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace bs {

constexpr int64_t kNallocMaxPairs = 1 << 18;   // 262144 pairs
constexpr int kNallocHdr = 64;                 // int32 slots before the order list; [0] = queue head

static __device__ __align__(256) int32_t g_nalloc_scratch[kNallocHdr + kNallocMaxPairs];

// Builds the queue in the scratch array: pairs whose table entry is out of
// range (W outside 1..16, K outside 1..2^24 - 1; the covariance scale 1/K is
// formed as a double-float that is exact only below 2^24) are placed first and skipped by setting
// the head past them (info = -3); the others follow in decreasing order of
// log2(W^2 K) (counting sort in shared memory, one CTA).
__global__ void __launch_bounds__(1024)
    nalloc_order_kernel(const int32_t *__restrict__ Wg, const int32_t *__restrict__ Kg, int64_t pairs,
                        int32_t *__restrict__ info) {
    constexpr int NB = 40;   // bucket 0: invalid; 1.. by decreasing cost
    __shared__ int cnt[NB], cur[NB];
    const int tid = threadIdx.x;
    if (tid < NB) cnt[tid] = 0;
    __syncthreads();
    auto bucket = [&](int64_t g) -> int {
        const int W = Wg[g], K = Kg[g];
        if (W < 1 || W > 16 || K < 1 || K >= (1 << 24)) return 0;
        const long long cost = (long long)W * W * K;   // < 2^32
        const int lg = 63 - __clzll(cost);             // 0 .. 31
        return NB - 1 - lg;                            // 8 .. 39, larger cost first
    };
    for (int64_t g = tid; g < pairs; g += blockDim.x) atomicAdd(&cnt[bucket(g)], 1);
    __syncthreads();
    if (tid == 0) {
        int s = 0;
        for (int b = 0; b < NB; ++b) {
            cur[b] = s;
            s += cnt[b];
        }
        g_nalloc_scratch[0] = cnt[0];   // queue head: skip the invalid pairs
    }
    __syncthreads();
    for (int64_t g = tid; g < pairs; g += blockDim.x) {
        const int b = bucket(g);
        const int pos = atomicAdd(&cur[b], 1);
        g_nalloc_scratch[kNallocHdr + pos] = (int32_t)g;
        if (b == 0) info[g] = -3;
    }
}

// Device address of the scratch array on the current device.  Host code
// only holds a stand-in for the array's name, so the address is looked up
// once per device (with that device current) and cached.
static std::mutex g_nalloc_mu;
static int32_t *g_nalloc_ptr[256] = {};

static bs_status nalloc_scratch(int dev, int32_t **out) {
    if (dev < 0 || dev >= 256) return set_error(BS_EUNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_nalloc_mu);
    if (!g_nalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_nalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        g_nalloc_ptr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_nalloc_ptr[dev];
    return BS_OK;
}

}  // namespace bs

using bs::set_error;

extern "C" bs_status bs_cov_solve_noalloc(const void *z_train, int32_t precision, float store_scale,
                                          const int32_t *W, const int32_t *K, const int64_t *ztr_off,
                                          const int64_t *woff, const bs_cf32 *a_hi, const bs_cf32 *a_lo,
                                          const bs_cf64 *a_fp64, int64_t pairs, double delta, double kappa_max,
                                          uint32_t flags, bs_cf32 *c, int32_t *info, bs_stream stream) {
    if (pairs < 0) return set_error(BS_EINVAL, "pairs must be >= 0");
    if (pairs > bs::kNallocMaxPairs)
        return set_error(BS_EINVAL, "bs_cov_solve_noalloc: pairs exceeds its fixed scratch of 262144 pairs");
    if (precision < BS_PREC_FP32 || precision > BS_PREC_BF16) return set_error(BS_EINVAL, "unknown precision");
    if (!(delta >= 0.0) || !std::isfinite(delta)) return set_error(BS_EINVAL, "delta must be finite and >= 0");
    if (pairs == 0) return BS_OK;
    if (!z_train || !W || !K || !ztr_off || !woff || !a_hi || !a_lo || !a_fp64 || !c || !info)
        return set_error(BS_EINVAL, "NULL buffer");
    if (!(store_scale > 0.f)) store_scale = 1.0f;
    if (!(kappa_max > 0.0)) kappa_max = 1e5;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bs::cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bs::cuda_error(e, "device attribute");
    int32_t *scr = nullptr;
    if (bs_status s = bs::nalloc_scratch(dev, &scr)) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    bs::nalloc_order_kernel<<<1, 1024, 0, st>>>(W, K, pairs, info);
    if (bs_status s = bs::check_launch("queue order launch")) return s;
    long long grid = (long long)sms * 5;
    if (grid > pairs) grid = pairs;
    return bs::launch_cov_solve_tables(z_train, precision, store_scale, W, K, ztr_off, woff,
                                       reinterpret_cast<const float2 *>(a_hi),
                                       reinterpret_cast<const float2 *>(a_lo),
                                       reinterpret_cast<const double2 *>(a_fp64), scr + bs::kNallocHdr, pairs,
                                       delta, kappa_max, flags, reinterpret_cast<float2 *>(c), info, scr,
                                       (int)grid, st);
}
