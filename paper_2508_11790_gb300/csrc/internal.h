// Plan object and launch helpers shared by the translation units of the
// library (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "bs.h"

namespace bs {
// Launch shape of the fused covariance + solve kernel (set by bs_autotune).
struct CovSolveLaunch {
    int threads = 128;      // threads per CTA (128)
    int ctas_per_sm = 5;
};
}  // namespace bs

struct bs_plan {
    bs_config cfg;              // host pointers cleared after create
    int B = 0, P = 0, Vte = 0, Wmax = 0, Kmax = 0, sumW = 0;
    // subbands of the plan: s0 .. s0 + Ls - 1 of the cfg.L (a shard, or all);
    // Fs = Ls B bins per record in the channelised cube
    int s0 = 0, Ls = 0, Fs = 0;
    int64_t pairs = 0;
    std::vector<int32_t> Wt, Kt;        // per target
    std::vector<double> u;              // per target
    // per pair (g = t * L + s)
    std::vector<int32_t> start, Wg, Kg;
    // planar arrays: vertical window start per pair, vertical window per target
    bool planar = false;
    int Nx = 0, Nz = 1, Mx = 0, Mz = 1;
    std::vector<int32_t> start_z, Wzt;
    int32_t *d_start_z = nullptr, *d_Wz = nullptr;
    std::vector<int64_t> woff, ztr_off, zte_off, roff;   // pairs + 1 entries
    std::vector<bs_cf64> at;                              // windowed steering, woff-packed
    int64_t ztr_elems = 0, zte_elems = 0, r_elems = 0, c_elems = 0;
    // beamspace gather: vectors per CTA and the (target, k) table of one CTA
    int vpb = 0;
    std::vector<int32_t> gather;        // [vpb * sumW]: (t << 10) | (c << 5) | w, target-major
    std::vector<int32_t> glist;         // [sumW]: (t << 8) | w, target-major (one vector)
    // per (subband, target), subband-major: {ztr_off, zte_off, start | W << 16, K}
    std::vector<int64_t> gsub;
    // device copies
    int device = 0;
    int32_t *d_start = nullptr, *d_Wg = nullptr, *d_Kg = nullptr, *d_gather = nullptr;
    int64_t *d_woff = nullptr, *d_ztr_off = nullptr, *d_zte_off = nullptr, *d_roff = nullptr;
    int64_t *d_gsub = nullptr;
    int32_t *d_glist = nullptr;
    float2 *d_at32 = nullptr;
    float2 *d_atlo = nullptr;                    // a~ - (float)a~ (double-float low parts)
    double2 *d_at64 = nullptr;
    float2 *d_twF = nullptr, *d_twM = nullptr;   // e^{-2 pi i k / F}, e^{-2 pi i k / M}
    int *d_err = nullptr;                        // device error word (bit 0: a bounded wait gave up)
    // bs_run_host: copy stream and events of its record-chunk pipeline
    static constexpr int kHostChunks = 8;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_start = nullptr, ev_chunk[kHostChunks] = {};
    // the stand-alone solve's window-size launches run on `stream` and these
    // side streams (forked from and joined back into `stream`)
    static constexpr int kSolveStreams = 4;
    cudaStream_t solve_st[kSolveStreams] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kSolveStreams] = {};
    int num_sms = 0;
    // fused covariance + solve: queue order (decreasing W^2 K), workspace head
    std::vector<int32_t> order;
    int32_t *d_order = nullptr;
    // stand-alone solve: pairs grouped by W (stable), its visiting order
    std::vector<int32_t> order_w;
    int32_t *d_order_w = nullptr;
    int Wmin = 0;
    int64_t nsmall = 0;   // pairs with W <= 16 (the first of order_w)
    int64_t wstart[34] = {};   // pairs of window size W are slots wstart[W] .. wstart[W + 1] - 1 of order_w
    int *d_head = nullptr;
    bs::CovSolveLaunch cs;
    // kernel variants chosen by bs_autotune_pass (-1: the built-in choice)
    int tune_beamspace = -1;   // 0 warp per residue, 1 bulk-copy staged, 2 one-shot
    int tune_cov = -1;         // 0 CTA per pair, 1 warp per pair, 2 tensor cores
    int tune_fused = -1;       // 0 covariance + solve as two launches, 1 one persistent launch
};

namespace bs {

bs_status set_error(bs_status s, const std::string &msg);
bs_status cuda_error(cudaError_t e, const char *where);
bs_status check_launch(const char *where);

// Launch settings that a kernel needs once per device: function attributes
// (the dynamic shared-memory limit) and occupancy apply to the current device
// only, so a process that uses several GPUs sets them on each.  get() runs
// init(&value) under a lock the first time the current device asks, caches
// the value for that device, and returns it in *out (may be NULL).
struct PerDevice {
    static constexpr int kMaxDevices = 64;
    std::mutex mu;
    bool done[kMaxDevices] = {};
    int val[kMaxDevices] = {};
    template <class Init>
    bs_status get(Init &&init, int *out = nullptr) {
        int dev = 0;
        const cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
        if (dev < 0 || dev >= kMaxDevices) return set_error(BS_EUNSUPPORTED, "device index above 63");
        std::lock_guard<std::mutex> lock(mu);
        if (!done[dev]) {
            int v = 0;
            if (const bs_status s = init(&v)) return s;
            val[dev] = v;
            done[dev] = true;
        }
        if (out) *out = val[dev];
        return BS_OK;
    }
};

// kernel launchers (one per translation unit)
bs_status launch_channelize(const bs_plan *p, const float2 *x, int P, float2 *xc, cudaStream_t st);
// records p0 .. p0+np-1 (np < 0: through the last record)
bs_status launch_beamspace(const bs_plan *p, const float2 *xc, void *ztr, float2 *zte, cudaStream_t st, int p0 = 0,
                           int np = -1);
bs_status launch_beamspace_full(const bs_plan *p, const float2 *y, int64_t nvec, float2 *yb,
                                cudaStream_t st);
// The covariance launcher's choice for this plan is the warp-per-pair kernel.
bool window_cov_uses_warp(const bs_plan *p);
// Warp-per-pair covariance of slots [slot0, slot1) of `order` (pair order if null).
bs_status launch_window_cov_warp(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                                 cudaStream_t st, int64_t slot0, int64_t slot1, const int32_t *order);
// Covariance and stand-alone solve as one chain per window size, the chains
// in parallel (plan side streams); applies to plans whose covariance takes
// the warp-per-pair kernel, with several window sizes, all at most 16 beams.
bool cov_solve_chains_apply(const bs_plan *p);
bs_status launch_cov_solve_chains(const bs_plan *p, const void *ztr, double2 *R, float2 *c, int32_t *info,
                                  cudaStream_t st);
bs_status launch_window_cov(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                            cudaStream_t st);
bs_status launch_window_cov_mma(const bs_plan *p, const void *ztr, const float *delta, double2 *R,
                                cudaStream_t st);
// dpre: optional diagonal preconditioner [c_elems] (woff-packed), NULL for none
bs_status launch_mvdr_solve(const bs_plan *p, const double2 *R, float2 *c, int32_t *info,
                            cudaStream_t st, const float *dpre = nullptr);
bs_status launch_apply(const bs_plan *p, const float2 *zte, const float2 *c, float2 *out,
                       cudaStream_t st);
bs_status launch_cov_solve(const bs_plan *p, const void *ztr, const float *delta, double2 *R, float2 *c,
                           int32_t *info, int *head, const CovSolveLaunch &cfg, cudaStream_t st);
bs_status launch_cov_solve_tables(const void *z, int precision, float store_scale, const int32_t *Wg,
                                  const int32_t *Kg, const int64_t *ztr_off, const int64_t *woff,
                                  const float2 *at32, const float2 *atlo, const double2 *at64,
                                  const int32_t *order, int64_t pairs, double delta, double kappa_max,
                                  uint32_t flags, float2 *c, int32_t *info, int *head, int grid,
                                  cudaStream_t st);
int beamspace_vectors_per_cta(int M);
// the tensor-core beamspace kernel serves this plan (beamspace_tc.cu)
bool beamspace_tc_applies(const bs_plan *p);
bs_status launch_lift(const bs_plan *p, const float2 *c, float2 *c_hat, cudaStream_t st);
// orthonormal F-point DFT of nvec contiguous rows of F elements (F-point twiddle table)
bs_status launch_fft_rows(const bs_plan *p, const float2 *y, int64_t nvec, float2 *yb, cudaStream_t st);
bs_status launch_range_doppler(const bs_plan *p, const float2 *out, const float2 *pulse, float2 *work, float *map,
                               cudaStream_t st);
bs_status launch_cfar(const bs_plan *p, const float *map, float threshold_db, float *floor, int32_t *count,
                      uint8_t *mask, int32_t *peak, cudaStream_t st);
bs_status launch_apply_lifted(const bs_plan *p, const float2 *xc, const float2 *c_hat, float2 *out,
                              cudaStream_t st);
bs_status launch_beam_pattern(const bs_plan *p, const float2 *c_hat, int n_dirs, const double *u, float *pattern,
                              cudaStream_t st);

}  // namespace bs
