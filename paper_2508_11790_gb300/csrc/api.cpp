// extern "C" entry points of the hot path: argument checks, then the
// kernel launchers of the individual translation units.
#include <algorithm>
#include <string>
#include <vector>

#include "host_chunks.h"
#include "internal.h"

using bs::set_error;

static bs_status check_device(const bs_plan *p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bs::cuda_error(e, "cudaGetDevice");
    if (dev != p->device) return set_error(BS_EINVAL, "current device differs from the plan's device");
    return BS_OK;
}

// Covariance and solve as one persistent launch: the plan flag, unless
// bs_autotune_pass has chosen.
static bool use_fused(const bs_plan *p) {
    return p->tune_fused >= 0 ? p->tune_fused == 1 : (p->cfg.flags & BS_FLAG_FUSED) != 0;
}

#define BS_REQUIRE(cond, msg)                                  \
    do {                                                       \
        if (!(cond)) return set_error(BS_EINVAL, (msg));       \
    } while (0)

extern "C" {

bs_status bs_channelize(const bs_plan *p, const bs_cf32 *x, int32_t P, bs_cf32 *xc, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(P >= 0, "P must be >= 0");
    if (P == 0) return BS_OK;
    BS_REQUIRE(x && xc, "NULL buffer");
    BS_REQUIRE((const void *)x != (const void *)xc, "x and xc must be distinct");
    BS_REQUIRE(P <= 65535, "at most 65535 records per call");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_channelize(p, (const float2 *)x, P, (float2 *)xc, (cudaStream_t)stream);
}

bs_status bs_beamspace(const bs_plan *p, const bs_cf32 *xc, void *z_train, bs_cf32 *z_test, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(xc && z_train, "NULL buffer");
    BS_REQUIRE(z_test || p->cfg.P_test == 0, "z_test is NULL but P_test > 0");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_beamspace(p, (const float2 *)xc, z_train, (float2 *)z_test, (cudaStream_t)stream);
}

bs_status bs_beamspace_full(const bs_plan *p, const bs_cf32 *y, int64_t nvec, bs_cf32 *yb, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->planar) return set_error(BS_EUNSUPPORTED, "bs_beamspace_full: linear arrays only");
    BS_REQUIRE(nvec >= 0, "nvec must be >= 0");
    if (nvec == 0) return BS_OK;
    BS_REQUIRE(y && yb, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_beamspace_full(p, (const float2 *)y, nvec, (float2 *)yb, (cudaStream_t)stream);
}

bs_status bs_window_cov(const bs_plan *p, const void *z_train, const float *delta_pair, bs_cf64 *R,
                        bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(z_train && R, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_window_cov(p, z_train, delta_pair, (double2 *)R, (cudaStream_t)stream);
}

bs_status bs_mvdr_solve(const bs_plan *p, const bs_cf64 *R, bs_cf32 *c, int32_t *info, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(R && c && info, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_mvdr_solve(p, (const double2 *)R, (float2 *)c, info, (cudaStream_t)stream);
}

bs_status bs_mvdr_solve_precond(const bs_plan *p, const bs_cf64 *R, const float *d, bs_cf32 *c, int32_t *info,
                                bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(R && d && c && info, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_mvdr_solve(p, (const double2 *)R, (float2 *)c, info, (cudaStream_t)stream, d);
}

bs_status bs_apply(const bs_plan *p, const bs_cf32 *z_test, const bs_cf32 *c, bs_cf32 *out, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->Vte == 0) return BS_OK;
    BS_REQUIRE(z_test && c && out, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_apply(p, (const float2 *)z_test, (const float2 *)c, (float2 *)out, (cudaStream_t)stream);
}

bs_status bs_lift(const bs_plan *p, const bs_cf32 *c, bs_cf32 *c_hat, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->planar) return set_error(BS_EUNSUPPORTED, "bs_lift: linear arrays only");
    BS_REQUIRE(c && c_hat, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_lift(p, (const float2 *)c, (float2 *)c_hat, (cudaStream_t)stream);
}

bs_status bs_apply_lifted(const bs_plan *p, const bs_cf32 *xc, const bs_cf32 *c_hat, bs_cf32 *out,
                          bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->planar) return set_error(BS_EUNSUPPORTED, "bs_apply_lifted: linear arrays only");
    if (p->Vte == 0) return BS_OK;
    BS_REQUIRE(xc && c_hat && out, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_apply_lifted(p, (const float2 *)xc, (const float2 *)c_hat, (float2 *)out,
                                   (cudaStream_t)stream);
}

bs_status bs_beam_pattern(const bs_plan *p, const bs_cf32 *c_hat, int32_t n_dirs, const double *u, float *pattern,
                          bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->planar) return set_error(BS_EUNSUPPORTED, "bs_beam_pattern: linear arrays only");
    BS_REQUIRE(n_dirs >= 0, "n_dirs must be >= 0");
    if (n_dirs == 0) return BS_OK;
    BS_REQUIRE(c_hat && u && pattern, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_beam_pattern(p, (const float2 *)c_hat, n_dirs, u, pattern, (cudaStream_t)stream);
}

bs_status bs_range_doppler(const bs_plan *p, const bs_cf32 *out, const bs_cf32 *pulse, bs_cf32 *work, float *map,
                           bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->Ls != p->cfg.L)
        return set_error(BS_EUNSUPPORTED, "bs_range_doppler: a subband shard lacks the other subbands of each target");
    if (p->Vte == 0) return BS_OK;
    BS_REQUIRE(out && pulse && work && map, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_range_doppler(p, (const float2 *)out, (const float2 *)pulse, (float2 *)work, map,
                                    (cudaStream_t)stream);
}

bs_status bs_cfar(const bs_plan *p, const float *map, float threshold_db, float *floor, int32_t *count,
                  uint8_t *mask, int32_t *peak, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    if (p->Vte == 0) return BS_OK;
    if (p->cfg.P_test < 2) return set_error(BS_EUNSUPPORTED, "bs_cfar: a CFAR across velocity bins needs P_test >= 2");
    BS_REQUIRE(map && floor && count, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_cfar(p, map, threshold_db, floor, count, mask, peak, (cudaStream_t)stream);
}

bs_status bs_cov_solve(const bs_plan *p, const void *z_train, const float *delta_pair, bs_cf64 *R, bs_cf32 *c,
                       int32_t *info, bs_stream stream) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(z_train && c && info, "NULL buffer");
    if (bs_status s = check_device(p)) return s;
    return bs::launch_cov_solve(p, z_train, delta_pair, (double2 *)R, (float2 *)c, info, p->d_head, p->cs,
                                (cudaStream_t)stream);
}

bs_status bs_run(const bs_plan *p, const bs_buffers *b, bs_stream stream) {
    BS_REQUIRE(p && b, "NULL argument");
    bs_status s;
    if ((s = bs_channelize(p, b->x, p->P, b->xc, stream))) return s;
    if ((s = bs_beamspace(p, b->xc, b->z_train, b->z_test, stream))) return s;
    if (use_fused(p)) {
        if ((s = bs_cov_solve(p, b->z_train, nullptr, b->R, b->c, b->info, stream))) return s;
    } else if (bs::cov_solve_chains_apply(p)) {
        // several window sizes on the warp-per-pair covariance: one
        // covariance + solve chain per size, the chains in parallel
        BS_REQUIRE(b->z_train && b->R && b->c && b->info, "NULL buffer");
        if ((s = check_device(p))) return s;
        if ((s = bs::launch_cov_solve_chains(p, b->z_train, (double2 *)b->R, (float2 *)b->c, b->info,
                                             (cudaStream_t)stream)))
            return s;
    } else {
        if ((s = bs_window_cov(p, b->z_train, nullptr, b->R, stream))) return s;
        if ((s = bs_mvdr_solve(p, b->R, b->c, b->info, stream))) return s;
    }
    return bs_apply(p, b->z_test, b->c, b->out, stream);
}

struct bs_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

bs_status bs_graph_create(const bs_plan *p, const bs_buffers *b, bs_stream stream, bs_graph **out) {
    BS_REQUIRE(p && b && out, "NULL argument");
    BS_REQUIRE(stream, "graph capture needs a non-default stream");
    *out = nullptr;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bs::cuda_error(e, "begin capture");
    const bs_status rs = bs_run(p, b, stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (rs) {
        if (g) cudaGraphDestroy(g);
        return rs;
    }
    if (e != cudaSuccess) return bs::cuda_error(e, "end capture");
    bs_graph *gr = new bs_graph();
    gr->graph = g;
    e = cudaGraphInstantiate(&gr->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        delete gr;
        return bs::cuda_error(e, "graph instantiate");
    }
    *out = gr;
    return BS_OK;
}

bs_status bs_graph_launch(bs_graph *g, bs_stream stream) {
    BS_REQUIRE(g, "NULL graph");
    return bs::cuda_error(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
}

bs_status bs_graph_kernel_count(const bs_graph *g, int32_t *kernels) {
    BS_REQUIRE(g && kernels, "NULL argument");
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(g->graph, nullptr, &n);
    if (e != cudaSuccess) return bs::cuda_error(e, "graph nodes");
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) e = cudaGraphGetNodes(g->graph, nodes.data(), &n);
    if (e != cudaSuccess) return bs::cuda_error(e, "graph nodes");
    int32_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess) return bs::cuda_error(e, "graph node type");
        k += t == cudaGraphNodeTypeKernel;
    }
    *kernels = k;
    return BS_OK;
}

void bs_graph_destroy(bs_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

bs_status bs_autotune(bs_plan *p, const void *z_train, bs_cf64 *R, bs_cf32 *c, int32_t *info, bs_stream stream,
                      int32_t *threads_out, int32_t *ctas_per_sm_out, float *ms_out) {
    BS_REQUIRE(p && z_train && c && info, "NULL argument");
    if (bs_status s = check_device(p)) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    const int thr[1] = {128};
    const int cps[7] = {1, 2, 3, 4, 5, 6, 8};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bs::cuda_error(cudaGetLastError(), "event create");
    bs::CovSolveLaunch best = p->cs;
    float best_ms = 1e30f;
    bs_status s = BS_OK;
    for (int ti = 0; ti < 1 && !s; ++ti) {
        for (int ci = 0; ci < 7 && !s; ++ci) {
            bs::CovSolveLaunch cand;
            cand.threads = thr[ti];
            cand.ctas_per_sm = cps[ci];
            s = bs::launch_cov_solve(p, z_train, nullptr, (double2 *)R, (float2 *)c, info, p->d_head, cand, st);
            if (s) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && !s; ++r)
                s = bs::launch_cov_solve(p, z_train, nullptr, (double2 *)R, (float2 *)c, info, p->d_head, cand, st);
            cudaEventRecord(e1, st);
            if (s) break;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { s = bs::cuda_error(e, "autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    p->cs = best;
    if (threads_out) *threads_out = best.threads;
    if (ctas_per_sm_out) *ctas_per_sm_out = best.ctas_per_sm;
    if (ms_out) *ms_out = best_ms;
    return BS_OK;
}

bs_status bs_autotune_pass(bs_plan *p, const bs_buffers *b, bs_stream stream, bs_tune_report *rep) {
    BS_REQUIRE(p && b, "NULL argument");
    BS_REQUIRE(b->x && b->xc && b->z_train && b->R && b->c && b->info, "buf->x, xc, z_train, R, c, info needed");
    if (bs_status s = check_device(p)) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    bs_tune_report r;
    for (int k = 0; k < 3; ++k) r.covariance_ms[k] = -1.f;
    for (int k = 0; k < 4; ++k) r.beamspace_ms[k] = -1.f;
    r.solve_ms = r.fused_ms = -1.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bs::cuda_error(cudaGetLastError(), "event create");
    // mean time of `reps` runs after one warm-up run; < 0 if it failed
    auto time_of = [&](auto &&run, float *ms) -> bs_status {
        bs_status s = run();
        if (s) return s;
        cudaEventRecord(e0, st);
        constexpr int reps = 3;
        for (int k = 0; k < reps && !s; ++k) s = run();
        cudaEventRecord(e1, st);
        if (s) return s;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return bs::cuda_error(e, "autotune");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= reps;
        return BS_OK;
    };
    const int saved_b = p->tune_beamspace, saved_c = p->tune_cov, saved_f = p->tune_fused;
    bs_status s = bs::launch_channelize(p, (const float2 *)b->x, p->P, (float2 *)b->xc, st);
    // beamspace: the variants that apply to this plan
    int best_b = -1;
    float best = 1e30f;
    if (!s && !p->planar) {
        for (int v = 0; v < 4 && !s; ++v) {
            const bool applies = (v == 0) ? (p->cfg.M == 1024 || p->cfg.M == 2048 || p->cfg.M == 4096) &&
                                                p->cfg.N <= 1024 && p->cfg.T <= 256 && !(p->cfg.flags & BS_FLAG_NO_TMA)
                                 : (v == 1) ? p->cfg.M >= 512 && !(p->cfg.N & 1) && !(p->cfg.flags & BS_FLAG_NO_TMA) &&
                                                  (p->Fs % p->vpb) == 0 && (p->B % p->vpb) == 0
                                 : (v == 3) ? bs::beamspace_tc_applies(p)
                                            : true;
            if (!applies) continue;
            p->tune_beamspace = v;
            float ms = 0.f;
            s = time_of([&] { return bs::launch_beamspace(p, (const float2 *)b->xc, b->z_train, (float2 *)b->z_test, st); },
                        &ms);
            r.beamspace_ms[v] = ms;
            if (!s && ms < best) best = ms, best_b = v;
        }
    }
    p->tune_beamspace = best_b;
    if (!s) s = bs::launch_beamspace(p, (const float2 *)b->xc, b->z_train, (float2 *)b->z_test, st);
    // covariance
    int best_c = -1;
    best = 1e30f;
    const bool narrow = p->Wmax <= 16;
    for (int v = 0; v < 3 && !s; ++v) {
        const bool applies = (v == 0) || (v == 1 && narrow && p->Kmax <= 128) ||
                             (v == 2 && narrow && p->cfg.precision != BS_PREC_FP32);
        if (!applies || (p->cfg.flags & BS_FLAG_PLAIN)) continue;
        p->tune_cov = v;
        float ms = 0.f;
        s = time_of([&] { return bs::launch_window_cov(p, b->z_train, nullptr, (double2 *)b->R, st); }, &ms);
        r.covariance_ms[v] = ms;
        if (!s && ms < best) best = ms, best_c = v;
    }
    p->tune_cov = best_c;
    if (!s) s = bs::launch_window_cov(p, b->z_train, nullptr, (double2 *)b->R, st);
    if (!s) s = time_of([&] { return bs::launch_mvdr_solve(p, (const double2 *)b->R, (float2 *)b->c, b->info, st); },
                        &r.solve_ms);
    // the fused persistent kernel (W <= 16) at its best CTAs per SM, against the two launches
    int best_f = 0;
    if (!s && narrow && !(p->cfg.flags & BS_FLAG_PLAIN)) {
        int32_t thr = 0, cps = 0;
        float fms = 0.f;
        s = bs_autotune(p, b->z_train, b->R, b->c, b->info, stream, &thr, &cps, &fms);
        r.fused_ms = fms;
        if (!s && fms < best + r.solve_ms) best_f = 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) {
        p->tune_beamspace = saved_b;
        p->tune_cov = saved_c;
        p->tune_fused = saved_f;
        return s;
    }
    p->tune_fused = best_f;
    r.beamspace = best_b;
    r.covariance = best_c;
    r.fused = best_f;
    r.ctas_per_sm = p->cs.ctas_per_sm;
    if (rep) *rep = r;
    return BS_OK;
}

bs_status bs_set_launch(bs_plan *p, int32_t threads, int32_t ctas_per_sm) {
    BS_REQUIRE(p, "NULL plan");
    BS_REQUIRE(threads == 128, "threads must be 128");
    BS_REQUIRE(ctas_per_sm >= 1 && ctas_per_sm <= 32, "ctas_per_sm must be in 1..32");
    p->cs.threads = threads;
    p->cs.ctas_per_sm = ctas_per_sm;
    return BS_OK;
}

bs_status bs_run_host(const bs_plan *p, const bs_cf32 *x_host, bs_cf32 *out_host, const bs_buffers *b,
                      bs_stream stream) {
    BS_REQUIRE(p && b && x_host && out_host, "NULL argument");
    BS_REQUIRE(b->x && b->xc && b->z_train && b->out, "buf->x, xc, z_train and out must be device buffers");
    BS_REQUIRE(b->z_test || p->cfg.P_test == 0, "z_test is NULL but P_test > 0");
    if (bs_status s = check_device(p)) return s;
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t rec = (size_t)p->cfg.F * p->cfg.N;   // elements per raw record
    const size_t crec = (size_t)p->Fs * p->cfg.N;     // elements per channelised record (the plan's bins)
    const size_t obytes = (size_t)p->pairs * p->Vte * sizeof(bs_cf32);
    // Record chunks: the copy of chunk k+1 (on the plan's copy stream) runs
    // while chunk k is channelised and transformed on `stream`; the host link
    // is slower than the two stages.  Chunk boundaries fall at P_train, and
    // the covariance and solve (training windows only) run as soon as the
    // training chunks are transformed, under the copy of the test records;
    // the last test chunk is one record, so that little work (its two
    // stages, apply and the output copy) is left after the last copy.
    const int Ptr = p->cfg.P_train;
    int bounds[bs_plan::kHostChunks + 1];
    const int nch = bs::host_chunk_bounds(Ptr, p->P - Ptr, bs_plan::kHostChunks, bounds);
    cudaError_t e = cudaEventRecord(p->ev_start, st);   // earlier work on `stream` is done with x
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_st, p->ev_start, 0);
    for (int k = 0; k < nch && e == cudaSuccess; ++k) {
        const int p0 = bounds[k], np = bounds[k + 1] - bounds[k];
        e = cudaMemcpyAsync((void *)(b->x + p0 * rec), x_host + p0 * rec, np * rec * sizeof(bs_cf32),
                            cudaMemcpyHostToDevice, p->copy_st);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_chunk[k], p->copy_st);
    }
    if (e != cudaSuccess) return bs::cuda_error(e, "host to device copy");
    bs_status s;
    for (int k = 0; k < nch; ++k) {
        const int p0 = bounds[k], np = bounds[k + 1] - bounds[k];
        e = cudaStreamWaitEvent(st, p->ev_chunk[k], 0);
        if (e != cudaSuccess) return bs::cuda_error(e, "stream wait");
        if ((s = bs::launch_channelize(p, (const float2 *)(b->x + p0 * rec), np, (float2 *)(b->xc + p0 * crec), st)))
            return s;
        if ((s = bs::launch_beamspace(p, (const float2 *)b->xc, b->z_train, (float2 *)b->z_test, st, p0, np)))
            return s;
        if (bounds[k + 1] == Ptr) {   // every training window is in place
            if (use_fused(p)) {
                if ((s = bs_cov_solve(p, b->z_train, nullptr, b->R, b->c, b->info, stream))) return s;
            } else {
                if ((s = bs_window_cov(p, b->z_train, nullptr, b->R, stream))) return s;
                if ((s = bs_mvdr_solve(p, b->R, b->c, b->info, stream))) return s;
            }
        }
    }
    if ((s = bs_apply(p, b->z_test, b->c, b->out, stream))) return s;
    if (obytes) {
        e = cudaMemcpyAsync(out_host, b->out, obytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return bs::cuda_error(e, "device to host copy");
    }
    return bs::cuda_error(cudaStreamSynchronize(st), "stream synchronise");
}

}  // extern "C"
