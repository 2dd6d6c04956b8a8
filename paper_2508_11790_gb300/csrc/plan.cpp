// Plan creation: per-pair window tables and windowed steering vectors
// (host, FP64), device upload, error reporting.  Compiled with
// -ffp-contract=off so that the window decision is evaluated exactly in the
// documented order (no fused multiply-add).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace bs {

static thread_local std::string g_last_error;

bs_status set_error(bs_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

bs_status cuda_error(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return BS_OK;
    return set_error(BS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bs_status check_launch(const char *where) { return cuda_error(cudaGetLastError(), where); }

int beamspace_vectors_per_cta(int M) {
    int v = 4096 / M;
    if (v < 1) v = 1;
    if (v > 16) v = 16;
    return v;
}

}  // namespace bs

using bs::set_error;

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Centre frequency of subband s (Eq. SubChannelFreq), l = s - L/2 + 1.
static double subband_freq(int s, int L, double fc, double fs) {
    const int ell = s - L / 2 + 1;
    const double frac = (ell - 0.5) / L;
    const double off = frac * fs;
    return fc + off;
}

// First beam of the W-beam window: x = Omega M / (2 pi) with
// Omega = pi u (f / f_d) (Eq. SubOmegaX); start = floor(x - W/2 + 1) mod M.
static int window_start(double u, int s, int W, int L, int M, double fc, double fs, double fd) {
    const double f = subband_freq(s, L, fc, fs);
    const double ratio = f / fd;
    const double omega = M_PI * u * ratio;
    const double x = omega * (double)M / (2.0 * M_PI);
    const double lo = x - W / 2.0;
    const double fl = std::floor(lo + 1.0);
    long long st = (long long)fl % M;
    if (st < 0) st += M;
    return (int)st;
}

// Windowed steering entry [S D a]_m = M^-1/2 sum_{n<N} e^{j (Omega - 2 pi m/M) n}
// in closed form: M^-1/2 e^{j (N-1) d/2} sin(N d/2) / sin(d/2), d = Omega - 2 pi m / M,
// reduced to (-pi, pi] (the kernel is 2 pi periodic).
static bs_cf64 windowed_steering(double omega, int N, int M, int m) {
    double d = omega - 2.0 * M_PI * (double)m / (double)M;
    d -= 2.0 * M_PI * std::nearbyint(d / (2.0 * M_PI));
    const double h = 0.5 * d;
    const double amp = (std::fabs(h) < 1e-9) ? (double)N : std::sin(N * h) / std::sin(h);
    const double ph = 0.5 * (double)(N - 1) * d;
    const double sc = 1.0 / std::sqrt((double)M);
    return bs_cf64{amp * std::cos(ph) * sc, amp * std::sin(ph) * sc};
}

// Array geometry: linear (Nz = Mz = 1) or planar (Nx x Nz elements,
// Mx x Mz beams).
struct Geom {
    bool planar;
    int Nx, Nz, Mx, Mz;
};
static Geom geometry(const bs_config &c) {
    Geom g;
    g.planar = c.Nz > 1 || c.Mz > 1;
    g.Nz = g.planar ? std::max(c.Nz, 1) : 1;
    g.Mz = g.planar ? std::max(c.Mz, 1) : 1;
    g.Nx = c.N / g.Nz;
    g.Mx = c.M / g.Mz;
    return g;
}

// Window starts of pair (t, s): each axis centred on its own squinted spatial
// frequency (Eq. OverallWindow per axis); sz = 0 for a linear array.
static void pair_starts(const bs_config &c, const Geom &G, int t, int s, int *sx, int *sz) {
    const int Wz = G.planar ? c.Wz[t] : 1;
    *sx = window_start(c.u[t], s, c.W[t] / Wz, c.L, G.Mx, c.fc, c.fs, c.fd);
    *sz = G.planar ? window_start(c.v[t], s, Wz, c.L, G.Mz, c.fc, c.fs, c.fd) : 0;
}

// Entry w = w_x Wz + w_z of the windowed steering vector S D a: the product
// of the two axes' closed forms (S D a = (S_h D_h^T a_x) (x) (S_v D_v a_z)).
static bs_cf64 pair_steering(const bs_config &c, const Geom &G, int t, int s, int sx, int sz, int w) {
    const double ratio = subband_freq(s, c.L, c.fc, c.fs) / c.fd;
    const int Wz = G.planar ? c.Wz[t] : 1;
    const bs_cf64 ax = windowed_steering(M_PI * c.u[t] * ratio, G.Nx, G.Mx, (sx + w / Wz) % G.Mx);
    if (!G.planar) return ax;
    const bs_cf64 az = windowed_steering(M_PI * c.v[t] * ratio, G.Nz, G.Mz, (sz + w % Wz) % G.Mz);
    return bs_cf64{ax.re * az.re - ax.im * az.im, ax.re * az.im + ax.im * az.re};
}

template <class T>
static bs_status upload(T **dst, const std::vector<T> &src) {
    if (src.empty()) return BS_OK;
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return set_error(BS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return bs::cuda_error(e, "plan upload");
}

static std::vector<float2> twiddles(int n) {
    std::vector<float2> tw(n);
    for (int k = 0; k < n; ++k) {
        const double a = -2.0 * M_PI * (double)k / (double)n;
        tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return tw;
}

extern "C" {

const char *bs_status_string(bs_status s) {
    switch (s) {
        case BS_OK: return "ok";
        case BS_EINVAL: return "invalid argument";
        case BS_ENOMEM: return "out of device memory";
        case BS_ECUDA: return "CUDA error";
        case BS_ENOTPD: return "matrix not positive definite";
        case BS_ETIMEOUT: return "device wait timed out";
        case BS_EUNSUPPORTED: return "unsupported size";
    }
    return "unknown status";
}

const char *bs_last_error(void) { return bs::g_last_error.c_str(); }

void bs_plan_destroy(bs_plan *p) {
    if (!p) return;
    cudaFree(p->d_start);
    cudaFree(p->d_Wg);
    cudaFree(p->d_Kg);
    cudaFree(p->d_gather);
    cudaFree(p->d_gsub);
    cudaFree(p->d_glist);
    cudaFree(p->d_start_z);
    cudaFree(p->d_Wz);
    cudaFree(p->d_woff);
    cudaFree(p->d_ztr_off);
    cudaFree(p->d_zte_off);
    cudaFree(p->d_roff);
    cudaFree(p->d_at32);
    cudaFree(p->d_at64);
    cudaFree(p->d_atlo);
    cudaFree(p->d_twF);
    cudaFree(p->d_twM);
    cudaFree(p->d_err);
    cudaFree(p->d_order);
    cudaFree(p->d_order_w);
    cudaFree(p->d_head);
    for (cudaEvent_t e : p->ev_chunk)
        if (e) cudaEventDestroy(e);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
    for (int k = 0; k < bs_plan::kSolveStreams; ++k) {
        if (p->solve_st[k]) cudaStreamDestroy(p->solve_st[k]);
        if (p->ev_join[k]) cudaEventDestroy(p->ev_join[k]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    delete p;
}

static bs_status validate_config(const bs_config *cfg) {
    if (!cfg) return set_error(BS_EINVAL, "config is NULL");
    const bs_config &c = *cfg;
    if (c.N < 1 || c.N > 4096) return set_error(BS_EUNSUPPORTED, "N must be in 1..4096");
    if (!is_pow2(c.F) || c.F < 16 || c.F > 4096)
        return set_error(BS_EUNSUPPORTED, "F must be a power of two in 16..4096");
    if (!is_pow2(c.L) || c.L > c.F) return set_error(BS_EINVAL, "L must be a power of two dividing F");
    if (!is_pow2(c.M) || c.M < 16 || c.M > 4096 || c.M < c.N)
        return set_error(BS_EUNSUPPORTED, "M must be a power of two in 16..4096 with M >= N");
    if (c.T < 1 || c.T > 32767) return set_error(BS_EINVAL, "T must be in 1..32767");
    if (c.P_train < 1 || c.P_test < 0) return set_error(BS_EINVAL, "P_train >= 1 and P_test >= 0 required");
    if (!c.u || !c.W || !c.K) return set_error(BS_EINVAL, "u, W and K must be given");
    if (!(c.fd > 0) || !(c.fs > 0)) return set_error(BS_EINVAL, "fs and fd must be positive");
    if (!(c.delta >= 0) || !std::isfinite(c.delta)) return set_error(BS_EINVAL, "delta must be finite and >= 0");
    if (c.precision < BS_PREC_FP32 || c.precision > BS_PREC_BF16)
        return set_error(BS_EINVAL, "unknown precision");
    const int B = c.F / c.L;
    if (c.s_count > 0 && c.s_count < c.L) {
        if (!is_pow2(c.s_count) || c.s_begin < 0 || c.s_begin % c.s_count || c.s_begin + c.s_count > c.L)
            return set_error(BS_EINVAL, "subband shard: s_count a power of two, s_begin a multiple of it, "
                                        "s_begin + s_count <= L");
    }
    if (c.Nz > 1 || c.Mz > 1) {
        if (c.Nz < 1 || c.N % c.Nz) return set_error(BS_EINVAL, "planar: Nz must divide N");
        if (!is_pow2(c.Mz) || c.Mz < c.Nz || c.M % c.Mz || c.M / c.Mz < c.N / c.Nz)
            return set_error(BS_EINVAL, "planar: Mz a power of two, Nz <= Mz, N/Nz <= M/Mz");
        if (c.N > 1024 || c.M > 2048) return set_error(BS_EUNSUPPORTED, "planar: N <= 1024 and M <= 2048");
        if (!c.Wz || !c.v) return set_error(BS_EINVAL, "planar: Wz and v must be given");
        for (int t = 0; t < c.T; ++t) {
            if (c.Wz[t] < 1 || c.W[t] % c.Wz[t] || c.Wz[t] > c.Mz || c.W[t] / c.Wz[t] > c.M / c.Mz)
                return set_error(BS_EINVAL, "planar: Wz must divide W, Wz <= Mz, W/Wz <= M/Mz");
            if (!std::isfinite(c.v[t]) || std::fabs(c.v[t]) > 1.0)
                return set_error(BS_EINVAL, "direction sines must lie in [-1, 1]");
        }
    }
    for (int t = 0; t < c.T; ++t) {
        if (c.W[t] < 1 || c.W[t] > 32) return set_error(BS_EUNSUPPORTED, "window sizes must be in 1..32");
        if (c.W[t] > c.M) return set_error(BS_EINVAL, "window larger than M");
        if (c.K[t] < 1 || (int64_t)c.K[t] > (int64_t)c.P_train * B)
            return set_error(BS_EINVAL, "K must be in 1..P_train*B");
        if (!std::isfinite(c.u[t]) || std::fabs(c.u[t]) > 1.0)
            return set_error(BS_EINVAL, "direction sines must lie in [-1, 1]");
    }
    return BS_OK;
}

// The plan's subbands: the first and how many (a shard, or all L).
static void shard_range(const bs_config &c, int *s0, int *Ls) {
    const bool shard = c.s_count > 0 && c.s_count < c.L;
    *s0 = shard ? c.s_begin : 0;
    *Ls = shard ? c.s_count : c.L;
}

bs_status bs_plan_tables_host(const bs_config *cfg, int32_t *start, bs_cf64 *a_tilde) {
    if (bs_status st = validate_config(cfg)) return st;
    const bs_config &c = *cfg;
    const Geom G = geometry(c);
    int s0, Ls;
    shard_range(c, &s0, &Ls);
    int64_t e = 0;
    for (int t = 0; t < c.T; ++t) {
        for (int sl = 0; sl < Ls; ++sl) {
            const int s = s0 + sl;
            const int64_t g = (int64_t)t * Ls + sl;
            int sx, sz;
            pair_starts(c, G, t, s, &sx, &sz);
            if (start) start[g] = sx;
            for (int w = 0; w < c.W[t]; ++w, ++e)
                if (a_tilde) a_tilde[e] = pair_steering(c, G, t, s, sx, sz, w);
        }
    }
    return BS_OK;
}

bs_status bs_plan_create(bs_plan **out, const bs_config *cfg) {
    if (!out) return set_error(BS_EINVAL, "plan pointer is NULL");
    *out = nullptr;
    if (bs_status st = validate_config(cfg)) return st;
    const bs_config &c = *cfg;
    const int B = c.F / c.L;
    bs_plan *p = new bs_plan();
    p->cfg = c;
    p->cfg.u = nullptr;
    p->cfg.W = nullptr;
    p->cfg.K = nullptr;
    p->cfg.Wz = nullptr;
    p->cfg.v = nullptr;
    const Geom geo = geometry(c);
    p->planar = geo.planar;
    p->Nx = geo.Nx;
    p->Nz = geo.Nz;
    p->Mx = geo.Mx;
    p->Mz = geo.Mz;
    p->Wzt.assign((size_t)c.T, 1);
    if (geo.planar) p->Wzt.assign(c.Wz, c.Wz + c.T);
    if (!(p->cfg.kappa_max > 0)) p->cfg.kappa_max = 1e5;
    if (!(p->cfg.store_scale > 0)) p->cfg.store_scale = 1.0f;
    p->B = B;
    shard_range(c, &p->s0, &p->Ls);
    p->Fs = p->Ls * B;
    p->P = c.P_train + c.P_test;
    p->Vte = c.P_test * B;
    p->pairs = (int64_t)c.T * p->Ls;
    p->Wt.assign(c.W, c.W + c.T);
    p->Kt.assign(c.K, c.K + c.T);
    p->u.assign(c.u, c.u + c.T);
    for (int t = 0; t < c.T; ++t) {
        p->Wmax = std::max(p->Wmax, p->Wt[t]);
        p->Kmax = std::max(p->Kmax, p->Kt[t]);
        p->sumW += p->Wt[t];
    }
    const int64_t G = p->pairs;
    p->start.resize(G);
    p->start_z.resize(G);
    p->Wg.resize(G);
    p->Kg.resize(G);
    p->woff.assign(G + 1, 0);
    p->ztr_off.assign(G + 1, 0);
    p->zte_off.assign(G + 1, 0);
    p->roff.assign(G + 1, 0);
    for (int t = 0; t < c.T; ++t) {
        for (int sl = 0; sl < p->Ls; ++sl) {
            const int s = p->s0 + sl;
            const int64_t g = (int64_t)t * p->Ls + sl;
            const int W = p->Wt[t], K = p->Kt[t];
            p->Wg[g] = W;
            p->Kg[g] = K;
            int sx, sz;
            pair_starts(c, geo, t, s, &sx, &sz);
            p->start[g] = sx;
            p->start_z[g] = sz;
            p->woff[g + 1] = p->woff[g] + W;
            p->ztr_off[g + 1] = p->ztr_off[g] + (int64_t)W * K;
            p->zte_off[g + 1] = p->zte_off[g] + (int64_t)W * p->Vte;
            p->roff[g + 1] = p->roff[g] + (int64_t)W * W;
        }
    }
    p->c_elems = p->woff[G];
    p->ztr_elems = p->ztr_off[G];
    p->zte_elems = p->zte_off[G];
    p->r_elems = p->roff[G];
    p->at.resize(p->c_elems);
    std::vector<float2> at32(p->c_elems), atlo(p->c_elems);
    std::vector<double2> at64(p->c_elems);
    for (int t = 0; t < c.T; ++t) {
        for (int sl = 0; sl < p->Ls; ++sl) {
            const int s = p->s0 + sl;
            const int64_t g = (int64_t)t * p->Ls + sl;
            for (int w = 0; w < p->Wg[g]; ++w) {
                const bs_cf64 a = pair_steering(c, geo, t, s, p->start[g], p->start_z[g], w);
                const int64_t e = p->woff[g] + w;
                p->at[e] = a;
                at32[e] = make_float2((float)a.re, (float)a.im);
                atlo[e] = make_float2((float)(a.re - (double)at32[e].x), (float)(a.im - (double)at32[e].y));
                at64[e] = make_double2(a.re, a.im);
            }
        }
    }
    // beamspace gather table: one CTA handles vpb consecutive vectors; for
    // target t its vpb windows are contiguous in z, entry k = c * W_t + w.
    p->vpb = bs::beamspace_vectors_per_cta(c.M);
    p->gather.reserve((size_t)p->vpb * p->sumW);
    for (int t = 0; t < c.T; ++t)
        for (int cc = 0; cc < p->vpb; ++cc)
            for (int w = 0; w < p->Wt[t]; ++w) p->gather.push_back((t << 10) | (cc << 5) | w);
    p->glist.reserve((size_t)p->sumW);
    for (int t = 0; t < c.T; ++t)
        for (int w = 0; w < p->Wt[t]; ++w) p->glist.push_back((t << 8) | w);
    // the same per-pair fields subband-major, so that the per-group entries
    // of consecutive targets are one contiguous read
    p->gsub.resize((size_t)4 * G);
    for (int s = 0; s < p->Ls; ++s)
        for (int t = 0; t < c.T; ++t) {
            const int64_t g = (int64_t)t * p->Ls + s;
            int64_t *e = &p->gsub[(size_t)4 * ((int64_t)s * c.T + t)];
            e[0] = p->ztr_off[g];
            e[1] = p->zte_off[g];
            e[2] = (int64_t)(p->start[g] | (p->Wg[g] << 16));
            e[3] = p->Kg[g];
        }

    // work-queue order of the fused covariance + solve: decreasing W^2 K
    p->order.resize(G);
    std::iota(p->order.begin(), p->order.end(), 0);
    std::stable_sort(p->order.begin(), p->order.end(), [&](int32_t x, int32_t y) {
        return (int64_t)p->Wg[x] * p->Wg[x] * p->Kg[x] > (int64_t)p->Wg[y] * p->Wg[y] * p->Kg[y];
    });
    // the stand-alone solve visits pairs grouped by W, so that the CTAs
    // resident together run the code of one window size (one solve body per
    // W: mixed sizes side by side thrashed the instruction cache)
    p->order_w.resize(G);
    std::iota(p->order_w.begin(), p->order_w.end(), 0);
    std::stable_sort(p->order_w.begin(), p->order_w.end(),
                     [&](int32_t x, int32_t y) { return p->Wg[x] < p->Wg[y]; });
    p->Wmin = *std::min_element(p->Wg.begin(), p->Wg.end());
    p->nsmall = std::count_if(p->Wg.begin(), p->Wg.end(), [](int32_t w) { return w <= 16; });
    for (int w = 1; w <= 33; ++w)   // order_w is sorted by W
        p->wstart[w] = p->wstart[w - 1] + std::count(p->Wg.begin(), p->Wg.end(), w - 1);

    cudaGetDevice(&p->device);
    bs_status st = BS_OK;
    if (!st) st = upload(&p->d_start, p->start);
    if (!st) st = upload(&p->d_Wg, p->Wg);
    if (!st) st = upload(&p->d_Kg, p->Kg);
    if (!st) st = upload(&p->d_gather, p->gather);
    if (!st) st = upload(&p->d_gsub, p->gsub);
    if (!st) st = upload(&p->d_glist, p->glist);
    if (!st) st = upload(&p->d_start_z, p->start_z);
    if (!st) st = upload(&p->d_Wz, p->Wzt);
    if (!st) st = upload(&p->d_woff, p->woff);
    if (!st) st = upload(&p->d_ztr_off, p->ztr_off);
    if (!st) st = upload(&p->d_zte_off, p->zte_off);
    if (!st) st = upload(&p->d_roff, p->roff);
    if (!st) st = upload(&p->d_at32, at32);
    if (!st) st = upload(&p->d_at64, at64);
    if (!st) st = upload(&p->d_atlo, atlo);
    if (!st) st = upload(&p->d_twF, twiddles(c.F));
    if (!st) st = upload(&p->d_twM, twiddles(c.M));
    if (!st) st = upload(&p->d_err, std::vector<int>(1, 0));
    if (!st) st = upload(&p->d_order, p->order);
    if (!st) st = upload(&p->d_order_w, p->order_w);
    if (!st) st = upload(&p->d_head, std::vector<int>(1, 0));
    if (!st) st = bs::cuda_error(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking), "copy stream");
    if (!st) st = bs::cuda_error(cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming), "event");
    if (!st) st = bs::cuda_error(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming), "event");
    for (int k = 0; k < bs_plan::kSolveStreams && !st; ++k) {
        st = bs::cuda_error(cudaStreamCreateWithFlags(&p->solve_st[k], cudaStreamNonBlocking), "solve stream");
        if (!st) st = bs::cuda_error(cudaEventCreateWithFlags(&p->ev_join[k], cudaEventDisableTiming), "event");
    }
    for (int k = 0; k < bs_plan::kHostChunks && !st; ++k)
        st = bs::cuda_error(cudaEventCreateWithFlags(&p->ev_chunk[k], cudaEventDisableTiming), "event");
    if (!st) st = bs::cuda_error(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device),
                                 "device attribute");
    if (st) {
        bs_plan_destroy(p);
        return st;
    }
    *out = p;
    return BS_OK;
}

bs_status bs_plan_device_status(const bs_plan *p, int32_t *flags) {
    if (!p) return set_error(BS_EINVAL, "NULL plan");
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bs::cuda_error(e, "device status read");
    if (flags) *flags = h;
    if (h) {
        const int zero = 0;
        e = cudaMemcpy(p->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bs::cuda_error(e, "device status reset");
        return set_error(BS_ETIMEOUT, "a bounded device wait gave up (device error word set)");
    }
    return BS_OK;
}

bs_status bs_plan_set_device_flags(bs_plan *p, int32_t flags) {
    if (!p) return set_error(BS_EINVAL, "NULL plan");
    const int h = flags;
    const cudaError_t e = cudaMemcpy(p->d_err, &h, sizeof(int), cudaMemcpyHostToDevice);
    return bs::cuda_error(e, "device error word write");
}

bs_status bs_plan_sizes(const bs_plan *p, bs_sizes *o) {
    if (!p || !o) return set_error(BS_EINVAL, "NULL argument");
    std::memset(o, 0, sizeof(*o));
    o->pairs = p->pairs;
    o->B = p->B;
    o->Vte = p->Vte;
    o->W_max = p->Wmax;
    o->K_max = p->Kmax;
    o->x_elems = (int64_t)p->P * p->cfg.F * p->cfg.N;
    o->xc_elems = (int64_t)p->P * p->Fs * p->cfg.N;
    o->ztrain_elems = p->ztr_elems;
    o->ztrain_bytes = p->ztr_elems * (p->cfg.precision == BS_PREC_FP32 ? 8 : 4);
    o->ztest_elems = p->zte_elems;
    o->r_elems = p->r_elems;
    o->c_elems = p->c_elems;
    o->out_elems = p->pairs * p->Vte;
    return BS_OK;
}

bs_status bs_plan_offsets(const bs_plan *p, int32_t *start, int32_t *W, int32_t *K, int64_t *woff,
                          int64_t *ztr_off, int64_t *zte_off, int64_t *roff, bs_cf64 *a_tilde) {
    if (!p) return set_error(BS_EINVAL, "NULL plan");
    const size_t G = (size_t)p->pairs;
    if (start) std::memcpy(start, p->start.data(), G * sizeof(int32_t));
    if (W) std::memcpy(W, p->Wg.data(), G * sizeof(int32_t));
    if (K) std::memcpy(K, p->Kg.data(), G * sizeof(int32_t));
    if (woff) std::memcpy(woff, p->woff.data(), (G + 1) * sizeof(int64_t));
    if (ztr_off) std::memcpy(ztr_off, p->ztr_off.data(), (G + 1) * sizeof(int64_t));
    if (zte_off) std::memcpy(zte_off, p->zte_off.data(), (G + 1) * sizeof(int64_t));
    if (roff) std::memcpy(roff, p->roff.data(), (G + 1) * sizeof(int64_t));
    if (a_tilde) std::memcpy(a_tilde, p->at.data(), p->at.size() * sizeof(bs_cf64));
    return BS_OK;
}

}  // extern "C"
