/*
 * bs.h - C ABI of the windowed beamspace MVDR hot path on GB300 (sm_103a).
 *
 * Method: "Scaling Wideband Massive MIMO Radar via Beamspace Dimension
 * Reduction" (arXiv 2508.11790).  Per record the array data are channelised
 * into L subbands by an F-point FFT (Sec. III-A), each subband vector is
 * taken to beamspace by a zero-padded M-point spatial DFT (Eq. VerDFT,
 * Eq. BeamTransform), a W-beam window is cut around every target's
 * frequency-squinted beam (Eq. SubOmegaX, Eq. OverallWindow,
 * Eq. ApplyWindow), the windowed training vectors give a diagonally loaded
 * W x W covariance (Eq. EmpiricalCov), the MVDR correlator
 * c = R^-1 a / (a^H R^-1 a) is solved per (target, subband) pair
 * (Eq. BeamCorrMVDR) and applied to the test vectors as c^H y (Sec. II-B).
 * The array is a half-wavelength uniform linear array (the paper's planar
 * array with N_z = 1), so the beamspace transform is one truncated DFT.
 *
 * Conventions (all entry points):
 *  - Data pointers are DEVICE pointers owned by the caller, except where a
 *    name ends in _host.  The library never allocates or frees on the hot
 *    path; a plan owns its small tables and workspace, allocated at create.
 *  - Calls are asynchronous on the given stream (NULL = legacy default
 *    stream).  Argument and launch errors are returned at once; numerical
 *    failures are reported per pair in `info` (bs_mvdr_solve).
 *  - Complex values are interleaved (re, im) pairs, C-contiguous.
 *  - Pair index g = t * L + s for target t and subband s.  Subband s is the
 *    paper's l = s - L/2 + 1 with centre f(l) = f_c + ((l - 1/2)/L) f_s
 *    (Eq. SubChannelFreq); s = 0 is the lowest.
 *  - "vector" v of a pair is record p, bin i of its subband, v = p*B + i
 *    (record-major), B = F / L.  Training vectors are those of the first
 *    P_train records; the first K_t of them enter the covariance of every
 *    pair of target t.  Test vectors are those of the next P_test records,
 *    v' = (p - P_train) * B + i.
 *  - Ragged per-pair arrays are packed back to back in pair order:
 *      weights / steering : W_g complex values per pair
 *      training windows   : K_g * W_g per pair, [v][w]
 *      test windows       : Vte * W_g per pair, [v'][w], Vte = P_test * B
 *      covariance         : W_g * W_g per pair, [i][j] row-major
 *    bs_plan_sizes() returns the totals and bs_plan_offsets() the offsets.
 *  - Not thread-safe per plan if two threads launch on one plan with
 *    different buffers at the same time (plan workspace is shared).  The
 *    same holds for two streams: bs_run_host and the stand-alone solve fork
 *    work onto streams and events the plan owns (joined back into the
 *    caller's stream before they return), so calls on one plan are issued
 *    one after another, in stream order.
 */
#ifndef BS_H
#define BS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *bs_stream; /* same handle as cudaStream_t */

typedef enum {
    BS_OK = 0,
    BS_EINVAL = 1,        /* bad argument (message in bs_last_error()) */
    BS_ENOMEM = 2,        /* device allocation failed at plan create */
    BS_ECUDA = 3,         /* CUDA runtime error (message in bs_last_error()) */
    BS_ENOTPD = 4,        /* reserved: reported per pair through info */
    BS_ETIMEOUT = 5,      /* a bounded device wait gave up */
    BS_EUNSUPPORTED = 6   /* size outside the compiled kernel range */
} bs_status;

/* Storage / arithmetic precision of the training windows and covariance. */
typedef enum {
    BS_PREC_FP32 = 0,     /* cf32 windows, FP32 SIMT products */
    BS_PREC_FP16 = 1,     /* fp16 windows (x store_scale), tensor-core products (mma.sync m16n8k16) */
    BS_PREC_BF16 = 2      /* bf16 windows (x store_scale), tensor-core products */
} bs_precision;

/* Plan flags. */
#define BS_FLAG_PLAIN      (1u << 0) /* plain FP32 per-pair path: one CTA per pair,
                                        FP32 sums, FP32 Cholesky, no refinement */
#define BS_FLAG_NO_REFINE  (1u << 1) /* skip the iterative-refinement step */
#define BS_FLAG_NO_FP64    (1u << 2) /* never escalate a pair to the FP64 solve */
#define BS_FLAG_NO_TMA     (1u << 3) /* channeliser without the TMA-staged persistent kernel */
#define BS_FLAG_FUSED      (1u << 4) /* bs_run: bs_cov_solve instead of bs_window_cov + bs_mvdr_solve */
#define BS_FLAG_SIMT_COV   (1u << 5) /* 16-bit windows: FP32 SIMT products instead of the tensor cores */
#define BS_FLAG_STAGED_FFT (1u << 6) /* beamspace at M = 1024..4096, N <= 1024: the bulk-copy-staged
                                        Stockham kernel instead of the warp-per-transform kernel */
#define BS_FLAG_SIMT_FFT   (1u << 7) /* beamspace at N = 1024, M = 2048: the CUDA-core kernels instead
                                        of the tensor-core DFT */

typedef struct { float re, im; } bs_cf32;
typedef struct { double re, im; } bs_cf64;

typedef struct {
    int32_t N;        /* array elements, 1..4096 */
    int32_t F;        /* fast-time samples per record; power of 2, 16..4096 */
    int32_t L;        /* subbands; power of 2 dividing F */
    int32_t M;        /* spatial FFT size; power of 2, N <= M <= 4096 */
    int32_t T;        /* targets, >= 1 */
    int32_t P_train;  /* target-free training records, >= 1 */
    int32_t P_test;   /* test records, >= 0 */
    double fc;        /* carrier frequency, Hz */
    double fs;        /* sampling rate, Hz */
    double fd;        /* design frequency of the lambda/2 spacing, Hz */
    const double  *u; /* [T] host: direction sine sin(phi_t) of each target */
    const int32_t *W; /* [T] host: window size per target, 1..16 */
    const int32_t *K; /* [T] host: training vectors per target, 1..P_train*B */
    double delta;     /* diagonal loading added to every window covariance */
    int32_t precision;   /* bs_precision */
    uint32_t flags;      /* BS_FLAG_* */
    double kappa_max;    /* FP64 escalation threshold on the Cholesky pivot
                            ratio (max L_ii / min L_ii)^2; <= 0 selects 1e5 */
    float store_scale;   /* 16-bit windows hold value * store_scale (<= 0: 1) */
    /* Uniform planar array (Eq. ArrayFactor, Eq. OverallDFT, Eq. OverallWindow);
     * Nz <= 1 (with Mz <= 1, Wz and v NULL) is the linear array above.
     * Elements n = n_x Nz + n_z (N = Nx Nz), beams m = m_x Mz + m_z
     * (M = Mx Mz), window entries w = w_x Wz + w_z (W = Wx Wz, the selector
     * read as S_h (x) S_v).  u[t] = cos(theta) sin(phi) (horizontal),
     * v[t] = sin(theta) (vertical).  Planar plans need N <= 1024 and
     * M <= 2048; bs_lift, bs_beam_pattern and bs_beamspace_full are
     * linear-array only. */
    int32_t Nz;          /* vertical elements (0 or 1: linear array) */
    int32_t Mz;          /* vertical FFT size, power of 2, Nz <= Mz */
    const int32_t *Wz;   /* [T] host: vertical window size per target, dividing W[t] */
    const double  *v;    /* [T] host: vertical direction sine sin(theta) per target */
    /* Subband shard (the subbands are processed independently once
     * channelised, Sec. III-A): a plan with 0 < s_count < L covers only
     * subbands s_begin .. s_begin + s_count - 1 of the L, so that G ranks can
     * each run their own block.  s_count must be a power of two and s_begin
     * a multiple of it.  Such a plan has pairs = T * s_count, pair
     * g = t * s_count + (s - s_begin), and a channelised cube xc of
     * [P][s_count * B][N] (the shard's bins of every record, in the order of
     * the full cube); bs_channelize still reads whole raw records and writes
     * only those bins.  Window starts and steering vectors use each
     * subband's own centre frequency, so every pair's results equal those of
     * the same pair of the unsharded plan.  bs_range_doppler needs every
     * subband of a target and refuses a shard (BS_EUNSUPPORTED).
     * s_count <= 0 or s_count == L: every subband (s_begin ignored). */
    int32_t s_begin;
    int32_t s_count;
} bs_config;

typedef struct {
    int64_t pairs;        /* T * L (T * s_count for a subband shard) */
    int32_t B;            /* bins per subband, F / L */
    int32_t Vte;          /* test vectors per pair, P_test * B */
    int32_t W_max, K_max;
    int64_t x_elems;      /* cf32 elements of one raw cube, P*F*N, P = P_train+P_test */
    int64_t xc_elems;     /* cf32 elements of the channelised cube, P*F*N (P*s_count*B*N for a shard) */
    int64_t ztrain_elems; /* complex elements of the training windows, sum W_g K_g */
    int64_t ztrain_bytes; /* bytes: 8 per element (FP32) or 4 (FP16/BF16) */
    int64_t ztest_elems;  /* cf32 elements of the test windows, sum W_g Vte */
    int64_t r_elems;      /* cf64 elements of the covariances, sum W_g^2 */
    int64_t c_elems;      /* cf32 elements of the weights, sum W_g */
    int64_t out_elems;    /* cf32 elements of the output, pairs * Vte */
} bs_sizes;

/* Buffers of one whole pass, for bs_run / bs_run_host (device pointers). */
typedef struct {
    bs_cf32 *x;        /* [P][F][N] raw IQ (bs_run_host copies the host cube here) */
    bs_cf32 *xc;       /* [P][F][N] channelised */
    void    *z_train;  /* training windows */
    bs_cf32 *z_test;   /* test windows */
    bs_cf64 *R;        /* covariances */
    bs_cf32 *c;        /* weights */
    int32_t *info;     /* [pairs] */
    bs_cf32 *out;      /* [pairs][Vte] */
} bs_buffers;

typedef struct bs_plan bs_plan;

/* ---------------------------------------------------------------- plan --- */

/* Create a plan on the current CUDA device.  Computes in FP64 on the host,
 * per pair: the squinted spatial frequency Omega = pi*u*(f(l)/f_d)
 * (Eq. SubOmegaX), x = Omega*M/(2*pi), the window start
 * floor(x - W/2 + 1) mod M (the W consecutive beams whose centre is nearest
 * to x; evaluated in exactly this order with no fused multiply-add), and
 * the windowed steering vector a~ = S D a(Omega) (Sec. III-C) from the
 * closed-form Dirichlet kernel.  Uploads these tables.
 * Errors: BS_EINVAL (sizes, NULL pointers), BS_EUNSUPPORTED, BS_ENOMEM,
 * BS_ECUDA.  On error *plan is NULL. */
bs_status bs_plan_create(bs_plan **plan, const bs_config *cfg);
void      bs_plan_destroy(bs_plan *plan);
bs_status bs_plan_sizes(const bs_plan *plan, bs_sizes *out);

/* Host copies of the per-pair tables (any pointer may be NULL):
 * start[pairs] window start beam; W[pairs], K[pairs]; woff[pairs+1],
 * ztr_off[pairs+1], zte_off[pairs+1], roff[pairs+1] element offsets of the
 * packed arrays; a_tilde[c_elems] windowed steering vectors (FP64). */
bs_status bs_plan_offsets(const bs_plan *plan, int32_t *start, int32_t *W, int32_t *K,
                          int64_t *woff, int64_t *ztr_off, int64_t *zte_off,
                          int64_t *roff, bs_cf64 *a_tilde);

/* The same per-pair tables as bs_plan_create, computed on the host only (no
 * device is touched): start[pairs] window start beams and a_tilde[sum W_g]
 * windowed steering vectors (pair order, W_g values each; for a subband
 * shard the shard's pairs).  Either output may be NULL.  Errors: as
 * bs_plan_create's argument checks. */
bs_status bs_plan_tables_host(const bs_config *cfg, int32_t *start, bs_cf64 *a_tilde);

/* Synchronises the device and reads the plan's device error word, which a
 * kernel sets when one of its bounded waits (TMA / mbarrier) gives up.
 * flags (may be NULL) receives the word; it is cleared after reading.
 * Returns BS_ETIMEOUT if it was set, else BS_OK. */
bs_status bs_plan_device_status(const bs_plan *plan, int32_t *flags);

/* Writes the plan's device error word from the host (synchronous copy).
 * flags = 0 clears it; a non-zero value makes the next
 * bs_plan_device_status report BS_ETIMEOUT exactly as a kernel whose
 * bounded wait gave up would, so that callers can test their handling of
 * that error without a device wait running out. */
bs_status bs_plan_set_device_flags(bs_plan *plan, int32_t flags);

/* ----------------------------------------------------------- hot path --- */

/* Channelise (Sec. III-A): for every record p < P and element n,
 *   xc[p][s*B + i][n] = F^-1/2 sum_t x[p][t][n] e^{-j 2 pi k t / F}
 * with k = ((s - L/2) B + i) mod F.  x, xc: [P][F][N] cf32, distinct.  For
 * a subband shard only s in s_begin .. s_begin + s_count - 1 is written,
 * to xc[p][(s - s_begin) B + i][n] (xc: [P][s_count B][N]). */
bs_status bs_channelize(const bs_plan *plan, const bs_cf32 *x, int32_t P,
                        bs_cf32 *xc, bs_stream stream);

/* Beamspace + window (Eq. BeamTransform, Eq. ApplyWindow): for every record
 * p < P_train + P_test and bin q = s*B + i, y^ = M^-1/2 sum_{n<N}
 * xc[p][q][n] e^{-j 2 pi m n / M} (zero-padded to M), then for every target
 * t the W_t beams (start_g + w) mod M, g = t*L + s, are written:
 *   training records (p < P_train), v = p*B + i < K_t : z_train, in the
 *     plan precision (FP16 / BF16 hold value * store_scale);
 *   test records: z_test (cf32).
 * z_test may be NULL when P_test == 0. */
bs_status bs_beamspace(const bs_plan *plan, const bs_cf32 *xc, void *z_train,
                       bs_cf32 *z_test, bs_stream stream);

/* Full zero-padded beamspace transform of nvec vectors (Eq. BeamTransform
 * without the window): yb[v][m] = M^-1/2 sum_{n<N} y[v][n] e^{-j2pi mn/M}.
 * y: [nvec][N] cf32, yb: [nvec][M] cf32. */
bs_status bs_beamspace_full(const bs_plan *plan, const bs_cf32 *y, int64_t nvec,
                            bs_cf32 *yb, bs_stream stream);

/* Loaded window covariance (Eq. EmpiricalCov on the windowed vectors, plus
 * loading): R_g = (1/K_g) sum_{v<K_g} z_v z_v^H + delta_g I, stored in FP64
 * (full Hermitian matrix).  delta_pair: NULL = plan delta, else a device
 * array [pairs] of per-pair loading (float).  FP32 windows: FP32 products;
 * FP32 partial sums of at most 16 vectors (a CTA per pair) or of 4 vectors
 * (a warp per pair, taken when K <= 128 and there are at least 4 pairs per
 * SM) are combined in double-float (pairs of FP32, about 2^-47 relative).
 * 16-bit windows: products on the tensor cores with FP32 accumulation,
 * folded into double-float every 128 vectors. */
bs_status bs_window_cov(const bs_plan *plan, const void *z_train, const float *delta_pair,
                        bs_cf64 *R, bs_stream stream);

/* MVDR correlator (Eq. BeamCorrMVDR): c_g = R_g^-1 a~_g / (a~_g^H R_g^-1 a~_g).
 * FP32 Cholesky R = L L^H and two triangular solves, one refinement step
 * whose residual a~ - R v is formed with error-free FP32 transformations
 * from the double-float (hi + lo FP32) parts of R and a~ (about twice FP32
 * precision; no FP64 arithmetic), then c = v / (a~^H v) in FP32.  Pairs whose
 * pivot ratio (max L_ii / min L_ii)^2 exceeds kappa_max, or whose FP32
 * factorisation fails, are solved again entirely in FP64.
 * info[g]: 0 = FP32 solve, -2 = solved in FP64, -1 = non-finite input,
 * k >= 1 = pivot k-1 not positive in FP64 (c_g set to NaN). */
bs_status bs_mvdr_solve(const bs_plan *plan, const bs_cf64 *R, bs_cf32 *c, int32_t *info,
                        bs_stream stream);

/* bs_mvdr_solve with a diagonal preconditioner (the seed the learned-loading
 * network predicts, or any positive scaling): each d_i is rounded to the
 * nearest power of two, 2^e_i (exponents clamped to [-30, 30]; non-positive
 * or non-finite d_i count as 1), and with D = diag(2^e) the pair is solved
 * as (D R D) y = D a~, c = D y / (a~^H D y) -- in exact arithmetic the c of
 * bs_mvdr_solve (R^-1 a~ = D (D R D)^-1 D a~), and every scaling is exact,
 * so only the conditioning the FP32 Cholesky sees (and with it the pivot
 * ratio test for FP64 escalation) changes.  Jacobi scaling
 * d_i = R_ii^-1/2 makes the diagonal of D R D lie in [1/2, 2].
 * d: device [c_elems] FP32, packed like c (W_g values per pair).  Plans
 * with BS_FLAG_PLAIN ignore d.  Results and info as bs_mvdr_solve.  The
 * paper solves Eq. BeamCorrMVDR unscaled; the scaling follows the
 * workload's learned preconditioner. */
bs_status bs_mvdr_solve_precond(const bs_plan *plan, const bs_cf64 *R, const float *d, bs_cf32 *c, int32_t *info,
                                bs_stream stream);

/* Fused covariance + solve of every pair in one persistent launch (the
 * default of bs_run): the same results as bs_window_cov followed by
 * bs_mvdr_solve (R is optional here and may be NULL).  CTAs take pairs from
 * a work queue ordered by decreasing W_g^2 K_g, so pairs of uneven W and K
 * share one launch.  The queue head lives in the plan's workspace, so calls
 * on one plan must not overlap on the GPU.  Launch shape: bs_autotune or
 * bs_set_launch.  bs_run uses it when the plan has BS_FLAG_FUSED. */
bs_status bs_cov_solve(const bs_plan *plan, const void *z_train, const float *delta_pair, bs_cf64 *R,
                       bs_cf32 *c, int32_t *info, bs_stream stream);

/* Times bs_cov_solve for every launch shape (128 threads per CTA; 1, 2, 3,
 * 4, 5, 6 or 8 persistent CTAs per SM) on the caller's buffers (3 runs each,
 * after one warm-up), keeps the fastest in the plan and returns it (any
 * output pointer may be NULL).  Synchronises `stream`; overwrites R, c,
 * info. */
bs_status bs_autotune(bs_plan *plan, const void *z_train, bs_cf64 *R, bs_cf32 *c, int32_t *info,
                      bs_stream stream, int32_t *threads, int32_t *ctas_per_sm, float *ms);

/* Choices of bs_autotune_pass (-1 where a stage was not tuned) and the
 * time of every candidate (ms per launch, < 0 where it does not apply). */
typedef struct {
    int32_t beamspace;       /* 0 warp per beam residue, 1 bulk-copy-staged Stockham, 2 one-shot,
                                3 tensor-core DFT (N = 1024, M = 2048) */
    int32_t covariance;      /* 0 CTA per pair, 1 warp per pair (K <= 128), 2 tensor cores (16-bit windows) */
    int32_t fused;           /* 1: covariance + solve as one persistent launch (bs_cov_solve) */
    int32_t ctas_per_sm;     /* of that launch, from bs_autotune */
    float beamspace_ms[4];
    float covariance_ms[3];
    float solve_ms;          /* bs_mvdr_solve after the chosen covariance */
    float fused_ms;          /* the fused launch at its best shape */
} bs_tune_report;

/* Autotunes a whole pass on the caller's buffers (buf->x holding a
 * representative raw cube): channelises once, then times every kernel
 * variant that applies to the plan for the beamspace stage and for the
 * covariance (each a different tiling of the same stage: a warp per beam
 * residue, bulk-copy-staged radix-16 passes, a one-shot CTA per group or
 * the tensor-core DFT;
 * a CTA, a warp or tensor-core fragments per pair), the fused covariance +
 * solve at every CTAs-per-SM shape (bs_autotune) against the two launches,
 * and keeps the fastest of each in the plan; bs_run, bs_run_host and
 * bs_graph_create use them from then on.  Results of the chosen variants
 * meet the same tolerances (their sums round differently).  Synchronises
 * `stream`; overwrites xc, the windows, R, c and info.  rep may be NULL. */
bs_status bs_autotune_pass(bs_plan *plan, const bs_buffers *buf, bs_stream stream, bs_tune_report *rep);

/* Sets the launch shape of bs_cov_solve (threads 128; 1..32 CTAs per SM). */
bs_status bs_set_launch(bs_plan *plan, int32_t threads, int32_t ctas_per_sm);

/* Allocation-free covariance + solve.  The paper has no counterpart: this
 * is a service for callers that may not allocate device memory while they
 * run (a real-time processing loop whose memory is fixed at start-up, where
 * an allocation could stall the device; a host application that owns all
 * device buffers and forbids libraries to allocate).  Such callers cannot
 * create a bs_plan (plan creation allocates), so every per-pair table is
 * passed in, as device arrays of `pairs` entries:
 *   W, K        window size (1..16) and training-vector count
 *               (1..2^24 - 1);
 *   ztr_off     element offset of the pair's K x W training windows in
 *               z_train (as bs_plan_offsets' ztr_off);
 *   woff        offset of the pair's W values in a_hi, a_lo, a_fp64 and c;
 *   a_hi, a_lo  windowed steering vectors as FP32 high and low parts
 *               (hi = (float)a, lo = (float)(a - hi)); a_fp64 the same in FP64.
 * Results are those of bs_cov_solve (R is not produced): c, info; a pair
 * whose W or K is out of range gets info = -3 and its c is not written.
 * delta must be finite and >= 0 (BS_EINVAL otherwise); pairs == 0 is a
 * no-op returning BS_OK.
 * This call allocates nothing: its scratch (queue head and cost-ordered pair
 * list) is a fixed array in device memory with room for 262144 pairs, held
 * by every GPU that loads the library until the process exits; larger
 * `pairs` are refused with BS_EINVAL.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) and caches it, so make
 * the first call on each device before any stream capture.  All calls share
 * the array: calls whose kernels could overlap on the GPU (other streams,
 * other host threads on the same device) race and must not be issued; each
 * call rewrites the parts it uses, so earlier contents do no harm. */
bs_status bs_cov_solve_noalloc(const void *z_train, int32_t precision, float store_scale,
                               const int32_t *W, const int32_t *K, const int64_t *ztr_off,
                               const int64_t *woff, const bs_cf32 *a_hi, const bs_cf32 *a_lo,
                               const bs_cf64 *a_fp64, int64_t pairs, double delta, double kappa_max,
                               uint32_t flags, bs_cf32 *c, int32_t *info, bs_stream stream);

/* Beamformer output (Sec. II-B): out[g][v'] = c_g^H z_test[g][v'], v' < Vte. */
bs_status bs_apply(const bs_plan *plan, const bs_cf32 *z_test, const bs_cf32 *c,
                   bs_cf32 *out, bs_stream stream);

/* Lifted correlator (Sec. III-C, Eq. AntennaEqCorr): c_hat_g = D^H S_g^T c_g,
 * the antenna-space weights whose output c_hat_g^H y equals the windowed
 * beamspace output c_g^H S_g D y.  c: weights packed as bs_mvdr_solve writes
 * them ([pair][W_g], offsets woff); c_hat: [pair][N] cf32 (caller-owned
 * device memory; pair g = t L + s).  Errors: BS_EINVAL for NULL buffers or a
 * wrong device, BS_EUNSUPPORTED for W > 16. */
bs_status bs_lift(const bs_plan *plan, const bs_cf32 *c, bs_cf32 *c_hat, bs_stream stream);

/* The lifted correlator applied in antenna space (Sec. III-C, below Eq.
 * AntennaEqCorr: no per-sample spatial FFT or window at inference):
 * out[g][v'] = c_hat_g^H y_v', y_v' the channelised element vector xc[p][q]
 * of test vector v' (record p = P_train + v'/B, bin q = s B + v' mod B) of
 * pair g's subband s.  xc: [P][F][N] as bs_channelize writes it; c_hat as
 * bs_lift writes it; out: [pair][Vte] cf32, the layout of bs_apply.  FP32
 * arithmetic; equals bs_apply's output up to rounding. */
bs_status bs_apply_lifted(const bs_plan *plan, const bs_cf32 *xc, const bs_cf32 *c_hat, bs_cf32 *out,
                          bs_stream stream);

/* Beam pattern of every lifted correlator (Eq. Cosine Sim):
 * pattern[g][k] = |c_hat_g^H a(Omega_gk)| / (||c_hat_g|| sqrt(N)) with
 * a(Omega) = [e^{j Omega n}]_n (Eq. ArrayX) and Omega_gk = pi u_k f_s / f_d,
 * f_s the centre frequency of pair g's subband (Eq. SubOmegaX).  u: device
 * array of n_dirs direction sines (FP64); pattern: device [pair][n_dirs]
 * FP32.  Distortionless weights give 1 / (||c_hat|| sqrt(N)) at the target. */
bs_status bs_beam_pattern(const bs_plan *plan, const bs_cf32 *c_hat, int32_t n_dirs, const double *u,
                          float *pattern, bs_stream stream);

/* Processing after the beamformer (Sec. II, Fig. 1: synthesis of the
 * wideband output, then standard range-Doppler processing): for target t,
 * test record r and FFT bin k, Y[t][r][k] is the beamformed output
 * out[t L + s][r B + i] of bin q = s B + i, k = (q - F/2) mod F; the matched
 * filter and the synthesis IFFT (orthonormal) give the range profiles
 * rp[t][r] = IFFT_k(Y[t][r][k] conj(P[k])), and the Doppler DFT over the
 * records the power map
 *   map[t][d][tau] = |sum_r rp[t][r][tau] e^{-j 2 pi d r / P_test}|^2.
 * out: bs_apply's output [pairs][Vte]; pulse: [F] cf32 orthonormal spectrum
 * of the transmitted pulse (FFT order); work: caller-owned device scratch of
 * 2 T P_test F cf32; map: [T][P_test][F] FP32.  F is a power of two in
 * 16..4096 (plan validation).  A subband-shard plan is refused
 * (BS_EUNSUPPORTED): every subband of a target enters its map. */
bs_status bs_range_doppler(const bs_plan *plan, const bs_cf32 *out, const bs_cf32 *pulse, bs_cf32 *work,
                           float *map, bs_stream stream);

/* CFAR detection (Sec. IV-B: a one-dimensional CFAR across all velocity
 * bins of the range-Doppler map, 10 dB above the noise floor in the paper):
 * the floor of cell (d, tau) of target t is the mean of the other
 * P_test - 1 velocity bins of the same range cell,
 *   floor[t][d][tau] = (sum_{d' != d} map[t][d'][tau]) / (P_test - 1)
 * (FP32, summed in order of d'; the cell under test is left out), and the
 * cell is a detection when map > floor * 10^(dB/10), compared in FP32.
 * floor: [T][P_test][F] FP32; count: [T] detections; mask (may be NULL):
 * [T][P_test][F] bytes, 1 for a detection; peak (may be NULL): [T] flat
 * index d F + tau of the strongest detected cell (the smallest index on
 * ties), -1 when the target has none -- its range and velocity bins, whose
 * differences from the truth are the paper's detection errors.
 * P_test == 0: no-op; P_test == 1: BS_EUNSUPPORTED. */
bs_status bs_cfar(const bs_plan *plan, const float *map, float threshold_db, float *floor, int32_t *count,
                  uint8_t *mask, int32_t *peak, bs_stream stream);

/* The whole pass on device buffers: channelise, beamspace, covariance,
 * solve (bs_cov_solve with BS_FLAG_FUSED), apply (delta = plan delta). */
bs_status bs_run(const bs_plan *plan, const bs_buffers *buf, bs_stream stream);

/* The whole pass from host memory: copies x_host ([P][F][N] cf32; pinned
 * memory makes the copy asynchronous and fast) into the device buffer
 * buf->x, runs the pass of bs_run, and copies buf->out back to out_host
 * ([pairs][Vte]). The copy is split into up to 8 record chunks issued on
 * a stream owned by the plan; channelisation and beamspace of chunk k run
 * on `stream` while chunk k+1 is copied, and the covariance and solve run
 * once the training records are done, while the test records are copied
 * (the last chunk is one record), so the host link, not the kernels, sets
 * the time. Results are those of bs_run bit for bit.
 * Synchronises `stream` before returning; one call per plan at a time. */
bs_status bs_run_host(const bs_plan *plan, const bs_cf32 *x_host, bs_cf32 *out_host,
                      const bs_buffers *buf, bs_stream stream);

/* CUDA graph of one whole pass (bs_run on `buf`), captured on `stream`
 * (must not be the legacy default stream).  Launch it as often as needed;
 * the buffers and plan must outlive it. */
typedef struct bs_graph bs_graph;
bs_status bs_graph_create(const bs_plan *plan, const bs_buffers *buf, bs_stream stream, bs_graph **graph);
bs_status bs_graph_launch(bs_graph *graph, bs_stream stream);
void      bs_graph_destroy(bs_graph *graph);
/* Number of kernel nodes in the captured pass (the kernels one launch of
 * the graph runs), written to *kernels. */
bs_status bs_graph_kernel_count(const bs_graph *graph, int32_t *kernels);

/* ---------------------------------------------------- learned loading --- */
/* A small MLP predicts, from a window's covariance estimated with few
 * training vectors (K = 2W), the diagonal loading delta and a diagonal
 * preconditioner d of the MVDR solve.  The paper loads nothing and learns
 * nothing (Eq. BeamCorrMVDR is solved as is); this follows the workload's
 * learned-loading direction, with plain MVDR at a fixed delta as fallback
 * and SINR judge.  Layers: n_in -> n_hidden -> n_hidden -> n_out, ReLU
 * between, y = [log10 delta, log10 d_1 .. log10 d_W]. */

/* Parameters (all device memory, caller-owned, P = bs_mlp_param_count()
 * floats each, layout W1 [H][n_in] | b1 [H] | W2 [H][H] | b2 [H] |
 * W3 [n_out][H] | b3 [n_out]).  master: FP32 parameters (Adam updates these);
 * weights_bf16: BF16 copy read by the forward and backward products (FP32
 * accumulation); grad, adam_m, adam_v: FP32.  step counts Adam updates. */
typedef struct {
    int32_t n_in, n_hidden, n_out;
    int32_t step;
    float *master;
    void *weights_bf16;
    float *grad, *adam_m, *adam_v;
} bs_mlp;

/* Activations of one batch (device, caller-owned): z1, h1, z2, h2, dh1, dh2
 * [capacity][n_hidden]; y, dy [capacity][n_out]. */
typedef struct {
    int64_t capacity;
    float *z1, *h1, *z2, *h2;
    float *y, *dy;
    float *dh1, *dh2;
} bs_mlp_work;

int64_t   bs_mlp_param_count(int32_t n_in, int32_t n_hidden, int32_t n_out);

/* Features of every pair (plan with one window size W for all targets) from
 * its unloaded covariance R (bs_window_cov with zero loading): with
 * tau = tr(R)/W, [diag(R)/tau | Re R_ij/tau (i > j, row-major) | Im R_ij/tau |
 * Re a~/|a~| | Im a~/|a~| | log10 tau | log10(K/W)], W^2 + 2W + 2 floats per
 * pair, X: [pairs][W^2 + 2W + 2]. */
bs_status bs_features(const bs_plan *plan, const bs_cf64 *R_unloaded, float *X, bs_stream stream);

/* Output SINR of each pair's weights against a reference covariance:
 * sinr[g] = |c^H a~|^2 / (c^H R_ref c) (FP64). */
bs_status bs_output_sinr(const bs_plan *plan, const bs_cf32 *c, const bs_cf64 *R_ref, double *sinr,
                         bs_stream stream);

/* Training targets: for each pair, the loading grid[k] of largest
 * sinr[k][pair] (first on ties), T[pair] = [log10 delta*,
 * -0.5 log10(R_ii + delta*)] (nout = 1 + W), best_delta (may be NULL). */
bs_status bs_loading_labels(const bs_plan *plan, const double *sinr, int32_t ngrid, const double *grid,
                            const bs_cf64 *R_unloaded, int32_t nout, float *T, float *best_delta,
                            bs_stream stream);

/* Forward pass: Y [batch][n_out] from X [batch][n_in] (batch <= capacity). */
bs_status bs_mlp_forward(const bs_mlp *mlp, const float *X, int64_t batch, float *Y, const bs_mlp_work *work,
                         bs_stream stream);

/* One training step on a batch: forward (into work->y), mean-squared-error
 * gradient against T [batch][n_out] (loss, if not NULL, is incremented by the
 * batch loss, FP64 device scalar), backward, and an Adam update (lr > 0;
 * beta 0.9 / 0.999, eps 1e-8, bias-corrected) of master with a fresh BF16
 * copy.  lr = 0 stops after the gradients (left in mlp->grad). */
bs_status bs_mlp_train_step(bs_mlp *mlp, const float *X, const float *T, int64_t batch, const bs_mlp_work *work,
                            float lr, double *loss, bs_stream stream);

/* Refresh the BF16 weight copy from master. */
bs_status bs_mlp_sync_bf16(const bs_mlp *mlp, bs_stream stream);

/* dst[r] = src[idx[r]] for rows of `cols` floats (minibatch assembly). */
bs_status bs_gather_rows(const float *src, const int64_t *idx, int64_t rows, int32_t cols, float *dst,
                         bs_stream stream);

/* delta[g] = 10^Y[g][0] clipped to [lo, hi]; non-finite -> fallback.  The
 * result feeds bs_window_cov's per-pair loading. */
bs_status bs_loading_from_mlp(const float *Y, int32_t nout, int64_t pairs, float lo, float hi, float fallback,
                              float *delta, bs_stream stream);

/* The preconditioner seed: d[g][i] = 10^Y[g][1 + i], i < W (plans with one
 * window size W; nout >= 1 + W), non-finite -> 1.  d: device [pairs][W],
 * the packing of bs_mvdr_solve_precond's d for such plans. */
bs_status bs_precond_from_mlp(const float *Y, int32_t nout, int64_t pairs, int32_t W, float *d, bs_stream stream);

/* ------------------------------------------------------------- errors --- */
const char *bs_status_string(bs_status s);
const char *bs_last_error(void);   /* thread-local text of the last error */

#ifdef __cplusplus
}
#endif
#endif /* BS_H */
