// Launchers of the fused covariance + solve kernel (cov_solve_dev.cuh): from
// a plan, and from explicit per-pair tables.
#include "cov_solve_dev.cuh"

namespace bs {

bs_status launch_cov_solve(const bs_plan *p, const void *ztr, const float *delta, double2 *R, float2 *c,
                           int32_t *info, int *head, const CovSolveLaunch &cfg, cudaStream_t st) {
    if (p->Wmax > WMAX) return set_error(BS_EUNSUPPORTED, "W > 16");
    CovSolveArgs a;
    a.z = ztr;
    a.ztr_off = p->d_ztr_off;
    a.Wg = p->d_Wg;
    a.Kg = p->d_Kg;
    a.woff = p->d_woff;
    a.roff = p->d_roff;
    a.at32 = p->d_at32;
    a.atlo = p->d_atlo;
    a.at64 = p->d_at64;
    a.order = p->d_order;
    a.pairs = p->pairs;
    a.delta_pair = delta;
    a.delta = p->cfg.delta;
    a.delta_df = df_from_double(p->cfg.delta);
    a.inv_sc = 1.0f / p->cfg.store_scale;
    a.kappa_max = p->cfg.kappa_max;
    a.refine = (p->cfg.flags & BS_FLAG_NO_REFINE) ? 0 : 1;
    a.allow_f64 = (p->cfg.flags & BS_FLAG_NO_FP64) ? 0 : 1;
    a.c = c;
    a.info = info;
    a.R = R;
    a.head = head;
    cudaError_t e = cudaMemsetAsync(head, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "work queue reset");
    long long grid = (long long)p->num_sms * (cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : 5);
    if (grid > p->pairs) grid = p->pairs;
    if (grid < 1) grid = 1;
    switch (p->cfg.precision) {
        case BS_PREC_FP32: return launch_cs_prec<BS_PREC_FP32>(a, (int)grid, st);
        case BS_PREC_FP16: return launch_cs_prec<BS_PREC_FP16>(a, (int)grid, st);
        default: return launch_cs_prec<BS_PREC_BF16>(a, (int)grid, st);
    }
}

// Launch of the fused kernel from explicit per-pair device tables (no plan),
// for the allocation-free entry point.  `order` / `head` point into the
// caller's scratch; R is not produced.
bs_status launch_cov_solve_tables(const void *z, int precision, float store_scale, const int32_t *Wg,
                                  const int32_t *Kg, const int64_t *ztr_off, const int64_t *woff,
                                  const float2 *at32, const float2 *atlo, const double2 *at64,
                                  const int32_t *order, int64_t pairs, double delta, double kappa_max,
                                  uint32_t flags, float2 *c, int32_t *info, int *head, int grid,
                                  cudaStream_t st) {
    CovSolveArgs a;
    a.z = z;
    a.ztr_off = ztr_off;
    a.Wg = Wg;
    a.Kg = Kg;
    a.woff = woff;
    a.roff = nullptr;
    a.at32 = at32;
    a.atlo = atlo;
    a.at64 = at64;
    a.order = order;
    a.pairs = pairs;
    a.delta_pair = nullptr;
    a.delta = delta;
    a.delta_df = df_from_double(delta);
    a.inv_sc = 1.0f / store_scale;
    a.kappa_max = kappa_max;
    a.refine = (flags & BS_FLAG_NO_REFINE) ? 0 : 1;
    a.allow_f64 = (flags & BS_FLAG_NO_FP64) ? 0 : 1;
    a.c = c;
    a.info = info;
    a.R = nullptr;
    a.head = head;
    switch (precision) {
        case BS_PREC_FP32: return launch_cs_prec<BS_PREC_FP32>(a, grid, st);
        case BS_PREC_FP16: return launch_cs_prec<BS_PREC_FP16>(a, grid, st);
        default: return launch_cs_prec<BS_PREC_BF16>(a, grid, st);
    }
}

}  // namespace bs
