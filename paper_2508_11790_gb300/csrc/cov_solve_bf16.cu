// Fused covariance + solve kernel instantiated for bf16 training windows.
#include "cov_solve_dev.cuh"

namespace bs {

template <>
bs_status launch_cs_prec<BS_PREC_BF16>(const CovSolveArgs &a, int grid, cudaStream_t st) {
    return launch_cs_t<BS_PREC_BF16, 128>(a, grid, st);
}

}  // namespace bs
