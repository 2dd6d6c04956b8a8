// Record chunks of the host pipeline (bs_run_host): plain C++, no CUDA, so
// that the schedule can be checked on its own.
//
// Records [0, P_train) are training records and [P_train, P_train + P_test)
// test records.  The schedule has at most `max_chunks` chunks, every one
// non-empty; a chunk boundary falls at P_train (the covariance and solve
// need only the training windows, so they can run while the test records are
// still being copied), the test records get up to three chunks of which the
// last holds one record (little work is left after the last copy), and the
// training records share the remaining chunks evenly.
#pragma once

namespace bs {

// Fills bounds[0..n] (bounds[0] = 0, bounds[n] = P_train + P_test, strictly
// increasing) and returns n.  Needs P_train >= 1, P_test >= 0, max_chunks >= 4
// and room for max_chunks + 1 entries.
inline int host_chunk_bounds(int P_train, int P_test, int max_chunks, int *bounds) {
    const int nte = P_test > 0 ? (P_test < 3 ? P_test : 3) : 0;
    int ntr = max_chunks - nte;
    if (ntr > P_train) ntr = P_train;
    if (ntr < 1) ntr = 1;
    int n = 0;
    bounds[0] = 0;
    for (int k = 1; k <= ntr; ++k) bounds[++n] = (int)((long long)P_train * k / ntr);
    if (nte > 0) {   // nte - 1 even chunks, then one record
        for (int k = 1; k < nte; ++k) bounds[++n] = P_train + (int)((long long)(P_test - 1) * k / (nte - 1));
        bounds[++n] = P_train + P_test;
    }
    return n;
}

}  // namespace bs
