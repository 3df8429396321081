// wd_solve_batch: several right-hand sides on several lattices.
#include "handle.h"

extern "C" int wd_solve_batch(int n, wd_handle* const* h, const int* nrhs, const double* const* b, double* const* x,
                              double tol, int scheme, const wd_solve_params* params, wd_solve_stats* per_rhs_stats,
                              void* stream) {
    if (n < 1 || !h || !nrhs || !b || !x) return WD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!h[i] || nrhs[i] < 0 || (nrhs[i] > 0 && (!b[i] || !x[i]))) return WD_ERR_INVALID_ARG;
    int worst = WD_OK;
    int k = 0;
    for (int i = 0; i < n; ++i) {
        const size_t len = (size_t)2 * h[i]->g.Vh * 24;
        for (int j = 0; j < nrhs[i]; ++j, ++k) {
            wd_solve_stats st{};
            int rc = wd_solve(h[i], b[i] + j * len, x[i] + j * len, tol, scheme, params, &st, stream);
            if (per_rhs_stats) per_rhs_stats[k] = st;
            if (rc == WD_ERR_INVALID_ARG || rc == WD_ERR_CUDA || rc == WD_ERR_NO_GAUGE || rc == WD_ERR_NOT_SU3) return rc;
            if (rc != WD_OK && worst == WD_OK) worst = rc;
        }
    }
    return worst;
}
