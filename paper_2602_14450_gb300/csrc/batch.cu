// wd_solve_batch: several right-hand sides on several lattices in one launch
// chain. Each kernel of the inner iteration covers all right-hand sides of a
// lattice (blocks of different right-hand sides interleaved, so that blocks
// running together read the same links and share them through L2); the
// iterations of all lattices are captured into one CUDA graph.
#include "handle.h"

namespace wd {
int solve_systems(int n, wd_handle* const* hs, const int* nrhs, const double* const* b, double* const* x, double tol,
                  int scheme, const wd_solve_params* params, wd_solve_stats* stats, cudaStream_t s);
}

extern "C" int wd_solve_batch(int n, wd_handle* const* h, const int* nrhs, const double* const* b, double* const* x,
                              double tol, int scheme, const wd_solve_params* params, wd_solve_stats* per_rhs_stats,
                              void* stream) {
    if (n < 1 || !h || !nrhs || !b || !x) return WD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!h[i] || nrhs[i] < 0 || (nrhs[i] > 0 && (!b[i] || !x[i]))) return WD_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (h[i]->g.part) return wd::fail(h[i], WD_ERR_INVALID_ARG, "wd_solve_batch: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    return wd::solve_systems(n, h, nrhs, b, x, tol, scheme, params, per_rhs_stats, (cudaStream_t)stream);
}
