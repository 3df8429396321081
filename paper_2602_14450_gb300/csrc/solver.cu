// Solver driver: FP64 iterative refinement (Alg. 2 / Alg. 3) around the
// rescaled low-precision BiCGStab (Alg. 4 / Alg. 5) on the even-odd system of
// Eq. 4, followed by the odd-site reconstruction of Eq. 5, for a batch of
// systems (lattices), each with one or more right-hand sides.
//
// Device-resident design: every scalar of the recurrences lives in a
// SolverState (one per right-hand side) in device memory and is updated by
// the last block of the reducing kernel that produces its inputs. One inner
// BiCGStab iteration of every system is a fixed chain of 7-8 kernels, each
// launch covering all right-hand sides of a system (blocks of different
// right-hand sides interleaved so that they share links through L2); several
// iterations are captured in one CUDA graph. Kernels of a right-hand side
// whose inner solve is done return at once; the host polls one flag per
// graph launch, one launch behind. Right-hand sides that have converged in
// the refinement loop are marked `skip` and every later kernel leaves them
// alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handle.h"

namespace wd {

struct SchemeCfg {
    int prec;          // inner storage precision
    bool fp64_inner;   // WD_FP64_BICGSTAB: the "inner" solve is the whole solve
    bool learned;      // inner BiCGStab on A M with the learned right preconditioner
};

cudaError_t ptc_apply_m(wd_handle* h, int prec, const uint4* in_e, uint4* out_e, uint4* PHI, const float2* V,
                        const uint4* le, const uint4* lo, cudaStream_t s, const SolverState* guard, int* err);
int* ptc_err(wd_handle* h);
const float2* ptc_collapsed(wd_handle* h);
uint4* ptc_phi16(wd_handle* h);

static bool scheme_cfg(int scheme, SchemeCfg* c) {
    c->learned = scheme == WD_MIXED_FP16_LEARNED;
    switch (scheme) {
    case WD_FP64_BICGSTAB: c->prec = WD_FP64; c->fp64_inner = true; return true;
    case WD_MIXED_FP16_LEARNED: c->prec = WD_FP16; c->fp64_inner = false; return true;
    case WD_MIXED_FP32: c->prec = WD_FP32; c->fp64_inner = false; return true;
    case WD_MIXED_FP16_PLAIN: c->prec = WD_FP16; c->fp64_inner = false; return true;
    case WD_MIXED_FP16: c->prec = WD_FP16; c->fp64_inner = false; return true;
    case WD_MIXED_BF16: c->prec = WD_BF16; c->fp64_inner = false; return true;
    default: return false;
    }
}

// Flag "some right-hand side of this system is still in its inner solve".
// flag := "some right-hand side of the system is still iterating" (or_in = 0), or
// flag |= it (or_in = 1: the systems after the first of a batch).
__global__ void k_any_active(int nrhs, const SolverState* st, int* flag, int or_in) {
    const int r = threadIdx.x;
    const bool act = r < nrhs && !st[r].done && !st[r].skip;
    const int any = __syncthreads_or(act) ? 1 : 0;
    if (r == 0 && (any || !or_in)) *(volatile int*)flag = any;
}

// Device buffers of one system for one call.
struct Sys {
    wd_handle* h = nullptr;
    int nrhs = 0;
    const double* b = nullptr;
    double* x = nullptr;
    bool b_dev = true, x_dev = true;
    double* bl = nullptr;       // device lexicographic sources (b or staging)
    double* xl = nullptr;       // device lexicographic solutions (x or staging)
    const uint4 *le64 = nullptr, *lo64 = nullptr, *le = nullptr, *lo = nullptr;
    long long vs64 = 0, vs = 0; // units per right-hand side
    uint4 *eta_e, *eta_o, *bhat, *x64, *r64, *tmp64, *xo;             // FP64, nrhs each
    uint4 *r, *rs, *p, *v, *t, *xt, *tmp;                              // inner precision, nrhs each
    uint4 *phat = nullptr, *shat = nullptr, *PHI = nullptr;            // M p, M s, fields of the collapsed M
    const float2* V = nullptr;                                         // collapsed preconditioner weights
    int* err = nullptr;                                                // raised by a bounded wait that gave up
    // clover blocks (null without a clover term): C^-1 in FP64 and in the inner precision, C in FP64
    const uint4 *mi64e = nullptr, *mi64o = nullptr, *mf64e = nullptr, *mf64o = nullptr, *mie = nullptr, *mio = nullptr;
    std::vector<double> eta_norm;
    std::vector<bool> active;
};

static int prepare(Sys& S, int prec, int recon_lo, bool learned) {
    wd_handle* h = S.h;
    if (learned) {
        if (!h->have_precond) return fail(h, WD_ERR_INVALID_ARG, "learned scheme: no preconditioner weights loaded");
        if (S.nrhs != 1) return fail(h, WD_ERR_INVALID_ARG, "learned scheme: one right-hand side per lattice");
    }
    int rc = ensure_solver_state(h, S.nrhs);
    if (rc != WD_OK) return rc;
    if ((rc = ensure_links(h, WD_FP64, 18, &S.le64, &S.lo64)) != WD_OK) return rc;
    if ((rc = ensure_links(h, prec, recon_lo, &S.le, &S.lo)) != WD_OK) return rc;
    if (h->have_clover) {
        if (learned) return fail(h, WD_ERR_INVALID_ARG, "learned scheme: not available with a clover term");
        if ((rc = ensure_clover(h, WD_FP64, 0, &S.mi64e, &S.mi64o)) != WD_OK) return rc;
        if ((rc = ensure_clover(h, WD_FP64, 1, &S.mf64e, &S.mf64o)) != WD_OK) return rc;
        if ((rc = ensure_clover(h, prec, 0, &S.mie, &S.mio)) != WD_OK) return rc;
    }
    const size_t b64 = vec_bytes(h, WD_FP64) * S.nrhs, blo = vec_bytes(h, prec) * S.nrhs;
    S.vs64 = (long long)spinor_units(WD_FP64) * h->g.Vh;
    S.vs = (long long)spinor_units(prec) * h->g.Vh;
    uint4** f64[7] = {&S.eta_e, &S.eta_o, &S.bhat, &S.x64, &S.r64, &S.tmp64, &S.xo};
    const char* n64[7] = {"eta_e", "eta_o", "bhat", "x", "r", "tmp", "xo"};
    for (int i = 0; i < 7; ++i) {
        *f64[i] = (uint4*)workspace(h, std::string("f64.") + n64[i], b64);
        if (!*f64[i]) return fail(h, WD_ERR_CUDA, "out of device memory (%s)", n64[i]);
    }
    uint4** flo[7] = {&S.r, &S.rs, &S.p, &S.v, &S.t, &S.xt, &S.tmp};
    const char* nlo[7] = {"r", "rs", "p", "v", "t", "x", "tmp"};
    const std::string pre = "in" + std::to_string(prec) + ".";
    for (int i = 0; i < 7; ++i) {
        *flo[i] = (uint4*)workspace(h, pre + nlo[i], blo);
        if (!*flo[i]) return fail(h, WD_ERR_CUDA, "out of device memory (%s)", nlo[i]);
    }
    // raised by any kernel of the solve whose bounded device wait gave up
    S.err = ptc_err(h);
    if (!S.err) return fail(h, WD_ERR_CUDA, "out of device memory");
    if (cudaMemset(S.err, 0, sizeof(int)) != cudaSuccess) return fail(h, WD_ERR_CUDA, "cudaMemset");
    if (learned) {
        S.phat = (uint4*)workspace(h, pre + "phat", blo);
        S.shat = (uint4*)workspace(h, pre + "shat", blo);
        S.PHI = ptc_phi16(h);
        S.V = ptc_collapsed(h);
        if (!S.phat || !S.shat || !S.PHI || !S.V)
            return fail(h, WD_ERR_CUDA, "out of device memory (preconditioner)");
    }
    const size_t lexb = (size_t)S.nrhs * 2 * h->g.Vh * 24 * sizeof(double);
    S.bl = const_cast<double*>(S.b);
    S.xl = S.x;
    if (!S.b_dev || !S.x_dev) {
        double* stage = (double*)workspace(h, "lex.stage", lexb);
        if (!stage) return fail(h, WD_ERR_CUDA, "out of device memory");
        if (!S.b_dev) S.bl = stage;
        if (!S.x_dev) S.xl = stage;   // b is consumed (packed) before x is written
    }
    S.eta_norm.assign(S.nrhs, 0.0);
    S.active.assign(S.nrhs, false);
    return WD_OK;
}

static HopParams hop_params(const Sys& S, int stage, int guard_kind) {
    HopParams P{};
    P.g = S.h->g;
    P.nrhs = S.nrhs;
    P.rc = red_ctx(S.h, stage);
    P.guard = S.h->st;
    P.guard_kind = guard_kind;
    P.wait_rounds = S.h->wait_rounds;
    P.err = S.err;
    return P;
}

// One FP64 hop over all right-hand sides of a system.
static cudaError_t hop64(const Sys& S, int parity, const uint4* in, uint4* out, int epi, int red, double a,
                         const uint4* y, double b, const uint4* z, double c, int stage, int guard_kind,
                         cudaStream_t s, const uint4* mat = nullptr) {
    HopParams P = hop_params(S, stage, guard_kind);
    apply_tuning(S.h, WD_FP64, 18, P);
    P.mat = mat;
    P.vs = S.vs64;
    P.parity = parity;
    P.links = parity == 0 ? S.le64 : S.lo64;
    P.in = in;
    P.out = out;
    P.y = y;
    P.z = z;
    P.a = a;
    P.b = b;
    P.c = c;
    return Ops<double>::hop(18, epi, red, P, s);
}

// Enqueue one inner BiCGStab iteration (Alg. 4 / Alg. 5 loop body) of every
// right-hand side of a system; with a right preconditioner M the operator is
// A M: v = A (M p), t = A (M s), x += lambda'/gamma' (omega M s + alpha M p).
static cudaError_t enqueue_iteration(const Sys& S, int prec, int recon, int xr_mode, bool learned,
                                     cudaStream_t s) {
    const int n = S.h->g.Vh, nr = S.nrhs;
    const long long vs = S.vs;
    const double k2 = S.h->kappa * S.h->kappa;
    SolverState* st = S.h->st;
    wd_handle* h = S.h;
    return by_prec(prec, [&](auto tag) -> cudaError_t {
        typedef typename decltype(tag)::type T;
        cudaError_t e;
        HopParams P = hop_params(S, ST_NONE, GUARD_INNER);
        apply_tuning(h, prec, recon, P);
        P.vs = vs;
        // p := beta (p - omega' v) + r   (gamma of p and v folded in)
        if ((e = Ops<T>::pupdate(n, nr, vs, S.p, S.v, S.r, st, s)) != cudaSuccess) return e;
        const uint4* pa = S.p;   // operand of A
        if (learned) {
            if ((e = ptc_apply_m(h, WD_FP16, S.p, S.phat, S.PHI, S.V, S.le, S.lo, s, st, S.err)) != cudaSuccess) return e;
            pa = S.phat;
        }
        // v = A p = p - kappa^2 H_eo H_oe p ; alpha = rho / (r*, v)
        P.parity = 1; P.links = S.lo; P.in = pa; P.out = S.tmp; P.a = 1.0; P.mat = S.mio;
        if ((e = Ops<T>::hop(recon, EPI_H, RED_NONE, P, s)) != cudaSuccess) return e;
        P.parity = 0; P.links = S.le; P.in = S.tmp; P.out = S.v; P.y = pa; P.a = -k2; P.b = 1.0; P.mat = S.mie;
        P.rstar = S.rs; P.rc = red_ctx(h, ST_ALPHA);
        if ((e = Ops<T>::hop(recon, EPI_Y, RED_RSV, P, s)) != cudaSuccess) return e;
        // r := r - alpha v
        if ((e = Ops<T>::supdate(n, nr, vs, S.r, S.v, st, s)) != cudaSuccess) return e;
        const uint4* sa = S.r;   // operand of A
        if (learned) {
            if ((e = ptc_apply_m(h, WD_FP16, S.r, S.shat, S.PHI, S.V, S.le, S.lo, s, st, S.err)) != cudaSuccess) return e;
            sa = S.shat;
        }
        // t = A s ; omega from (t, s), (t, t), (s, s)
        P.rc = red_ctx(h, ST_NONE);
        P.parity = 1; P.links = S.lo; P.in = sa; P.out = S.tmp; P.y = nullptr; P.a = 1.0; P.b = 0.0;
        P.rstar = nullptr; P.mat = S.mio;
        if ((e = Ops<T>::hop(recon, EPI_H, RED_NONE, P, s)) != cudaSuccess) return e;
        P.parity = 0; P.links = S.le; P.in = S.tmp; P.out = S.t; P.y = sa; P.a = -k2; P.b = 1.0; P.mat = S.mie;
        P.rstar = learned ? S.r : nullptr;   // dot partner s when t = A M s
        P.rc = red_ctx(h, ST_OMEGA);
        if ((e = Ops<T>::hop(recon, EPI_Y, RED_TS, P, s)) != cudaSuccess) return e;
        // x += lambda'/gamma' (omega s + alpha p) ; r := s - omega t ; |r|, |x|
        //   (with XR_FUSED r is stored rescaled and the iteration ends here)
        if ((e = Ops<T>::xr(xr_mode, n, nr, vs, S.xt, S.r, S.p, S.t, S.rs, learned ? S.shat : nullptr,
                            learned ? S.phat : nullptr, st, red_ctx(h, xr_mode == XR_FUSED ? ST_RFUSED : ST_RNORM),
                            s)) != cudaSuccess)
            return e;
        // r := (sigma / g) r ; gamma ; [x := lambda x] ; next rho, beta
        if (xr_mode == XR_NORMS)
            if ((e = Ops<T>::scale(n, nr, vs, S.r, S.xt, S.rs, st, red_ctx(h, ST_END), s)) != cudaSuccess) return e;
        return cudaSuccess;
    });
}

// Capture `iters` iterations of every system plus the activity flag. Systems
// of different handles are independent (their own vectors, scalar states,
// partial sums and tickets), so each is captured on its own handle's stream,
// forked from and joined back into the first: the graph runs the lattices'
// iterations side by side, and the kernels of a small lattice overlap those of
// a large one instead of queueing behind them.
static int capture_inner(std::vector<Sys>& sys, int prec, int recon, int xr_mode, bool learned, int iters,
                         cudaGraphExec_t* out) {
    wd_handle* h0 = sys[0].h;
    bool branches = sys.size() > 1;
    for (size_t i = 0; i < sys.size() && branches; ++i)
        for (size_t j = 0; j < i; ++j)
            if (sys[i].h == sys[j].h) branches = false;   // one handle twice: its stream cannot fork from itself
    cudaGraph_t graph = nullptr;
    WD_CUDA(h0, cudaStreamBeginCapture(h0->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    if (branches) {
        e = cudaEventRecord(h0->ev[1], h0->cap);                                   // fork
        for (size_t i = 1; i < sys.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(sys[i].h->cap, h0->ev[1], 0);
        for (size_t i = 0; i < sys.size() && e == cudaSuccess; ++i)
            for (int it = 0; it < iters && e == cudaSuccess; ++it)
                e = enqueue_iteration(sys[i], prec, recon, xr_mode, learned, sys[i].h->cap);
        for (size_t i = 1; i < sys.size() && e == cudaSuccess; ++i) {              // join
            e = cudaEventRecord(sys[i].h->ev[0], sys[i].h->cap);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h0->cap, sys[i].h->ev[0], 0);
        }
    } else {
        for (int i = 0; i < iters && e == cudaSuccess; ++i)
            for (auto& S : sys)
                if (e == cudaSuccess) e = enqueue_iteration(S, prec, recon, xr_mode, learned, h0->cap);
    }
    for (size_t i = 0; i < sys.size() && e == cudaSuccess; ++i) {   // the activity flag, in mapped host memory
        k_any_active<<<1, 1024, 0, h0->cap>>>(sys[i].nrhs, sys[i].h->st, h0->dflag, i > 0 ? 1 : 0);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(h0->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h0, e, "capture of the inner iteration");
    }
    WD_CUDA(h0, e2);
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    WD_CUDA(h0, e);
    return WD_OK;
}

static int read_states(std::vector<Sys>& sys, cudaStream_t s) {
    for (auto& S : sys)
        WD_CUDA(S.h, cudaMemcpyAsync(S.h->hst, S.h->st, sizeof(SolverState) * S.nrhs, cudaMemcpyDeviceToHost, s));
    WD_CUDA(sys[0].h, cudaStreamSynchronize(s));
    return WD_OK;
}

static int write_states(std::vector<Sys>& sys, cudaStream_t s) {
    for (auto& S : sys)
        WD_CUDA(S.h, cudaMemcpyAsync(S.h->st, S.h->hst, sizeof(SolverState) * S.nrhs, cudaMemcpyHostToDevice, s));
    return WD_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The driver behind wd_solve and wd_solve_batch.
int solve_systems(int n, wd_handle* const* hs, const int* nrhs, const double* const* b, double* const* x, double tol,
                  int scheme, const wd_solve_params* params, wd_solve_stats* stats, cudaStream_t s) {
    wd_handle* h0 = hs[0];
    SchemeCfg cfg;
    if (!(tol > 0) || !scheme_cfg(scheme, &cfg)) return fail(h0, WD_ERR_INVALID_ARG, "bad tolerance or scheme");
    wd_solve_params prm;
    if (params) prm = *params; else wd_solve_params_default(scheme, &prm);
    if (!valid_recon(prm.recon) || prm.max_outer < 1 || prm.max_inner < 2 || !(prm.s > 0) || prm.sigma < 0 ||
        prm.iters_per_sync < 1 || (prm.rescale_x && !(prm.sigma_lambda > 0)))
        return fail(h0, WD_ERR_INVALID_ARG, "bad solver parameters");
    const int prec = cfg.prec;
    const int recon_lo = cfg.fp64_inner ? 18 : prm.recon;
    // rescaling of r (Alg. 4): none (sigma = 0), fused into the r-update, or a separate pass (also the
    // pass that rescales x in Alg. 5)
    const int xr_mode = prm.rescale_x ? XR_NORMS : !(prm.sigma > 0) ? XR_PLAIN : prm.fused_rescale ? XR_FUSED : XR_NORMS;
    const bool scale_pass = xr_mode == XR_NORMS;
    const int ips = prm.iters_per_sync;
    const int kpi = (scale_pass ? 8 : 7) + (cfg.learned ? 4 : 0);   // kernels per inner iteration

    std::vector<Sys> sys;
    int total_rhs = 0;
    for (int i = 0; i < n; ++i) {
        if (nrhs[i] == 0) continue;
        Sys S;
        S.h = hs[i];
        S.nrhs = nrhs[i];
        S.b = b[i];
        S.x = x[i];
        if (!S.h->have_gauge) return fail(S.h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
        for (auto& o : sys)
            if (o.h == S.h) return fail(S.h, WD_ERR_INVALID_ARG, "a handle appears twice in one batch");
        S.b_dev = is_device_ptr(S.b);
        S.x_dev = is_device_ptr(S.x);
        int rc = prepare(S, prec, recon_lo, cfg.learned);
        if (rc != WD_OK) return rc;
        sys.push_back(S);
        total_rhs += S.nrhs;
    }
    if (sys.empty()) return WD_OK;
    if (total_rhs > 1024) return fail(h0, WD_ERR_INVALID_ARG, "at most 1024 right-hand sides per call");

    long long nk = 0;   // kernels launched by this call
    std::vector<wd_solve_stats> out(total_rhs);
    WD_CUDA(h0, cudaEventRecord(h0->t0, s));
    // Eq. 4 right-hand side b^ = eta_e + kappa H_eo eta_o, |eta|^2, and r = b^ - A x
    for (auto& S : sys) {
        wd_handle* h = S.h;
        const int nv = h->g.Vh;
        const size_t len = (size_t)2 * nv * 24;
        const size_t lexb = S.nrhs * len * sizeof(double);
        if (!S.b_dev) WD_CUDA(h, cudaMemcpyAsync(S.bl, S.b, lexb, cudaMemcpyHostToDevice, s));
        for (int r = 0; r < S.nrhs; ++r) {
            WD_CUDA(h, Ops<double>::pack(h->g, 0, S.bl + r * len, S.eta_e + r * S.vs64, s));
            WD_CUDA(h, Ops<double>::pack(h->g, 1, S.bl + r * len, S.eta_o + r * S.vs64, s));
        }
        for (int r = 0; r < S.nrhs; ++r) h->hst[r].skip = 0;
        WD_CUDA(h, cudaMemcpyAsync(h->st, h->hst, sizeof(SolverState) * S.nrhs, cudaMemcpyHostToDevice, s));
        WD_CUDA(h, Ops<double>::norm2(nv, S.nrhs, S.vs64, S.eta_e, red_ctx(h, ST_ACC_SET), GUARD_NONE, s));
        WD_CUDA(h, Ops<double>::norm2(nv, S.nrhs, S.vs64, S.eta_o, red_ctx(h, ST_ACC), GUARD_NONE, s));
        if (S.mi64e) {   // b^ = C_ee^-1 (eta_e + kappa H_eo C_oo^-1 eta_o)
            WD_CUDA(h, Ops<double>::apply_chiral(nv, S.nrhs, S.vs64, S.mi64o, S.eta_o, S.tmp64, s));
            WD_CUDA(h, Ops<double>::apply_chiral(nv, S.nrhs, S.vs64, S.mi64e, S.eta_e, S.bhat, s));
            WD_CUDA(h, hop64(S, 0, S.tmp64, S.bhat, EPI_Y, RED_NONE, h->kappa, S.bhat, 1.0, nullptr, 0.0, ST_NONE,
                             GUARD_NONE, s, S.mi64e));
            nk += 2;
        } else {
            WD_CUDA(h, hop64(S, 0, S.eta_o, S.bhat, EPI_Y, RED_NONE, h->kappa, S.eta_e, 1.0, nullptr, 0.0, ST_NONE,
                             GUARD_NONE, s));
        }
        nk += 2 * S.nrhs + 3;
        if (prm.x_is_guess) {
            if (!S.x_dev) WD_CUDA(h, cudaMemcpyAsync(S.xl, S.x, lexb, cudaMemcpyHostToDevice, s));
            for (int r = 0; r < S.nrhs; ++r)
                WD_CUDA(h, Ops<double>::pack(h->g, 0, S.xl + r * len, S.x64 + r * S.vs64, s));
            WD_CUDA(h, hop64(S, 1, S.x64, S.tmp64, EPI_H, RED_NONE, 1.0, nullptr, 0.0, nullptr, 0.0, ST_NONE,
                             GUARD_NONE, s, S.mi64o));
            WD_CUDA(h, hop64(S, 0, S.tmp64, S.r64, EPI_YZ, RED_NORM, h->kappa * h->kappa, S.bhat, 1.0, S.x64, -1.0,
                             ST_OUTER, GUARD_NONE, s, S.mi64e));
            nk += S.nrhs + 2;
        } else {
            WD_CUDA(h, cudaMemsetAsync(S.x64, 0, vec_bytes(h, WD_FP64) * S.nrhs, s));
            WD_CUDA(h, cudaMemcpyAsync(S.r64, S.bhat, vec_bytes(h, WD_FP64) * S.nrhs, cudaMemcpyDeviceToDevice, s));
            WD_CUDA(h, Ops<double>::norm2(nv, S.nrhs, S.vs64, S.r64, red_ctx(h, ST_OUTER), GUARD_NONE, s));
            nk += 1;
        }
    }
    int rc = read_states(sys, s);
    if (rc != WD_OK) return rc;

    // inner-iteration graph: cached in the handle for single-system calls
    cudaGraphExec_t exec = nullptr;
    bool own_exec = false;
    if (sys.size() == 1) {
        GraphKey key{prec, recon_lo, xr_mode | (cfg.learned ? 4 : 0), ips, sys[0].nrhs, h0->gen};
        auto it = h0->graphs.find(key);
        if (it != h0->graphs.end()) {
            exec = it->second;
        } else {
            if ((rc = capture_inner(sys, prec, recon_lo, xr_mode, cfg.learned, ips, &exec)) != WD_OK) return rc;
            h0->graphs[key] = exec;
        }
    } else {
        if ((rc = capture_inner(sys, prec, recon_lo, xr_mode, cfg.learned, ips, &exec)) != WD_OK) return rc;
        own_exec = true;
    }
    long long graph_kernels = 0;
    for (size_t i = 0; i < sys.size(); ++i) graph_kernels += (long long)ips * kpi + 1;

    std::vector<int> status(total_rhs, WD_OK);
    int trips = 0;

    // convergence history (one system with one right-hand side): device log of
    // the inner iterations of a trip, copied out and mapped after each trip
    const bool hist_on = prm.history && prm.history_cap > 0 && sys.size() == 1 && sys[0].nrhs == 1;
    const int hist_iters = prm.max_inner / 2 + 2;
    double* dhist = nullptr;
    if (hist_on) {
        dhist = (double*)workspace(h0, "hist", sizeof(double) * 2 * hist_iters);
        if (!dhist) return fail(h0, WD_ERR_CUDA, "out of device memory (history)");
    }
    std::vector<double> hbuf;
    int hlen = 0;
    long long hcum = 0;                 // low-precision matvecs so far
    double trip_res = 0.0, trip_rn = 0.0;
    auto hist_put = [&](double kind, double mv, double res, double nz) {
        if (hlen >= prm.history_cap) return;
        double* e = prm.history + 4 * (size_t)hlen++;
        e[0] = kind;
        e[1] = mv;
        e[2] = res;
        e[3] = nz;
    };

    for (;;) {
        // decide, per right-hand side, whether to continue (outer stopping rule)
        bool any = false;
        int k = 0;
        for (auto& S : sys) {
            for (int r = 0; r < S.nrhs; ++r, ++k) {
                SolverState& q = S.h->hst[r];
                if (trips == 0) S.eta_norm[r] = std::sqrt(q.acc);
                const double rn = q.rnorm, en = S.eta_norm[r];
                out[k].outer_residual = en > 0 ? rn / en : 0.0;
                // with clover blocks |eta - D xi| = |C_ee (b^ - A xi_e)| <= clover_bound |b^ - A xi_e|
                const double tol_eo = tol / clover_bound(S.h);
                bool act = (rn > tol_eo * en) && status[k] == WD_OK;
                if (act && !std::isfinite(rn)) {
                    status[k] = WD_ERR_NONFINITE;
                    act = false;
                }
                if (!std::isfinite(rn) && status[k] == WD_OK) status[k] = WD_ERR_NONFINITE;
                if (act && out[k].outer_iterations >= prm.max_outer) {
                    status[k] = WD_ERR_NOT_CONVERGED;
                    act = false;
                }
                S.active[r] = act;
                q.skip = act ? 0 : 1;
                if (hist_on) {
                    trip_rn = rn;
                    trip_res = en > 0 ? rn / en : 0.0;
                    if (!act) hist_put(1.0, (double)hcum, trip_res, 0.0);   // the final residual
                }
                if (act) {
                    any = true;
                    q.s = prm.s;
                    q.use_shat = prm.use_shat;
                    q.sigma = prm.sigma;
                    q.sigma_lambda = prm.sigma_lambda;
                    q.omega0 = prm.omega0;
                    q.recalc = prm.recalc_gamma;
                    q.rescale_x = prm.rescale_x;
                    q.scale_pass = scale_pass ? 1 : 0;
                    q.fused_scale = xr_mode == XR_FUSED ? 1 : 0;
                    q.ftz = prm.ftz ? 1 : 0;
                    q.hist = hist_on ? dhist : nullptr;
                    q.hist_cap = hist_on ? hist_iters : 0;
                    q.max_matvecs = prm.max_inner;
                    // FP64 BiCGStab: one inner solve to the outer tolerance; mixed: eps of Table 2
                    q.eps = cfg.fp64_inner ? std::max(0.5 * tol_eo * en / rn, 1e-15) : prm.inner_eps;
                    q.done = 0;
                }
            }
        }
        if ((rc = write_states(sys, s)) != WD_OK) return rc;
        if (!any) break;
        // y~ = low_prec((s / |r|) r) ; s^ = |single(y~)| ; inner start
        for (auto& S : sys) {
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                return Ops<T>::rescale_in(S.h->g.Vh, S.nrhs, S.vs, S.vs64, S.r64, S.r, S.rs, prm.ftz, S.h->st,
                                          red_ctx(S.h, ST_INIT), s);
            });
            WD_CUDA(S.h, e);
            nk += 1;
        }
        // inner BiCGStab of all systems: graph launches, the activity flag read one launch behind (once
        // launch kk - 1 has completed the mapped flag holds its value or a later launch's; within a trip the
        // flag only falls from 1 to 0, so a later value is the more recent answer)
        const int max_launch = prm.max_inner / (2 * ips) + 3;
        for (int kk = 0;; ++kk) {
            WD_CUDA(h0, cudaGraphLaunch(exec, s));
            nk += graph_kernels;
            WD_CUDA(h0, cudaEventRecord(h0->ev[kk & 1], s));
            if (kk >= 1) {
                WD_CUDA(h0, cudaEventSynchronize(h0->ev[(kk - 1) & 1]));
                if (!*(volatile int*)h0->hflag) break;
            }
            if (kk + 1 >= max_launch) break;
        }
        // x += (|r| / s^) double(t~) / lambda' ; r = b^ - A x in FP64
        for (auto& S : sys) {
            wd_handle* h = S.h;
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                return Ops<T>::correct(h->g.Vh, S.nrhs, S.vs, S.vs64, S.x64, S.xt, h->st, s);
            });
            WD_CUDA(h, e);
            WD_CUDA(h, hop64(S, 1, S.x64, S.tmp64, EPI_H, RED_NONE, 1.0, nullptr, 0.0, nullptr, 0.0, ST_NONE,
                             GUARD_OUTER, s, S.mi64o));
            WD_CUDA(h, hop64(S, 0, S.tmp64, S.r64, EPI_YZ, RED_NORM, h->kappa * h->kappa, S.bhat, 1.0, S.x64, -1.0,
                             ST_OUTER, GUARD_OUTER, s, S.mi64e));
            nk += 3;
        }
        if ((rc = read_states(sys, s)) != WD_OK) return rc;
        ++trips;
        k = 0;
        for (auto& S : sys) {
            for (int r = 0; r < S.nrhs; ++r, ++k) {
                if (!S.active[r]) continue;
                const SolverState& q = S.h->hst[r];
                out[k].outer_iterations += 1;
                out[k].inner_iterations += q.iter;
                out[k].inner_matvecs += q.matvecs;
                out[k].outer_matvecs += 1;
                if (out[k].outer_iterations == 1) out[k].first_inner_nonzeros = q.nonzeros;
                if (q.status == S_NONFINITE) status[k] = WD_ERR_NONFINITE;
                if (hist_on) {
                    hist_put(1.0, (double)hcum, trip_res, (double)q.nonzeros);
                    const int ni = q.iter < hist_iters ? q.iter : hist_iters;
                    hbuf.resize(2 * (size_t)(ni > 0 ? ni : 1));
                    if (ni > 0)
                        WD_CUDA(S.h, cudaMemcpy(hbuf.data(), dhist, sizeof(double) * 2 * ni, cudaMemcpyDeviceToHost));
                    const double en = S.eta_norm[r];
                    const double map = (q.shat > 0 && en > 0) ? trip_rn / (q.shat * en) : 0.0;
                    for (int i = 0; i < ni; ++i) hist_put(0.0, (double)hcum + hbuf[2 * i], hbuf[2 * i + 1] * map, 0.0);
                    hcum += q.matvecs;
                }
            }
        }
    }
    if (own_exec) cudaGraphExecDestroy(exec);

    // Eq. 5: xi_o = eta_o + kappa H_oe xi_e ; true residual |eta - D xi| in FP64
    for (auto& S : sys)
        for (int r = 0; r < S.nrhs; ++r) S.h->hst[r].skip = 0;
    if ((rc = write_states(sys, s)) != WD_OK) return rc;
    for (auto& S : sys) {
        wd_handle* h = S.h;
        const double kap = h->kappa;
        const size_t len = (size_t)2 * h->g.Vh * 24;
        if (S.mi64o) {   // xi_o = C_oo^-1 (eta_o + kappa H_oe xi_e); residual eta - (C xi - kappa H xi)
            const int nv = h->g.Vh;
            WD_CUDA(h, Ops<double>::apply_chiral(nv, S.nrhs, S.vs64, S.mi64o, S.eta_o, S.xo, s));
            WD_CUDA(h, hop64(S, 1, S.x64, S.xo, EPI_Y, RED_NONE, kap, S.xo, 1.0, nullptr, 0.0, ST_NONE, GUARD_NONE, s,
                             S.mi64o));
            WD_CUDA(h, Ops<double>::apply_mat(nv, S.nrhs, S.vs64, S.mf64e, S.x64, S.r64, s));
            WD_CUDA(h, hop64(S, 0, S.xo, S.r64, EPI_YZ, RED_NORM, kap, S.eta_e, 1.0, S.r64, -1.0, ST_ACC_SET,
                             GUARD_NONE, s));
            WD_CUDA(h, Ops<double>::apply_mat(nv, S.nrhs, S.vs64, S.mf64o, S.xo, S.tmp64, s));
            WD_CUDA(h, hop64(S, 1, S.x64, S.tmp64, EPI_YZ, RED_NORM, kap, S.eta_o, 1.0, S.tmp64, -1.0, ST_ACC,
                             GUARD_NONE, s));
            nk += 3;
        } else {   // t = H_oe xi_e; xi_o = eta_o + kappa t, |r_o|^2; r_e = eta_e - xi_e + kappa H_eo xi_o, |r_e|^2
            WD_CUDA(h, hop64(S, 1, S.x64, S.tmp64, EPI_H, RED_NONE, 1.0, nullptr, 0.0, nullptr, 0.0, ST_NONE,
                             GUARD_NONE, s));
            WD_CUDA(h, Ops<double>::odd_reconstruct(h->g.Vh, S.nrhs, S.vs64, kap, S.eta_o, S.tmp64, S.xo,
                                                    red_ctx(h, ST_ACC_SET), s));
            WD_CUDA(h, hop64(S, 0, S.xo, S.r64, EPI_YZ, RED_NORM, kap, S.eta_e, 1.0, S.x64, -1.0, ST_ACC,
                             GUARD_NONE, s));
        }
        for (int r = 0; r < S.nrhs; ++r) {
            WD_CUDA(h, Ops<double>::unpack(h->g, 0, S.x64 + r * S.vs64, S.xl + r * len, s));
            WD_CUDA(h, Ops<double>::unpack(h->g, 1, S.xo + r * S.vs64, S.xl + r * len, s));
        }
        if (!S.x_dev) WD_CUDA(h, cudaMemcpyAsync(S.x, S.xl, S.nrhs * len * sizeof(double), cudaMemcpyDeviceToHost, s));
        nk += 3 + 2 * S.nrhs;
    }
    WD_CUDA(h0, cudaEventRecord(h0->t1, s));
    if ((rc = read_states(sys, s)) != WD_OK) return rc;
    bool timed_out = false;   // a bounded device wait of a kernel gave up
    for (auto& S : sys) {
        if (!S.err) continue;
        int herr = 0;
        WD_CUDA(S.h, cudaMemcpy(&herr, S.err, sizeof(int), cudaMemcpyDeviceToHost));
        timed_out = timed_out || herr != 0;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, h0->t0, h0->t1);
    int worst = WD_OK;
    int k = 0;
    for (auto& S : sys) {
        for (int r = 0; r < S.nrhs; ++r, ++k) {
            const double en = S.eta_norm[r];
            wd_solve_stats& o = out[k];
            o.elapsed_ms = ms;
            o.kernel_launches = nk;
            o.history_len = hist_on ? hlen : 0;
            o.true_residual = en > 0 ? std::sqrt(S.h->hst[r].acc) / en : 0.0;
            if (o.outer_iterations == 0) o.first_inner_nonzeros = -1;
            int st = status[k];
            if (timed_out) st = WD_ERR_TIMEOUT;
            if (st == WD_OK && !(o.true_residual <= tol))
                st = std::isfinite(o.true_residual) ? WD_ERR_NOT_CONVERGED : WD_ERR_NONFINITE;
            o.status = st;
            if (st != WD_OK && worst == WD_OK) worst = st;
            if (stats) stats[k] = o;
        }
    }
    if (worst != WD_OK)
        fail(h0, worst, "solve: %s (first failing right-hand side of %d, %d refinement trips)",
             wd_status_string(worst), total_rhs, trips);
    return worst;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_solve_params_default(int scheme, wd_solve_params* p) {
    if (!p) return WD_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof *p);
    p->omega0 = 0.7;
    p->inner_eps = 1e-2;      // eps^2 = 1e-4 (Table 2)
    p->max_outer = 100;
    p->max_inner = 5000;
    p->recon = 12;
    p->iters_per_sync = 4;
    p->fused_rescale = 1;
    switch (scheme) {
    case WD_FP64_BICGSTAB:
        p->s = 1.0;
        p->max_inner = 100000;
        p->recon = 18;
        break;
    case WD_MIXED_FP32:
    case WD_MIXED_FP16_PLAIN:   // Alg. 2: unit-norm input, no s-hat, no inner rescaling
        p->s = 1.0;
        break;
    case WD_MIXED_FP16:
    case WD_MIXED_BF16:         // Alg. 3 + Alg. 4, Table 2 row s = 128, sigma = 64
    case WD_MIXED_FP16_LEARNED:
        p->s = 128.0;
        p->sigma = 64.0;
        p->sigma_lambda = 64.0;
        p->recalc_gamma = 1;
        p->use_shat = 1;
        break;
    default:
        return WD_ERR_INVALID_ARG;
    }
    return WD_OK;
}

extern "C" int wd_solve(wd_handle* h, const double* b, double* x, double tol, int scheme,
                        const wd_solve_params* params, wd_solve_stats* stats, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!b || !x) return fail(h, WD_ERR_INVALID_ARG, "wd_solve: null source or solution");
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "wd_solve: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    const int one = 1;
    return solve_systems(1, &h, &one, &b, &x, tol, scheme, params, stats, (cudaStream_t)stream);
}
