// wd_solve: FP64 iterative refinement (Alg. 1 / Alg. 2) around the rescaled
// low-precision BiCGStab (Alg. 3 / Alg. 4) on the even-odd system of Eq. 4,
// followed by the odd-site reconstruction of Eq. 5.
//
// Device-resident design: every scalar of the recurrences lives in a
// SolverState in device memory and is updated by the last block of the
// reducing kernel that produces its inputs; one inner BiCGStab iteration is
// a fixed chain of 7-8 kernels captured once in a CUDA graph (several
// iterations per graph). Kernels return immediately once the state says the
// inner solve is done, so the host only polls a flag every few launches.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "handle.h"

namespace wd {

struct SchemeCfg {
    int prec;          // inner storage precision
    bool fp64_inner;   // WD_FP64_BICGSTAB: the "inner" solve is the whole solve
};

static bool scheme_cfg(int scheme, SchemeCfg* c) {
    switch (scheme) {
    case WD_FP64_BICGSTAB: c->prec = WD_FP64; c->fp64_inner = true; return true;
    case WD_MIXED_FP32: c->prec = WD_FP32; c->fp64_inner = false; return true;
    case WD_MIXED_FP16_PLAIN: c->prec = WD_FP16; c->fp64_inner = false; return true;
    case WD_MIXED_FP16: c->prec = WD_FP16; c->fp64_inner = false; return true;
    case WD_MIXED_BF16: c->prec = WD_BF16; c->fp64_inner = false; return true;
    default: return false;
    }
}

// Low-precision work vectors of the inner solve (even sites unless noted).
struct InnerVecs {
    uint4 *r, *rs, *p, *v, *t, *x, *tmp;   // tmp: odd sites
};

static int inner_vecs(wd_handle* h, int prec, InnerVecs* iv) {
    const size_t b = vec_bytes(h, prec);
    const std::string k = "in" + std::to_string(prec) + ".";
    uint4** slots[7] = {&iv->r, &iv->rs, &iv->p, &iv->v, &iv->t, &iv->x, &iv->tmp};
    const char* names[7] = {"r", "rs", "p", "v", "t", "x", "tmp"};
    for (int i = 0; i < 7; ++i) {
        *slots[i] = (uint4*)workspace(h, k + names[i], b);
        if (!*slots[i]) return fail(h, WD_ERR_CUDA, "out of device memory (%s)", names[i]);
    }
    return WD_OK;
}

// Enqueue one inner BiCGStab iteration (Alg. 3 / Alg. 4 loop body).
static cudaError_t enqueue_iteration(wd_handle* h, int prec, int recon, bool scale_pass, const InnerVecs& iv,
                                     const uint4* le, const uint4* lo, cudaStream_t s) {
    const int n = h->g.Vh;
    const double k2 = h->kappa * h->kappa;
    SolverState* st = h->st;
    return by_prec(prec, [&](auto tag) -> cudaError_t {
        typedef typename decltype(tag)::type T;
        cudaError_t e;
        HopParams P{};
        P.g = h->g;
        P.rc = red_ctx(h, ST_NONE);
        P.guard = st;
        // p := beta (p - omega' v) + r   (gamma of p and v folded in)
        if ((e = Ops<T>::pupdate(n, iv.p, iv.v, iv.r, st, s)) != cudaSuccess) return e;
        // v = A p = p - kappa^2 H_eo H_oe p ; alpha = rho / (r*, v)
        P.parity = 1; P.links = lo; P.in = iv.p; P.out = iv.tmp; P.a = 1.0;
        if ((e = Ops<T>::hop(recon, EPI_H, RED_NONE, P, s)) != cudaSuccess) return e;
        P.parity = 0; P.links = le; P.in = iv.tmp; P.out = iv.v; P.y = iv.p; P.a = -k2; P.b = 1.0;
        P.rstar = iv.rs; P.rc = red_ctx(h, ST_ALPHA);
        if ((e = Ops<T>::hop(recon, EPI_Y, RED_RSV, P, s)) != cudaSuccess) return e;
        // r := r - alpha v
        if ((e = Ops<T>::supdate(n, iv.r, iv.v, st, s)) != cudaSuccess) return e;
        // t = A r ; omega from (t, r), (t, t), (r, r)
        P.rc = red_ctx(h, ST_NONE);
        P.parity = 1; P.links = lo; P.in = iv.r; P.out = iv.tmp; P.y = nullptr; P.a = 1.0; P.b = 0.0; P.rstar = nullptr;
        if ((e = Ops<T>::hop(recon, EPI_H, RED_NONE, P, s)) != cudaSuccess) return e;
        P.parity = 0; P.links = le; P.in = iv.tmp; P.out = iv.t; P.y = iv.r; P.a = -k2; P.b = 1.0;
        P.rc = red_ctx(h, ST_OMEGA);
        if ((e = Ops<T>::hop(recon, EPI_Y, RED_TS, P, s)) != cudaSuccess) return e;
        // x += lambda'/gamma' (omega r + alpha p) ; r := r - omega t ; |r|, |x|
        if ((e = Ops<T>::xr(!scale_pass, n, iv.x, iv.r, iv.p, iv.t, iv.rs, st, red_ctx(h, ST_RNORM), s)) != cudaSuccess)
            return e;
        // r := (sigma / g) r ; gamma ; [x := lambda x] ; next rho, beta
        if (scale_pass)
            if ((e = Ops<T>::scale(n, iv.r, iv.x, iv.rs, st, red_ctx(h, ST_END), s)) != cudaSuccess) return e;
        return cudaSuccess;
    });
}

static int inner_graph(wd_handle* h, int prec, int recon, bool scale_pass, int iters, const InnerVecs& iv,
                       const uint4* le, const uint4* lo, cudaGraphExec_t* out) {
    GraphKey key{prec, recon, scale_pass ? 1 : 0, iters};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = it->second;
        return WD_OK;
    }
    cudaGraph_t graph = nullptr;
    WD_CUDA(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < iters && e == cudaSuccess; ++i) e = enqueue_iteration(h, prec, recon, scale_pass, iv, le, lo, h->cap);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(h, e, "capture of the inner iteration");
    }
    WD_CUDA(h, e2);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    WD_CUDA(h, e);
    h->graphs[key] = exec;
    *out = exec;
    return WD_OK;
}

// Read the device state into the pinned mirror (synchronizes s).
static int read_state(wd_handle* h, cudaStream_t s) {
    WD_CUDA(h, cudaMemcpyAsync(h->hst, h->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaStreamSynchronize(s));
    return WD_OK;
}

static int write_state(wd_handle* h, cudaStream_t s) {
    WD_CUDA(h, cudaMemcpyAsync(h->st, h->hst, sizeof(SolverState), cudaMemcpyHostToDevice, s));
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
    p->iters_per_sync = 8;
    switch (scheme) {
    case WD_FP64_BICGSTAB:
        p->s = 1.0;
        p->max_inner = 100000;
        p->recon = 18;
        break;
    case WD_MIXED_FP32:
    case WD_MIXED_FP16_PLAIN:   // Alg. 1: unit-norm input, no s-hat, no inner rescaling
        p->s = 1.0;
        break;
    case WD_MIXED_FP16:
    case WD_MIXED_BF16:         // Alg. 2 + Alg. 3, Table 2 row s = 128, sigma = 64
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
    SchemeCfg cfg;
    if (!b || !x || !(tol > 0) || !scheme_cfg(scheme, &cfg)) return fail(h, WD_ERR_INVALID_ARG, "wd_solve: bad argument");
    wd_solve_params prm;
    if (params) prm = *params; else wd_solve_params_default(scheme, &prm);
    if (!valid_recon(prm.recon) || prm.max_outer < 1 || prm.max_inner < 2 || !(prm.s > 0) || prm.sigma < 0 ||
        prm.iters_per_sync < 1 || (prm.rescale_x && !(prm.sigma_lambda > 0)))
        return fail(h, WD_ERR_INVALID_ARG, "wd_solve: bad parameters");
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    int rc = ensure_solver_state(h);
    if (rc != WD_OK) return rc;
    const int prec = cfg.prec;
    const int recon_lo = cfg.fp64_inner ? 18 : prm.recon;
    const uint4 *le64, *lo64, *le, *lo;
    if ((rc = ensure_links(h, WD_FP64, 18, &le64, &lo64)) != WD_OK) return rc;
    if ((rc = ensure_links(h, prec, recon_lo, &le, &lo)) != WD_OK) return rc;

    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->g.Vh;
    const size_t b64 = vec_bytes(h, WD_FP64);
    const size_t lexb = (size_t)2 * n * 24 * sizeof(double);
    uint4* eta_e = (uint4*)workspace(h, "f64.eta_e", b64);
    uint4* eta_o = (uint4*)workspace(h, "f64.eta_o", b64);
    uint4* bhat = (uint4*)workspace(h, "f64.bhat", b64);
    uint4* x64 = (uint4*)workspace(h, "f64.x", b64);
    uint4* r64 = (uint4*)workspace(h, "f64.r", b64);
    uint4* tmp64 = (uint4*)workspace(h, "f64.tmp", b64);
    uint4* xo = (uint4*)workspace(h, "f64.xo", b64);
    if (!eta_e || !eta_o || !bhat || !x64 || !r64 || !tmp64 || !xo) return fail(h, WD_ERR_CUDA, "out of device memory");
    InnerVecs iv;
    if (cfg.fp64_inner || prec != WD_FP64) {
        if ((rc = inner_vecs(h, prec, &iv)) != WD_OK) return rc;
    }

    const bool b_dev = is_device_ptr(b), x_dev = is_device_ptr(x);
    double* bl = const_cast<double*>(b);
    double* xl = x;
    if (!b_dev || !x_dev) {
        double* stage = (double*)workspace(h, "lex.stage", lexb);
        if (!stage) return fail(h, WD_ERR_CUDA, "out of device memory");
        if (!b_dev) bl = stage;
        if (!x_dev) xl = stage;   // b is consumed (packed) before x is written
    }

    WD_CUDA(h, cudaEventRecord(h->t0, s));
    if (!b_dev) WD_CUDA(h, cudaMemcpyAsync(bl, b, lexb, cudaMemcpyHostToDevice, s));
    const double kappa = h->kappa;
    HopParams P{};
    P.g = h->g;
    P.rc = red_ctx(h, ST_NONE);
    P.guard = nullptr;   // FP64 refinement kernels never exit early

    auto hop64 = [&](int parity, const uint4* in, uint4* out, int epi, int red, double a, const uint4* y, double bb,
                     const uint4* z, double c, int stage) {
        P.parity = parity;
        P.links = parity == 0 ? le64 : lo64;
        P.in = in;
        P.out = out;
        P.y = y;
        P.z = z;
        P.a = a;
        P.b = bb;
        P.c = c;
        P.rc = red_ctx(h, stage);
        return Ops<double>::hop(18, epi, red, P, s);
    };

    long long nk = 0;   // kernels launched by this call
    // Eq. 4 right-hand side: b^ = eta_e + kappa H_eo eta_o ; |eta|^2
    nk += 5;
    WD_CUDA(h, Ops<double>::pack(h->g, 0, bl, eta_e, s));
    WD_CUDA(h, Ops<double>::pack(h->g, 1, bl, eta_o, s));
    WD_CUDA(h, Ops<double>::norm2(n, eta_e, red_ctx(h, ST_ACC_SET), s));
    WD_CUDA(h, Ops<double>::norm2(n, eta_o, red_ctx(h, ST_ACC), s));
    WD_CUDA(h, hop64(0, eta_o, bhat, EPI_Y, RED_NONE, kappa, eta_e, 1.0, nullptr, 0.0, ST_NONE));
    // r = b^ - A x
    nk += prm.x_is_guess ? 3 : 1;
    if (prm.x_is_guess) {
        if (!x_dev) WD_CUDA(h, cudaMemcpyAsync(xl, x, lexb, cudaMemcpyHostToDevice, s));
        WD_CUDA(h, Ops<double>::pack(h->g, 0, xl, x64, s));
        WD_CUDA(h, hop64(1, x64, tmp64, EPI_H, RED_NONE, 1.0, nullptr, 0.0, nullptr, 0.0, ST_NONE));
        WD_CUDA(h, hop64(0, tmp64, r64, EPI_YZ, RED_NORM, kappa * kappa, bhat, 1.0, x64, -1.0, ST_OUTER));
    } else {
        WD_CUDA(h, cudaMemsetAsync(x64, 0, b64, s));
        WD_CUDA(h, cudaMemcpyAsync(r64, bhat, b64, cudaMemcpyDeviceToDevice, s));
        WD_CUDA(h, Ops<double>::norm2(n, r64, red_ctx(h, ST_OUTER), s));
    }
    if ((rc = read_state(h, s)) != WD_OK) return rc;
    const double eta_norm = std::sqrt(h->hst->acc);

    wd_solve_stats out{};
    out.status = WD_OK;
    out.first_inner_nonzeros = -1;
    int status = WD_OK;
    const bool scale_pass = prm.sigma > 0 || prm.rescale_x;
    const int ips = prm.iters_per_sync;
    cudaGraphExec_t exec = nullptr;
    if ((rc = inner_graph(h, prec, recon_lo, scale_pass, ips, iv, le, lo, &exec)) != WD_OK) return rc;

    int trips = 0;
    for (;;) {
        const double rn = h->hst->rnorm;
        out.outer_residual = eta_norm > 0 ? rn / eta_norm : 0.0;
        if (!(rn > tol * eta_norm)) {
            if (!std::isfinite(rn)) status = WD_ERR_NONFINITE;
            break;
        }
        if (trips >= prm.max_outer) {
            status = WD_ERR_NOT_CONVERGED;
            break;
        }
        // configure the inner solve (Alg. 3 / Alg. 4 parameters)
        SolverState* hs = h->hst;
        hs->s = prm.s;
        hs->use_shat = prm.use_shat;
        hs->sigma = prm.sigma;
        hs->sigma_lambda = prm.sigma_lambda;
        hs->omega0 = prm.omega0;
        hs->recalc = prm.recalc_gamma;
        hs->rescale_x = prm.rescale_x;
        hs->scale_pass = scale_pass ? 1 : 0;
        hs->max_matvecs = prm.max_inner;
        // FP64 BiCGStab: one inner solve to the outer tolerance; mixed: eps of Table 2
        hs->eps = cfg.fp64_inner ? std::max(0.5 * tol * eta_norm / rn, 1e-15) : prm.inner_eps;
        hs->done = 0;
        if ((rc = write_state(h, s)) != WD_OK) return rc;
        // y~ = low_prec((s / |r|) r) ; s^ = |single(y~)| ; inner start
        cudaError_t e = by_prec(prec, [&](auto tag) {
            typedef typename decltype(tag)::type T;
            return Ops<T>::rescale_in(n, r64, iv.r, iv.rs, prm.ftz, h->st, red_ctx(h, ST_INIT), s);
        });
        WD_CUDA(h, e);
        // inner BiCGStab: graph launches, done flag read one launch behind
        const int max_launch = prm.max_inner / (2 * ips) + 3;
        nk += 4;   // rescale, correction, two FP64 hops
        for (int k = 0;; ++k) {
            WD_CUDA(h, cudaGraphLaunch(exec, s));
            nk += (long long)ips * (scale_pass ? 8 : 7);
            WD_CUDA(h, cudaMemcpyAsync(&h->hflag[k & 1], &h->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            WD_CUDA(h, cudaEventRecord(h->ev[k & 1], s));
            if (k >= 1) {
                WD_CUDA(h, cudaEventSynchronize(h->ev[(k - 1) & 1]));
                if (h->hflag[(k - 1) & 1]) break;
            }
            if (k + 1 >= max_launch) break;
        }
        // x += (|r| / s^) double(t~) / lambda'
        e = by_prec(prec, [&](auto tag) {
            typedef typename decltype(tag)::type T;
            return Ops<T>::correct(n, x64, iv.x, h->st, s);
        });
        WD_CUDA(h, e);
        // r = b^ - A x in FP64
        WD_CUDA(h, hop64(1, x64, tmp64, EPI_H, RED_NONE, 1.0, nullptr, 0.0, nullptr, 0.0, ST_NONE));
        WD_CUDA(h, hop64(0, tmp64, r64, EPI_YZ, RED_NORM, kappa * kappa, bhat, 1.0, x64, -1.0, ST_OUTER));
        if ((rc = read_state(h, s)) != WD_OK) return rc;
        ++trips;
        out.inner_iterations += h->hst->iter;
        out.inner_matvecs += h->hst->matvecs;
        out.outer_matvecs += 1;
        if (trips == 1) out.first_inner_nonzeros = h->hst->nonzeros;
        if (h->hst->status == S_NONFINITE) {
            status = WD_ERR_NONFINITE;
            break;
        }
    }

    // Eq. 5: xi_o = eta_o + kappa H_oe xi_e ; true residual |eta - D xi| in FP64
    nk += 5;
    WD_CUDA(h, hop64(1, x64, xo, EPI_Y, RED_NONE, kappa, eta_o, 1.0, nullptr, 0.0, ST_NONE));
    WD_CUDA(h, hop64(0, xo, r64, EPI_YZ, RED_NORM, kappa, eta_e, 1.0, x64, -1.0, ST_ACC_SET));
    WD_CUDA(h, hop64(1, x64, tmp64, EPI_YZ, RED_NORM, kappa, eta_o, 1.0, xo, -1.0, ST_ACC));
    WD_CUDA(h, Ops<double>::unpack(h->g, 0, x64, xl, s));
    WD_CUDA(h, Ops<double>::unpack(h->g, 1, xo, xl, s));
    if (!x_dev) WD_CUDA(h, cudaMemcpyAsync(x, xl, lexb, cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaEventRecord(h->t1, s));
    if ((rc = read_state(h, s)) != WD_OK) return rc;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->t0, h->t1);
    out.elapsed_ms = ms;
    out.outer_iterations = trips;
    out.kernel_launches = nk;
    out.true_residual = eta_norm > 0 ? std::sqrt(h->hst->acc) / eta_norm : 0.0;
    if (status == WD_OK && !(out.true_residual <= tol)) status = std::isfinite(out.true_residual) ? WD_ERR_NOT_CONVERGED : WD_ERR_NONFINITE;
    out.status = status;
    if (stats) *stats = out;
    if (status != WD_OK) fail(h, status, "wd_solve: %s (true residual %g, %d trips)", wd_status_string(status),
                              out.true_residual, trips);
    return status;
}
