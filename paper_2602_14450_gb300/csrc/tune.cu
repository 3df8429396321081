// wd_tune: per-handle choice of the hopping-kernel variant and block size by
// timing every candidate on this lattice (CUDA events on the caller's stream),
// separately for the plain hop and for the hop with fused epilogue and dot
// products that ends every even-odd operator of the inner solve.
#include <vector>

#include "handle.h"

using namespace wd;

namespace {

struct Cand {
    int variant, block;
};

std::vector<Cand> candidates(int prec, int recon) {
    std::vector<Cand> c = {{4, 128}, {4, 64}, {1, 128}};
    if (prec != WD_FP16) c.push_back({4, 256});   // the plain FP16 look-ahead kernel takes at most 128 threads
    if (prec != WD_FP64) c.push_back({2, 128});
    if (prec == WD_FP16 || prec == WD_BF16) {
        c.push_back({3, 128});
        c.push_back({6, 128});
        c.push_back({6, 64});
        if (prec == WD_BF16) c.push_back({6, 256});
        if (recon == 12) c.push_back({5, 128});
    }
    return c;
}

}  // namespace

extern "C" int wd_tune(wd_handle* h, int prec, int recon, int nrhs, void* stream, wd_tune_result* out) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || !valid_recon(recon) || nrhs < 1 || nrhs > 1024)
        return fail(h, WD_ERR_INVALID_ARG, "wd_tune: bad argument");
    const uint4 *le, *lo;
    int rc = ensure_links(h, prec, recon, &le, &lo);
    if (rc != WD_OK) return rc;
    if ((rc = ensure_solver_state(h, nrhs)) != WD_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vec_bytes(h, prec) * (size_t)nrhs;
    uint4* in = (uint4*)workspace(h, "tune.in", vb);
    uint4* y = (uint4*)workspace(h, "tune.y", vb);
    uint4* outv = (uint4*)workspace(h, "tune.out", vb);
    if (!in || !y || !outv) return fail(h, WD_ERR_CUDA, "out of device memory");
    // a byte pattern of ordinary finite values in every storage format (0x3C3C = 1.06 in FP16)
    WD_CUDA(h, cudaMemsetAsync(in, 0x3C, vb, s));
    WD_CUDA(h, cudaMemsetAsync(y, 0x3C, vb, s));
    HopParams P{};
    P.g = h->g;
    P.nrhs = nrhs;
    P.vs = (long long)spinor_units(prec) * h->g.Vh;
    P.parity = 0;
    P.links = le;
    P.in = in;
    P.out = outv;
    P.y = y;
    P.a = 1.0;
    P.b = 1.0;
    P.guard_kind = GUARD_NONE;
    P.rc = red_ctx(h, ST_NONE);   // the last block of a reduction finds no scalar stage to run
    cudaEvent_t e0, e1;
    WD_CUDA(h, cudaEventCreate(&e0));
    WD_CUDA(h, cudaEventCreate(&e1));
    const std::vector<Cand> cands = candidates(prec, recon);
    Cand best[2] = {cands[0], cands[0]};
    float best_ms[2] = {1e30f, 1e30f}, default_ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (int form = 0; form < 2 && err == cudaSuccess; ++form) {
        for (const Cand& c : cands) {
            P.variant[form] = c.variant;
            P.block[form] = c.block;
            auto launch = [&]() {
                return by_prec(prec, [&](auto tag) {
                    typedef typename decltype(tag)::type T;
                    return form == 0 ? Ops<T>::hop(recon, EPI_H, RED_NONE, P, s)
                                     : Ops<T>::hop(recon, EPI_Y, RED_TS, P, s);
                });
            };
            for (int i = 0; i < 2 && err == cudaSuccess; ++i) err = launch();
            if (err == cudaSuccess) err = cudaEventRecord(e0, s);
            for (int i = 0; i < 8 && err == cudaSuccess; ++i) err = launch();
            if (err == cudaSuccess) err = cudaEventRecord(e1, s);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err != cudaSuccess) break;
            ms /= 8.f;
            if (form == 0 && c.variant == 4 && c.block == 128) default_ms = ms;
            if (ms < best_ms[form]) {
                best_ms[form] = ms;
                best[form] = c;
            }
        }
    }
    // FP16 arithmetic (wd_set_arith(16)): right-hand sides per thread of the FP16-arithmetic hop, K dividing
    // nrhs (K = 1: one per thread), the site's links in registers or in shared memory
    const int ri = recon == 12 ? 0 : 1;
    int best_k[2] = {1, 1}, best_lsm[2] = {0, 0}, best_spt = 1;
    float best16[2] = {1e30f, 1e30f};
    int cands16 = 0;
    if (prec == WD_FP16 && h->arith16 && err == cudaSuccess) {
        P.arith16 = 1;
        P.variant[0] = P.variant[1] = 0;
        P.block[0] = P.block[1] = 0;
        for (int form = 0; form < 2 && err == cudaSuccess; ++form) {
            for (int k = 1; k <= 12 && err == cudaSuccess; ++k) {
                if (nrhs % k) continue;
                // K = 1: also 2 and 4 sites per thread for the plain hop (grid-stride)
                const int nshape = k > 1 ? 2 : (form == 0 ? 3 : 1);
                for (int shape = 0; shape < nshape && err == cudaSuccess; ++shape) {
                    const int lsm = k > 1 ? shape : 0;
                    const int spt = k > 1 ? 1 : (1 << shape);
                    P.rhs_group[form] = k;
                    P.rhs_smem[form] = lsm;
                    P.spt = spt;
                    auto launch = [&]() {
                        return form == 0 ? Ops<__half>::hop(recon, EPI_H, RED_NONE, P, s)
                                         : Ops<__half>::hop(recon, EPI_Y, RED_TS, P, s);
                    };
                    for (int i = 0; i < 2 && err == cudaSuccess; ++i) err = launch();
                    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
                    for (int i = 0; i < 8 && err == cudaSuccess; ++i) err = launch();
                    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
                    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                    if (err != cudaSuccess) break;
                    ms /= 8.f;
                    if (form == 0) ++cands16;
                    if (ms < best16[form]) {
                        best16[form] = ms;
                        best_k[form] = k;
                        best_lsm[form] = lsm;
                        if (form == 0) best_spt = spt;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(h, err, "wd_tune: timing a candidate");
    if (prec == WD_FP16 && h->arith16)
        for (int form = 0; form < 2; ++form) {
            h->tune_rhs[ri][form] = best_k[form];
            h->tune_rhs_smem[ri][form] = best_lsm[form];
            h->tune_spt[ri] = best_spt;
        }
    for (int form = 0; form < 2; ++form) {
        h->tune_variant[prec][ri][form] = best[form].variant;
        h->tune_block[prec][ri][form] = best[form].block;
    }
    h->gen += 1;   // captured solver graphs hold the old kernels
    if (out) {
        out->variant = best[0].variant;
        out->block = best[0].block;
        out->us = 1e3 * best_ms[0];
        out->default_us = 1e3 * default_ms;
        out->candidates = (int)cands.size();
        out->variant_reducing = best[1].variant;
        out->block_reducing = best[1].block;
        out->us_reducing = 1e3 * best_ms[1];
        const bool a16 = prec == WD_FP16 && h->arith16;
        out->rhs_per_thread = a16 ? best_k[0] : 1;
        out->rhs_links_smem = a16 ? best_lsm[0] : 0;
        out->us16 = a16 ? 1e3 * best16[0] : 0.0;
        out->rhs_per_thread_reducing = a16 ? best_k[1] : 1;
        out->rhs_links_smem_reducing = a16 ? best_lsm[1] : 0;
        out->us16_reducing = a16 ? 1e3 * best16[1] : 0.0;
        out->candidates16 = cands16;
        out->sites_per_thread = a16 ? best_spt : 1;
    }
    return WD_OK;
}
