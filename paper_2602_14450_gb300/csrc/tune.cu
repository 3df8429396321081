// wd_tune: per-handle choice of the hopping-kernel variant and block size by
// timing every candidate on this lattice (CUDA events on the caller's stream).
#include <vector>

#include "handle.h"

using namespace wd;

namespace {

struct Cand {
    int variant, block;
};

std::vector<Cand> candidates(int prec, int recon) {
    std::vector<Cand> c = {{4, 128}, {4, 64}, {4, 256}, {1, 128}};
    if (prec != WD_FP64) c.push_back({2, 128});
    if (prec == WD_FP16 || prec == WD_BF16) {
        c.push_back({3, 128});
        c.push_back({6, 128});
        c.push_back({6, 256});
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
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = vec_bytes(h, prec) * (size_t)nrhs;
    uint4* in = (uint4*)workspace(h, "tune.in", vb);
    uint4* outv = (uint4*)workspace(h, "tune.out", vb);
    if (!in || !outv) return fail(h, WD_ERR_CUDA, "out of device memory");
    // a byte pattern of ordinary finite values in every storage format (0x3C3C = 1.06 in FP16)
    WD_CUDA(h, cudaMemsetAsync(in, 0x3C, vb, s));
    HopParams P{};
    P.g = h->g;
    P.nrhs = nrhs;
    P.vs = (long long)spinor_units(prec) * h->g.Vh;
    P.parity = 0;
    P.links = le;
    P.in = in;
    P.out = outv;
    P.a = 1.0;
    P.guard_kind = GUARD_NONE;
    cudaEvent_t e0, e1;
    WD_CUDA(h, cudaEventCreate(&e0));
    WD_CUDA(h, cudaEventCreate(&e1));
    const std::vector<Cand> cands = candidates(prec, recon);
    Cand best = cands[0];
    float best_ms = 1e30f, default_ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (const Cand& c : cands) {
        P.variant = c.variant;
        P.block = c.block;
        auto launch = [&]() {
            return by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                return Ops<T>::hop(recon, EPI_H, RED_NONE, P, s);
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
        if (c.variant == 4 && c.block == 128) default_ms = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(h, err, "wd_tune: timing a candidate");
    const int ri = recon == 12 ? 0 : 1;
    h->tune_variant[prec][ri] = best.variant;
    h->tune_block[prec][ri] = best.block;
    h->gen += 1;   // captured solver graphs hold the old kernels
    if (out) {
        out->variant = best.variant;
        out->block = best.block;
        out->us = 1e3 * best_ms;
        out->default_us = 1e3 * default_ms;
        out->candidates = (int)cands.size();
    }
    return WD_OK;
}
