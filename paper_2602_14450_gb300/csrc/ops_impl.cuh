// Definitions of Ops<T>; included by exactly one translation unit per T.
#pragma once

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "blas_impl.cuh"
#include "hop2_impl.cuh"
#include "hop_impl.cuh"
#include "kernels.h"

namespace wd {

// Resident blocks per SM of a kernel at a block size (cached).
inline int blocks_per_sm(const void* kernel, int block) {
    static std::mutex m;
    static std::map<std::pair<const void*, int>, int> cache;
    std::lock_guard<std::mutex> lk(m);
    auto key = std::make_pair(kernel, block);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0) != cudaSuccess || n < 1) n = 1;
    cache[key] = n;
    return n;
}

// Grid of a reducing kernel: every block resident at once, no more blocks
// than needed to cover n items, and at most MAX_RED_BLOCKS partial sums.
inline int reduce_grid(const void* kernel, int n, int block) {
    long need = ((long)n + block - 1) / block;
    long g = (long)blocks_per_sm(kernel, block) * num_sms();
    if (g > need) g = need;
    if (g > MAX_RED_BLOCKS) g = MAX_RED_BLOCKS;
    return g < 1 ? 1 : (int)g;
}

inline int stream_grid(int n, int block) {
    long g = ((long)n + block - 1) / block;
    return g < 1 ? 1 : (int)g;
}

template <typename T, int R, int E, int D>
cudaError_t run_hop(const HopParams& P, cudaStream_t s) {
    const int block = hop_block();
    if constexpr (!std::is_same<T, double>::value) {
        if (hop_variant() == 2) {   // two sites per thread, packed FP32x2 arithmetic
            const int n = P.g.Vh / 2;
            const void* k2 = (const void*)hop2_kernel<T, R, E, D>;
            const int grid = (D == RED_NONE) ? stream_grid(n, block) : reduce_grid(k2, n, block);
            hop2_kernel<T, R, E, D><<<grid, block, 0, s>>>(P);
            return cudaGetLastError();
        }
    }
    const void* k = (const void*)hop_kernel<T, R, E, D>;
    const int grid = (D == RED_NONE) ? stream_grid(P.g.Vh, block) : reduce_grid(k, P.g.Vh, block);
    hop_kernel<T, R, E, D><<<grid, block, 0, s>>>(P);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::hop(int recon, int epi, int red, const HopParams& P, cudaStream_t s) {
#define WD_HOP_CASE(R, E, D) \
    if (recon == R && epi == E && red == D) return run_hop<T, R, E, D>(P, s);
    WD_HOP_CASE(12, EPI_H, RED_NONE)
    WD_HOP_CASE(12, EPI_Y, RED_NONE)
    WD_HOP_CASE(12, EPI_Y, RED_RSV)
    WD_HOP_CASE(12, EPI_Y, RED_TS)
    WD_HOP_CASE(12, EPI_YZ, RED_NORM)
    WD_HOP_CASE(18, EPI_H, RED_NONE)
    WD_HOP_CASE(18, EPI_Y, RED_NONE)
    WD_HOP_CASE(18, EPI_Y, RED_RSV)
    WD_HOP_CASE(18, EPI_Y, RED_TS)
    WD_HOP_CASE(18, EPI_YZ, RED_NORM)
#undef WD_HOP_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Ops<T>::pupdate(int n, uint4* p, const uint4* v, const uint4* r, const SolverState* st, cudaStream_t s) {
    k_pupdate<T><<<stream_grid(n, VEC_BLOCK), VEC_BLOCK, 0, s>>>(n, p, v, r, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::supdate(int n, uint4* r, const uint4* v, const SolverState* st, cudaStream_t s) {
    k_supdate<T><<<stream_grid(n, VEC_BLOCK), VEC_BLOCK, 0, s>>>(n, r, v, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::xr(bool with_rs, int n, uint4* x, uint4* r, const uint4* p, const uint4* t, const uint4* rstar,
                       SolverState* st, RedCtx rc, cudaStream_t s) {
    if (with_rs) {
        const int g = reduce_grid((const void*)k_xr<T, true>, n, VEC_BLOCK);
        k_xr<T, true><<<g, VEC_BLOCK, 0, s>>>(n, x, r, p, t, rstar, st, rc);
    } else {
        const int g = reduce_grid((const void*)k_xr<T, false>, n, VEC_BLOCK);
        k_xr<T, false><<<g, VEC_BLOCK, 0, s>>>(n, x, r, p, t, rstar, st, rc);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::scale(int n, uint4* r, uint4* x, const uint4* rstar, SolverState* st, RedCtx rc, cudaStream_t s) {
    const int g = reduce_grid((const void*)k_scale<T>, n, VEC_BLOCK);
    k_scale<T><<<g, VEC_BLOCK, 0, s>>>(n, r, x, rstar, st, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::rescale_in(int n, const uint4* r64, uint4* r, uint4* rstar, int ftz, SolverState* st, RedCtx rc,
                               cudaStream_t s) {
    const int g = reduce_grid((const void*)k_rescale_in<T>, n, VEC_BLOCK);
    k_rescale_in<T><<<g, VEC_BLOCK, 0, s>>>(n, r64, r, rstar, ftz, st, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::correct(int n, uint4* x64, const uint4* xt, const SolverState* st, cudaStream_t s) {
    k_correct<T><<<stream_grid(n, VEC_BLOCK), VEC_BLOCK, 0, s>>>(n, x64, xt, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::norm2(int n, const uint4* v, RedCtx rc, cudaStream_t s) {
    const int g = reduce_grid((const void*)k_norm2<T>, n, VEC_BLOCK);
    k_norm2<T><<<g, VEC_BLOCK, 0, s>>>(n, v, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::pack(const Geom& g, int parity, const double* lex, uint4* out, cudaStream_t s) {
    k_pack<T><<<stream_grid(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, lex, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::unpack(const Geom& g, int parity, const uint4* in, double* lex, cudaStream_t s) {
    k_unpack<T><<<stream_grid(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, in, lex);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::build_links(int recon, const Geom& g, int parity, const double* U, uint4* out, cudaStream_t s) {
    if (recon == 12)
        k_build_links<T, 12><<<stream_grid(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, U, out);
    else if (recon == 18)
        k_build_links<T, 18><<<stream_grid(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, U, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace wd
