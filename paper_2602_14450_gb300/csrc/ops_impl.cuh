// Definitions of Ops<T>; included by exactly one translation unit per T.
#pragma once

#include <cstdlib>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "blas_impl.cuh"
#include "hop2_impl.cuh"
#include "hop16_impl.cuh"
#include "hop16m_impl.cuh"
#include "hop3_impl.cuh"
#include "hop_impl.cuh"
#include "kernels.h"

namespace wd {

// Launch with programmatic stream serialization (programmatic dependent
// launch): the kernel may be scheduled while its predecessor in the stream
// finishes, and waits for it in pdl_begin(). Used only for kernels that call
// pdl_begin() before touching memory. Environment WD_PDL=0 turns it off.
inline bool pdl_on() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("WD_PDL");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), long grid, int block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_on() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

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

// Blocks per right-hand side of a reducing kernel: every block of the launch
// resident at once, no more blocks than needed to cover n items, and at most
// MAX_RED_BLOCKS partial sums per right-hand side.
inline int reduce_blocks(const void* kernel, int n, int block, int nrhs) {
    long need = ((long)n + block - 1) / block;
    long g = (long)blocks_per_sm(kernel, block) * num_sms() / nrhs;
    if (g > need) g = need;
    if (g > MAX_RED_BLOCKS) g = MAX_RED_BLOCKS;
    return g < 1 ? 1 : (int)g;
}

inline int stream_blocks(int n, int block) {
    long g = ((long)n + block - 1) / block;
    return g < 1 ? 1 : (int)g;
}

// Tiling of the staged hop kernel, or false when its shared memory would not
// allow two resident blocks per SM.
template <typename T, int R>
bool stage_geom(const Geom& g, StageGeom* sg, size_t* smem) {
    int TR = 0;
    for (int tr = 1; tr <= g.L[1]; ++tr)
        if (g.L[1] % tr == 0 && tr * g.Lxh <= 256 && (tr * g.Lxh) % 2 == 0) TR = tr;
    if (TR == 0) return false;
    sg->TR = TR;
    sg->TS = TR * g.Lxh;
    sg->ntiles = g.Vh / sg->TS;
    sg->nrows = 5 * TR + 2;
    sg->spin_units = Spinor<T>::UNITS;
    sg->link_units = LinkFmt<T, R>::UNITS;
    const size_t units = (size_t)sg->spin_units * sg->nrows * g.Lxh + (size_t)sg->link_units * sg->TS;
    *smem = units * 16;
    sg->bytes = (unsigned)*smem;
    return *smem <= 113 * 1024;
}

// The FP16-arithmetic hop over groups of K right-hand sides per thread.
template <int R, int E, int D, bool LSM>
cudaError_t run_hop16m(const HopParams& Q, int K, cudaStream_t s) {
    constexpr int blk = Hop16mShape<R>::THREADS;
    const void* k = (const void*)hop16m_kernel<R, E, D, LSM>;
    const size_t smem = hop16m_smem<R, D, LSM>(K);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (smem > 96 * 1024) return cudaErrorInvalidValue;
    const int groups = Q.nrhs / K;
    long nb = ((long)Q.g.Vh + blk - 1) / blk;
    if (D != RED_NONE) {   // one resident wave, at most MAX_RED_BLOCKS partial sums per right-hand side
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, blk, smem) != cudaSuccess || per < 1) per = 1;
        long wave = (long)per * num_sms() / groups;
        if (nb > wave) nb = wave;
        if (nb > MAX_RED_BLOCKS) nb = MAX_RED_BLOCKS;
    }
    if (nb < 1) nb = 1;
    return launch_k(hop16m_kernel<R, E, D, LSM>, nb * groups, blk, smem, s, Q);
}

template <typename T, int R, int E, int D>
cudaError_t run_hop(const HopParams& P, cudaStream_t s) {
    if constexpr (std::is_same<T, __half>::value) {
        if (P.arith16) {   // FP16 arithmetic (with or without a site-local block)
            constexpr int blk = Hop16Bounds<R, D, false, 2>::THREADS;
            HopParams Q = P;
            Q.acc_exp = acc_exponent(P.a);
            constexpr int form = D == RED_NONE ? 0 : 1;
            int K = P.rhs_group[form] < 12 ? P.rhs_group[form] : 12;
            while (K > 1 && P.nrhs % K) --K;                       // the largest divisor of nrhs up to the choice
            if (K > 1 && !P.mat) {                                 // several right-hand sides per thread
                Q.rhs_group[form] = K;
                const cudaError_t le_ = P.rhs_smem[form] ? run_hop16m<R, E, D, true>(Q, K, s)
                                                         : run_hop16m<R, E, D, false>(Q, K, s);
                if (le_ != cudaSuccess) return le_;
                return cudaGetLastError();
            }
            if (P.mat) {
                const void* km = (const void*)hop16_kernel<R, E, D, true, 1>;
                const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, blk) : reduce_blocks(km, P.g.Vh, blk, P.nrhs);
                { const cudaError_t le_ = launch_k(hop16_kernel<R, E, D, true, 1>, nb * P.nrhs, blk, 0, s, Q); if (le_ != cudaSuccess) return le_; }
            } else if (hop16_ahead() == 1) {
                const void* k = (const void*)hop16_kernel<R, E, D, false, 1>;
                const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, blk) : reduce_blocks(k, P.g.Vh, blk, P.nrhs);
                { const cudaError_t le_ = launch_k(hop16_kernel<R, E, D, false, 1>, nb * P.nrhs, blk, 0, s, Q); if (le_ != cudaSuccess) return le_; }
            } else {
                const void* k = (const void*)hop16_kernel<R, E, D, false, 2>;
                const int spt = P.spt > 1 ? P.spt : 1;             // sites per thread of the plain hop
                const int nb = (D == RED_NONE) ? stream_blocks((P.g.Vh + spt - 1) / spt, blk)
                                               : reduce_blocks(k, P.g.Vh, blk, P.nrhs);
                { const cudaError_t le_ = launch_k(hop16_kernel<R, E, D, false, 2>, nb * P.nrhs, blk, 0, s, Q); if (le_ != cudaSuccess) return le_; }
            }
            return cudaGetLastError();
        }
    }
    if (P.mat) {   // with a site-local block (clover): the one-site-per-thread look-ahead kernel
        const int blk = 128;
        const void* km = (const void*)hop_kernel<T, R, E, D, true, false, true>;
        const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, blk) : reduce_blocks(km, P.g.Vh, blk, P.nrhs);
        { const cudaError_t le_ = launch_k(hop_kernel<T, R, E, D, true, false, true>, nb * P.nrhs, blk, 0, s, P); if (le_ != cudaSuccess) return le_; }
        return cudaGetLastError();
    }
    constexpr int form = D == RED_NONE ? 0 : 1;
    const int block = P.block[form] > 0 ? P.block[form] : hop_block();
    const int variant = P.variant[form] > 0 ? P.variant[form] : hop_variant();
    const int nr = P.nrhs;
    if constexpr (sizeof(T) == 2) {
        StageGeom sg;
        size_t smem = 0;
        if (variant == 3 && stage_geom<T, R>(P.g, &sg, &smem)) {   // shared-memory staged tiles
            static bool attr = false;
            const void* k3 = (const void*)hop3_kernel<T, R, E, D>;
            if (!attr) {
                cudaError_t e = cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, 113 * 1024);
                if (e != cudaSuccess) return e;
                attr = true;
            }
            int per = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k3, block, smem) != cudaSuccess || per < 1) per = 1;
            long nb = (long)per * num_sms() / nr;
            if (nb > sg.ntiles) nb = sg.ntiles;
            if (nb > MAX_RED_BLOCKS) nb = MAX_RED_BLOCKS;
            if (nb < 1) nb = 1;
            { const cudaError_t le_ = launch_k(hop3_kernel<T, R, E, D>, (int)nb * nr, block, smem, s, P, sg, P.err); if (le_ != cudaSuccess) return le_; }
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(T) == 2 && R == 12) {
        if (variant == 5) {   // per-thread shared-memory ring of asynchronous copies
            typedef RingFmt<T, R> RF;
            const void* k5 = (const void*)hop_ring_kernel<T, R, E, D>;
            int per = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k5, RF::BLOCK, RF::SMEM) != cudaSuccess || per < 1)
                per = 1;
            long nb = (long)per * num_sms() / nr;
            const long need = ((long)P.g.Vh + RF::BLOCK - 1) / RF::BLOCK;
            if (nb > need) nb = need;
            if (D != RED_NONE && nb > MAX_RED_BLOCKS) nb = MAX_RED_BLOCKS;
            if (nb < 1) nb = 1;
            { const cudaError_t le_ = launch_k(hop_ring_kernel<T, R, E, D>, (int)nb * nr, RF::BLOCK, RF::SMEM, s, P); if (le_ != cudaSuccess) return le_; }
            return cudaGetLastError();
        }
    }
    if constexpr (!std::is_same<T, double>::value) {
        if (variant == 2) {   // two sites per thread, packed FP32x2 arithmetic
            const int n = P.g.Vh / 2;
            const void* k2 = (const void*)hop2_kernel<T, R, E, D>;
            const int nb = (D == RED_NONE) ? stream_blocks(n, block) : reduce_blocks(k2, n, block, nr);
            { const cudaError_t le_ = launch_k(hop2_kernel<T, R, E, D>, nb * nr, block, 0, s, P); if (le_ != cudaSuccess) return le_; }
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(T) == 2) {
        if (variant == 6) {   // as 4, with the SU(3) products on FP32x2 column pairs
            const void* k = (const void*)hop_kernel<T, R, E, D, true, true>;
            const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, block) : reduce_blocks(k, P.g.Vh, block, nr);
            { const cudaError_t le_ = launch_k(hop_kernel<T, R, E, D, true, true>, nb * nr, block, 0, s, P); if (le_ != cudaSuccess) return le_; }
            return cudaGetLastError();
        }
    }
    if (variant == 4) {   // one site per thread, loads one direction ahead
        const void* k = (const void*)hop_kernel<T, R, E, D, true>;
        const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, block) : reduce_blocks(k, P.g.Vh, block, nr);
        { const cudaError_t le_ = launch_k(hop_kernel<T, R, E, D, true>, nb * nr, block, 0, s, P); if (le_ != cudaSuccess) return le_; }
        return cudaGetLastError();
    }
    const void* k = (const void*)hop_kernel<T, R, E, D, false>;
    const int nb = (D == RED_NONE) ? stream_blocks(P.g.Vh, block) : reduce_blocks(k, P.g.Vh, block, nr);
    { const cudaError_t le_ = launch_k(hop_kernel<T, R, E, D, false>, nb * nr, block, 0, s, P); if (le_ != cudaSuccess) return le_; }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::hop(int recon, int epi, int red, const HopParams& P, cudaStream_t s) {
    if (P.nrhs < 1) return cudaErrorInvalidValue;
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
cudaError_t Ops<T>::apply_mat(int n, int nrhs, long long vs, const uint4* mat, const uint4* in, uint4* out,
                              cudaStream_t s) {
    k_apply_mat<T><<<stream_blocks(n, VEC_BLOCK) * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, mat, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::apply_chiral(int n, int nrhs, long long vs, const uint4* mat, const uint4* in, uint4* out,
                                 cudaStream_t s) {
    k_apply_chiral<T><<<stream_blocks(n, VEC_BLOCK) * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, mat, in, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::chiral_from64(int n, const uint4* src64, uint4* dst, cudaStream_t s) {
    k_chiral_from64<T><<<stream_blocks(n, 128), 128, 0, s>>>(n, src64, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::mat_from64(int n, const uint4* src64, uint4* dst, cudaStream_t s) {
    k_mat_from64<T><<<stream_blocks(n, VEC_BLOCK), VEC_BLOCK, 0, s>>>(n, src64, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::pupdate(int n, int nrhs, long long vs, uint4* p, const uint4* v, const uint4* r,
                            const SolverState* st, cudaStream_t s) {
    { const cudaError_t le_ = launch_k(k_pupdate<T>, stream_blocks((n + Stream<T>::SITES - 1) / Stream<T>::SITES, VEC_BLOCK) * nrhs, VEC_BLOCK, 0, s, n, nrhs, vs, p, v, r, st); if (le_ != cudaSuccess) return le_; }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::supdate(int n, int nrhs, long long vs, uint4* r, const uint4* v, const SolverState* st,
                            cudaStream_t s) {
    { const cudaError_t le_ = launch_k(k_supdate<T>, stream_blocks((n + Stream<T>::SITES - 1) / Stream<T>::SITES, VEC_BLOCK) * nrhs, VEC_BLOCK, 0, s, n, nrhs, vs, r, v, st); if (le_ != cudaSuccess) return le_; }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::xr(int mode, int n, int nrhs, long long vs, uint4* x, uint4* r, const uint4* p,
                       const uint4* t, const uint4* rstar, const uint4* xr_src, const uint4* xp_src,
                       SolverState* st, RedCtx rc, cudaStream_t s) {
#define WD_XR_CASE(M)                                                                                        \
    if (mode == M) {                                                                                         \
        const int nb = reduce_blocks((const void*)k_xr<T, M>, n, VEC_BLOCK, nrhs);                            \
        { const cudaError_t le_ = launch_k(k_xr<T, M>, nb * nrhs, VEC_BLOCK, 0, s, n, nrhs, vs, x, r, p, t, rstar, xr_src, xp_src, st, rc); if (le_ != cudaSuccess) return le_; }   \
        return cudaGetLastError();                                                                           \
    }
    WD_XR_CASE(XR_PLAIN)
    WD_XR_CASE(XR_NORMS)
    WD_XR_CASE(XR_FUSED)
#undef WD_XR_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Ops<T>::scale(int n, int nrhs, long long vs, uint4* r, uint4* x, const uint4* rstar, SolverState* st,
                          RedCtx rc, cudaStream_t s) {
    const int nb = reduce_blocks((const void*)k_scale<T>, n, VEC_BLOCK, nrhs);
    { const cudaError_t le_ = launch_k(k_scale<T>, nb * nrhs, VEC_BLOCK, 0, s, n, nrhs, vs, r, x, rstar, st, rc); if (le_ != cudaSuccess) return le_; }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::rescale_in(int n, int nrhs, long long vs, long long vs64, const uint4* r64, uint4* r,
                               uint4* rstar, int ftz, SolverState* st, RedCtx rc, cudaStream_t s) {
    const int nb = reduce_blocks((const void*)k_rescale_in<T>, n, VEC_BLOCK, nrhs);
    k_rescale_in<T><<<nb * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, vs64, r64, r, rstar, ftz, st, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::correct(int n, int nrhs, long long vs, long long vs64, uint4* x64, const uint4* xt,
                            const SolverState* st, cudaStream_t s) {
    k_correct<T><<<stream_blocks(n, VEC_BLOCK) * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, vs64, x64, xt, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::norm2(int n, int nrhs, long long vs, const uint4* v, RedCtx rc, int guard_kind,
                          cudaStream_t s) {
    const int nb = reduce_blocks((const void*)k_norm2<T>, n, VEC_BLOCK, nrhs);
    k_norm2<T><<<nb * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, v, rc, guard_kind);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::odd_reconstruct(int n, int nrhs, long long vs, double kappa, const uint4* eta, const uint4* t,
                                    uint4* xo, RedCtx rc, cudaStream_t s) {
    const int nb = reduce_blocks((const void*)k_odd_reconstruct<T>, n, VEC_BLOCK, nrhs);
    k_odd_reconstruct<T><<<nb * nrhs, VEC_BLOCK, 0, s>>>(n, nrhs, vs, kappa, eta, t, xo, rc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::pack(const Geom& g, int parity, const double* lex, uint4* out, cudaStream_t s) {
    k_pack<T><<<stream_blocks(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, lex, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::unpack(const Geom& g, int parity, const uint4* in, double* lex, cudaStream_t s) {
    k_unpack<T><<<stream_blocks(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, in, lex);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::build_links(int recon, const Geom& g, int parity, const double* U, uint4* out, cudaStream_t s) {
    if (recon == 12)
        k_build_links<T, 12><<<stream_blocks(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, U, out);
    else if (recon == 18)
        k_build_links<T, 18><<<stream_blocks(g.Vh, VEC_BLOCK), VEC_BLOCK, 0, s>>>(g, parity, U, out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace wd
