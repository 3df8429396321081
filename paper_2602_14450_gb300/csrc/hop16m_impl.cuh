// Hopping term of Eq. 1 in FP16 arithmetic for a batch of right-hand sides
// that share one gauge field: each thread takes one output site and K
// right-hand sides, loads the site's 8 links once and applies them to the K
// neighbour spinors in turn (the arithmetic of hop16_kernel, one right-hand
// side after the other). The links then cost 192 B (12-real) per site for K
// right-hand sides instead of per right-hand side: at K = 12 a right-hand side
// moves 48 + 48 + 192 / 12 = 112 B per site against 288.
//
// The site's link units live in registers (LSM = false), or the site's eight
// 3x3 links, the third row of a 12-real link rebuilt once per site instead of
// once per right-hand side, in the thread's own slots of shared memory
// (LSM = true: fewer registers and fewer instructions per right-hand side).
// The neighbour spinors of the next two directions are in flight while one is
// used, across the boundary between right-hand sides too. A launch serves
// nrhs / K groups of K right-hand sides (block b: group b % groups); the dot
// products of a reducing form are summed per right-hand side in shared memory
// and reduced over the grid one right-hand side after the other.
#pragma once

#include "hop16_impl.cuh"

namespace wd {

template <int R> struct Hop16mShape {
    static constexpr int THREADS = 128;
    static constexpr int UNITS = LinkFmt<__half, R>::UNITS;          // link units of a site
    static constexpr int GU = LinkFmt<__half, R>::GROUP_UNITS;
    static constexpr int G = LinkFmt<__half, R>::G;
    static constexpr int SM_UNITS = 8 * 3;                           // shared memory: 8 links x (9 words + 3 pad)
};

// Dynamic shared memory of a launch (bytes).
template <int R, int RED, bool LSM>
constexpr size_t hop16m_smem(int K) {
    return (LSM ? (size_t)Hop16mShape<R>::SM_UNITS * 16 * Hop16mShape<R>::THREADS : 0) +
           (RED != RED_NONE ? (size_t)K * RedSums<RED>::N * 4 * Hop16mShape<R>::THREADS : 0);
}

template <int R, int EPI, int RED, bool LSM>
__global__ void __launch_bounds__(128) hop16m_kernel(const HopParams P) {
    pdl_begin();
    typedef Hop16mShape<R> SH;
    constexpr int NS = RedSums<RED>::N;
    constexpr int SU = Spinor<__half>::UNITS;
    extern __shared__ __align__(16) unsigned char smem16m[];
    uint4* s_lk = reinterpret_cast<uint4*>(smem16m);                                   // [SM_UNITS][THREADS]
    float* s_part = reinterpret_cast<float*>(smem16m + (LSM ? (size_t)SH::SM_UNITS * 16 * SH::THREADS : 0));
    const int K = P.rhs_group[RED == RED_NONE ? 0 : 1];
    const int groups = P.nrhs / K;
    const int grp = blockIdx.x % groups, b = blockIdx.x / groups, nb = gridDim.x / groups;
    const int r0 = grp * K;
    const int tid = threadIdx.x;
    unsigned active = 0;    // right-hand sides of the group still iterating (uniform over the grid)
    for (int j = 0; j < K; ++j)
        if (!guarded(P.guard ? P.guard + r0 + j : nullptr, P.guard_kind)) active |= 1u << j;
    if (!active) return;
    const Geom& g = P.g;
    const int Vh = g.Vh;
    const int ke = P.acc_exp;
    const unsigned c_one = h2_pow2(ke), c_two = h2_pow2(ke + 1);
    const float unscale = __int_as_float((127 - ke) << 23);
    if constexpr (RED != RED_NONE)
        for (int i = 0; i < K * NS; ++i) s_part[i * SH::THREADS + tid] = 0.f;

    // first and next active right-hand side after j (K when none)
    const int jfirst = __ffs(active) - 1;
    auto next_active = [&](int j) {
        const unsigned rest = j + 1 < 32 ? (active >> (j + 1)) << (j + 1) : 0u;
        return rest ? __ffs(rest) - 1 : K;
    };

    for (int h = b * blockDim.x + tid; h < Vh; h += nb * blockDim.x) {
        int nbr[8];
        const unsigned wm = site_neighbours(g, P.parity, h, nbr);
        uint4 lk[LSM ? 1 : SH::UNITS];
        if constexpr (LSM) {   // the 8 links as 3x3 half2 matrices, built once for the K right-hand sides
#pragma unroll
            for (int gi = 0; gi < 8 / SH::G; ++gi) {
                uint4 lu[SH::GU];
#pragma unroll
                for (int k = 0; k < SH::GU; ++k) lu[k] = __ldcs(P.links + (size_t)(gi * SH::GU + k) * Vh + h);
#pragma unroll
                for (int jj = 0; jj < SH::G; ++jj) {
                    __half2 m[9];
                    link_load16<R, SH::GU>(lu, jj, m);
                    const int d = gi * SH::G + jj;
                    s_lk[(3 * d + 0) * SH::THREADS + tid] = make_uint4(as_w(m[0]), as_w(m[1]), as_w(m[2]), as_w(m[3]));
                    s_lk[(3 * d + 1) * SH::THREADS + tid] = make_uint4(as_w(m[4]), as_w(m[5]), as_w(m[6]), as_w(m[7]));
                    s_lk[(3 * d + 2) * SH::THREADS + tid] = make_uint4(as_w(m[8]), 0u, 0u, 0u);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < SH::UNITS; ++k) lk[k] = __ldcs(P.links + (size_t)k * Vh + h);
        }
        // neighbour slots: (right-hand side j, direction d) uses slot d & 3 (8 j + d = d mod 4)
        uint4 nbu[4][SU];
        {
            const uint4* v0 = P.in + (long long)(r0 + jfirst) * P.vs;
#pragma unroll
            for (int d = 0; d < 2; ++d)
#pragma unroll
                for (int u = 0; u < SU; ++u) nbu[d][u] = __ldg(v0 + (size_t)u * Vh + nbr[d]);
        }
#pragma unroll 1
        for (int j = jfirst; j < K; j = next_active(j)) {
            const int jn = next_active(j);
            const long long ro = (long long)(r0 + j) * P.vs;
            const uint4* __restrict__ vin = P.in + ro;
            const uint4* vnext = jn < K ? P.in + (long long)(r0 + jn) * P.vs : nullptr;
            __half2 acc[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i] = as_h2(0u);
#pragma unroll
            for (int gi = 0; gi < 8 / SH::G; ++gi) {
                uint4 lu[SH::GU];
                if constexpr (!LSM) {
#pragma unroll
                    for (int k = 0; k < SH::GU; ++k) lu[k] = lk[gi * SH::GU + k];
                }
#pragma unroll
                for (int jj = 0; jj < SH::G; ++jj) {
                    const int d = gi * SH::G + jj;
                    const int mu = d >> 1;
                    const bool fwd = (d & 1) == 0;
                    uint4 cur[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) cur[u] = nbu[d & 3][u];
                    if (d + 2 < 8) {
#pragma unroll
                        for (int u = 0; u < SU; ++u) nbu[(d + 2) & 3][u] = __ldg(vin + (size_t)u * Vh + nbr[d + 2]);
                    } else if (vnext) {   // the next right-hand side's first two directions
#pragma unroll
                        for (int u = 0; u < SU; ++u) nbu[(d + 2) & 3][u] = __ldg(vnext + (size_t)u * Vh + nbr[d - 6]);
                    }
                    __half2 hs[6], chi[6];
                    project16(mu, fwd, cur, hs);
                    if constexpr (LSM) {
                        const uint4 w0 = s_lk[(3 * d + 0) * SH::THREADS + tid];
                        const uint4 w1 = s_lk[(3 * d + 1) * SH::THREADS + tid];
                        const uint4 w2 = s_lk[(3 * d + 2) * SH::THREADS + tid];
                        const __half2 m[9] = {as_h2(w0.x), as_h2(w0.y), as_h2(w0.z), as_h2(w0.w), as_h2(w1.x),
                                              as_h2(w1.y), as_h2(w1.z), as_h2(w1.w), as_h2(w2.x)};
                        mul16(m, hs, chi);
                    } else {
                        link_mul16<R, SH::GU>(lu, jj, hs, chi);
                    }
                    const unsigned fb =
                        (mu == 3 ? c_two : c_one) ^ ((((wm >> d) & 1u) && g.bc[mu] < 0) ? 0x80008000u : 0u);
                    reconstruct16(mu, fwd, fb, chi, acc);
                }
            }
            const bool ftz = P.guard != nullptr && P.guard[r0 + j].ftz;
            uint4* vout = P.out + ro;
            if (EPI == EPI_H && RED == RED_NONE && P.a == 1.0) {   // the plain hop: undo 2^k in FP16 and store
                const __half2 up = as_h2(h2_pow2(-ke));
#pragma unroll
                for (int i = 0; i < 12; ++i) acc[i] = __hmul2(acc[i], up);
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    uint4 w = make_uint4(as_w(acc[4 * u]), as_w(acc[4 * u + 1]), as_w(acc[4 * u + 2]),
                                         as_w(acc[4 * u + 3]));
                    if (ftz) w = Unit<__half>::flush(w);
                    vout[(size_t)u * Vh + h] = w;
                }
            } else {
                float a32[24];
#pragma unroll
                for (int i = 0; i < 12; ++i) {
                    a32[2 * i] = __low2float(acc[i]) * unscale;
                    a32[2 * i + 1] = __high2float(acc[i]) * unscale;
                }
                float part[NS];
#pragma unroll
                for (int k = 0; k < NS; ++k) part[k] = 0.f;
                hop_epilogue<__half, EPI, RED, false>(P, vout, P.y ? P.y + ro : nullptr, P.z ? P.z + ro : nullptr,
                                                      P.rstar ? P.rstar + ro : nullptr, h, a32, part, ftz);
                if constexpr (RED != RED_NONE) {
#pragma unroll
                    for (int k = 0; k < NS; ++k) s_part[(j * NS + k) * SH::THREADS + tid] += part[k];
                }
            }
        }
    }

    if constexpr (RED != RED_NONE) {
        for (int j = 0; j < K; ++j) {
            if (!((active >> j) & 1u)) continue;
            float v[NS];
#pragma unroll
            for (int k = 0; k < NS; ++k) v[k] = s_part[(j * NS + k) * SH::THREADS + tid];
            Slice sl;
            sl.rhs = r0 + j;
            sl.b = b;
            sl.nb = nb;
            grid_reduce<NS, RedStage<RED>::HINT>(v, P.rc, sl);
        }
    }
}

}  // namespace wd
