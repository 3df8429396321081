// Hopping term of Eq. 1 on FP16 storage with FP16 arithmetic, the regime of
// the paper's implementation (Sec. 5: vectors and links of type _Float16 and
// the stencil's arithmetic carried out in FP16; only the reductions are
// widened to FP32 and FP64).
//
// Every complex number is one half2 word (re in the low half, im in the
// high half), so each instruction performs two FP16 operations and nothing is
// converted on the way from the loads to the accumulator:
//
//   m * x = re(m) (x.re, x.im) + im(m) (-x.im, x.re)   two packed FMAs,
//   i x   = (-x.im, x.re)                              a half swap and a sign flip,
//
// The three steps of a hop are those of Sec. 2 -- project the neighbour to two
// spin components (one packed add per complex number), multiply both by the
// SU(3) link (the third row of a 12-real link rebuilt in FP16 as well),
// rebuild and accumulate (one packed FMA per complex number, the boundary
// phase, the t projector's factor 2 and an exact power-of-two scale of the
// accumulator folded into its constant). The 24 accumulated reals are rounded
// to FP16 by those operations themselves; the epilogue (out = a acc + b y + c z
// and the fused dot products) widens them, undoes the power of two and runs in
// FP32 as in every other kernel.
#pragma once

#include <cmath>

#include "hop_impl.cuh"

namespace wd {

__device__ __forceinline__ __half2 as_h2(unsigned w) { return *reinterpret_cast<__half2*>(&w); }
__device__ __forceinline__ unsigned as_w(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }
// (im, re)
__device__ __forceinline__ __half2 hswap(__half2 x) { return as_h2(__byte_perm(as_w(x), 0u, 0x1032)); }
// i x = (-im, re): exact
__device__ __forceinline__ __half2 times_i(__half2 x) { return as_h2(__byte_perm(as_w(x), 0u, 0x1032) ^ 0x00008000u); }
// m x with ix = i x
__device__ __forceinline__ __half2 cmul16(__half2 m, __half2 x, __half2 ix) {
    return __hfma2(__high2half2(m), ix, __hmul2(__low2half2(m), x));
}
// acc + m x with ix = i x
__device__ __forceinline__ __half2 cmac16(__half2 m, __half2 x, __half2 ix, __half2 acc) {
    return __hfma2(__high2half2(m), ix, __hfma2(__low2half2(m), x, acc));
}

// XOR 0x80008000 negates both halves of a half2 word, 0x80000000 the high half
// only, 0x00008000 the low half only.
// Bits of the half2 word (2^k, 2^k), -14 <= k <= 15.
__host__ __device__ constexpr unsigned h2_pow2(int k) { return ((unsigned)(15 + k) << 10) * 0x10001u; }

// Exponent k of the accumulator scale 2^k: the FP16 sum over the eight
// directions holds 2^k H in, with 2^k the power of two at or below |a| / 8 (a
// the epilogue's coefficient of H in), so that it stays in the range of the
// output a H in with a factor 8 of headroom for partial sums; scaling by a power
// of two is exact in FP16 above the subnormal range. Clamped to [-14, 0];
// computed on the host once per launch.
inline int acc_exponent(double a) {
    int e = 1;
    if (a != 0.0) std::frexp(std::fabs(a), &e);   // |a| = m 2^e, 0.5 <= m < 1
    const int k = e - 1 - 3;
    return k < -14 ? -14 : (k > 0 ? 0 : k);
}

// Half spinor h[k * 3 + c] (spin component k, colour c) of the neighbour
// spinor u (word 3 s + c), projector (1 - gamma_mu) when fwd, else
// (1 + gamma_mu); for mu = 3 the factor 2 is left to the accumulation.
__device__ __forceinline__ void project16(int mu, bool fwd, const uint4 (&u)[3], __half2 (&h)[6]) {
    const __half2 pm = as_h2(fwd ? 0x3C00BC00u : 0xBC003C00u);   // (-s, s), s = +1 forward
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const __half2 p0 = cword(u, c), p1 = cword(u, 3 + c), p2 = cword(u, 6 + c), p3 = cword(u, 9 + c);
        if (mu == 0) {          // h0 = p0 + s i p3, h1 = p1 + s i p2
            h[c] = __hfma2(hswap(p3), pm, p0);
            h[3 + c] = __hfma2(hswap(p2), pm, p1);
        } else if (mu == 1) {   // h0 = p0 + s p3, h1 = p1 - s p2
            h[c] = fwd ? __hadd2(p0, p3) : __hsub2(p0, p3);
            h[3 + c] = fwd ? __hsub2(p1, p2) : __hadd2(p1, p2);
        } else if (mu == 2) {   // h0 = p0 + s i p2, h1 = p1 - s i p3
            h[c] = __hfma2(hswap(p2), pm, p0);
            h[3 + c] = __hfma2(hswap(p3), __hneg2(pm), p1);
        } else {                // fwd: (p2, p3); bwd: (p0, p1)
            h[c] = fwd ? p2 : p0;
            h[3 + c] = fwd ? p3 : p1;
        }
    }
}

// The 3x3 link j of a group of units as 9 half2 words, m[3 a + b] = M_ab
// (word j * R / 2 + 3 a + b of the group; R = 12: row 2 = conj(row0 x row1),
// rebuilt in FP16).
template <int R, int GU>
__device__ __forceinline__ void link_load16(const uint4 (&u)[GU], int j, __half2 (&m)[9]) {
    constexpr int W = R / 2;
#pragma unroll
    for (int e = 0; e < W; ++e) m[e] = as_h2(word_of(u[(j * W + e) >> 2], (j * W + e) & 3));
    if (R == 12) {
        __half2 i1[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) i1[b] = times_i(m[3 + b]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            __half2 z = cmul16(m[b1], m[3 + b2], i1[b2]);                          // row0[b1] row1[b2]
            z = cmac16(as_h2(as_w(m[b2]) ^ 0x80008000u), m[3 + b1], i1[b1], z);     // - row0[b2] row1[b1]
            m[6 + b] = as_h2(as_w(z) ^ 0x80000000u);                               // conjugate
        }
    }
}

// x[k * 3 + a] = sum_b M_ab h[k * 3 + b] for a link given as m[3 a + b].
__device__ __forceinline__ void mul16(const __half2 (&m)[9], const __half2 (&h)[6], __half2 (&x)[6]) {
    __half2 ih[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) ih[i] = times_i(h[i]);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            __half2 z = cmul16(m[3 * a], h[3 * k], ih[3 * k]);
            z = cmac16(m[3 * a + 1], h[3 * k + 1], ih[3 * k + 1], z);
            x[3 * k + a] = cmac16(m[3 * a + 2], h[3 * k + 2], ih[3 * k + 2], z);
        }
}

// x[k * 3 + a] = sum_b M_ab h[k * 3 + b] for link j of a group of units.
template <int R, int GU>
__device__ __forceinline__ void link_mul16(const uint4 (&u)[GU], int j, const __half2 (&h)[6], __half2 (&x)[6]) {
    __half2 m[9];
    link_load16<R, GU>(u, j, m);
    mul16(m, h, x);
}

// acc (word 3 s + c) += f * (rebuilt four-spinor of chi); fb = bits of (f, f).
__device__ __forceinline__ void reconstruct16(int mu, bool fwd, unsigned fb, const __half2 (&x)[6], __half2 (&acc)[12]) {
    const unsigned sfb = fwd ? fb : fb ^ 0x80008000u;      // (sf, sf), sf = s f
    const __half2 f2 = as_h2(fb);
    const __half2 sf2 = as_h2(sfb), nsf2 = as_h2(sfb ^ 0x80008000u);
    const __half2 sfm = as_h2(sfb ^ 0x80000000u);          // (sf, -sf)
    const __half2 msf = as_h2(sfb ^ 0x00008000u);          // (-sf, sf)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const __half2 x0 = x[c], x1 = x[3 + c];
        if (mu == 3) {
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            acc[3 * a0 + c] = __hfma2(f2, x0, acc[3 * a0 + c]);
            acc[3 * a1 + c] = __hfma2(f2, x1, acc[3 * a1 + c]);
            continue;
        }
        acc[c] = __hfma2(f2, x0, acc[c]);
        acc[3 + c] = __hfma2(f2, x1, acc[3 + c]);
        if (mu == 0) {          // comp2 = -s i chi1, comp3 = -s i chi0
            acc[6 + c] = __hfma2(hswap(x1), sfm, acc[6 + c]);
            acc[9 + c] = __hfma2(hswap(x0), sfm, acc[9 + c]);
        } else if (mu == 1) {   // comp2 = -s chi1, comp3 = s chi0
            acc[6 + c] = __hfma2(nsf2, x1, acc[6 + c]);
            acc[9 + c] = __hfma2(sf2, x0, acc[9 + c]);
        } else {                // comp2 = -s i chi0, comp3 = s i chi1
            acc[6 + c] = __hfma2(hswap(x0), sfm, acc[6 + c]);
            acc[9 + c] = __hfma2(hswap(x1), msf, acc[9 + c]);
        }
    }
}

// Epilogue of the FP16-arithmetic hop with Blackwell's packed FP32x2
// multiply and FMA (one complex number per float2): the half2 accumulator is
// widened and unscaled pairwise and out = a H + b y (+ c z) is formed with the
// same per-lane roundings as the scalar epilogue, then rounded to FP16 and
// stored. The dot products of the stored values are the scalar epilogue's
// expressions term for term, so every result has the scalar epilogue's bits.
template <int EPI, int RED>
__device__ __forceinline__ void epilogue16x2(const HopParams& P, uint4* vout, const uint4* vy, const uint4* vz,
                                             const uint4* vrs, int h, const __half2 (&acc)[12], float unscale,
                                             float (&part)[RedSums<RED>::N], bool ftz) {
    const int Vh = P.g.Vh;
    const float2 us = make_float2(unscale, unscale);
    const float ca = (float)P.a, cb = (float)P.b, cc = (float)P.c;
    const float2 ca2 = make_float2(ca, ca), cb2 = make_float2(cb, cb), cc2 = make_float2(cc, cc);
    float2 o[12];
    float2 y2[12];
    if constexpr (EPI >= EPI_Y) {   // o = a H + b y, the product a H fused: fma(a, H, b y)
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const uint4 w = __ldg(vy + (size_t)u * Vh + h);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * u + k;
                y2[i] = __half22float2(as_h2(word_of(w, k)));
                o[i] = __ffma2_rn(ca2, __fmul2_rn(__half22float2(acc[i]), us), __fmul2_rn(cb2, y2[i]));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const float2 a = __fmul2_rn(__half22float2(acc[i]), us);
            o[i] = (EPI == EPI_H && P.a == 1.0) ? a : __fmul2_rn(ca2, a);
        }
    }
    if constexpr (EPI >= EPI_YZ) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const uint4 w = __ldg(vz + (size_t)u * Vh + h);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[4 * u + k] = __ffma2_rn(cc2, __half22float2(as_h2(word_of(w, k))), o[4 * u + k]);
        }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {   // round to FP16, store, and keep the stored values for the dots
        uint4 w = make_uint4(as_w(__float22half2_rn(o[4 * u])), as_w(__float22half2_rn(o[4 * u + 1])),
                             as_w(__float22half2_rn(o[4 * u + 2])), as_w(__float22half2_rn(o[4 * u + 3])));
        if (ftz) w = Unit<__half>::flush(w);
        vout[(size_t)u * Vh + h] = w;
        if constexpr (RED != RED_NONE) {
#pragma unroll
            for (int k = 0; k < 4; ++k) o[4 * u + k] = __half22float2(as_h2(word_of(w, k)));
        }
    }
    if constexpr (RED == RED_RSV) {   // conj(r*) o
        float2 rs[12];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const uint4 w = __ldg(vrs + (size_t)u * Vh + h);
#pragma unroll
            for (int k = 0; k < 4; ++k) rs[4 * u + k] = __half22float2(as_h2(word_of(w, k)));
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            part[0] += rs[i].x * o[i].x + rs[i].y * o[i].y;
            part[1] += rs[i].x * o[i].y - rs[i].y * o[i].x;
        }
    } else if constexpr (RED == RED_TS) {   // (o, q), (o, o), (q, q); q = r* if given, else y
        float2 q2[12];
        if (vrs) {
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const uint4 w = __ldg(vrs + (size_t)u * Vh + h);
#pragma unroll
                for (int k = 0; k < 4; ++k) q2[4 * u + k] = __half22float2(as_h2(word_of(w, k)));
            }
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) q2[i] = y2[i];
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            part[0] += o[i].x * q2[i].x + o[i].y * q2[i].y;
            part[1] += o[i].x * q2[i].y - o[i].y * q2[i].x;
            part[2] += o[i].x * o[i].x + o[i].y * o[i].y;
            part[3] += q2[i].x * q2[i].x + q2[i].y * q2[i].y;
        }
    } else if constexpr (RED == RED_NORM) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            part[0] += o[i].x * o[i].x;
            part[0] += o[i].y * o[i].y;
        }
    }
}

// Launch shape: one site per thread, 128 threads; the plain hop fits 64
// registers with 12-real links (8 blocks per SM) and 72 with 18-real links;
// loading the neighbour spinors two directions ahead (AHEAD = 2) takes 72.
template <int R, int RED, bool MAT, int AHEAD = 2> struct Hop16Bounds {
    static constexpr int THREADS = 128;
    static constexpr int MIN_BLOCKS = (RED == RED_NONE && !MAT) ? ((R == 12 && AHEAD == 1) ? 8 : 7) : 5;
};

// One output site per thread (grid-stride), the neighbour spinors AHEAD
// directions and the next link group one group ahead of their use.
template <int R, int EPI, int RED, bool MAT, int AHEAD = 2>
__global__ void __launch_bounds__(Hop16Bounds<R, RED, MAT, AHEAD>::THREADS, Hop16Bounds<R, RED, MAT, AHEAD>::MIN_BLOCKS)
    hop16_kernel(const HopParams P) {
    [[maybe_unused]] constexpr unsigned wd_tl_tag = RED;   // timeline records: the reduction
    pdl_begin();
    typedef LinkFmt<__half, R> LF;
    constexpr int NS = RedSums<RED>::N;
    constexpr int SU = Spinor<__half>::UNITS;
    const Slice sl = slice_of(P.nrhs);
    if (guarded(P.guard ? P.guard + sl.rhs : nullptr, P.guard_kind)) return;
    const bool ftz = P.guard != nullptr && P.guard[sl.rhs].ftz;
    const long long ro = (long long)sl.rhs * P.vs;
    const uint4* __restrict__ vin = P.in + ro;
    uint4* vout = P.out + ro;
    const uint4* vy = P.y ? P.y + ro : nullptr;
    const uint4* vz = P.z ? P.z + ro : nullptr;
    const uint4* vrs = P.rstar ? P.rstar + ro : nullptr;
    const Geom& g = P.g;
    const int Vh = g.Vh;
    const int ke = P.acc_exp;
    const unsigned c_one = h2_pow2(ke), c_two = h2_pow2(ke + 1);   // (2^k, 2^k), (2^(k+1), 2^(k+1))
    const float unscale = __int_as_float((127 - ke) << 23);        // 2^-k
    float part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0.f;

    for (int h = sl.b * blockDim.x + threadIdx.x; h < Vh; h += sl.nb * blockDim.x) {
        int nbr[8];
        const unsigned wm = site_neighbours(g, P.parity, h, nbr);
        __half2 acc[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = as_h2(0u);

        constexpr int NB = AHEAD + 1;   // neighbour slots: the one in use and AHEAD in flight
        uint4 nbu[NB][SU];
        uint4 lgu[2][LF::GROUP_UNITS];
#pragma unroll
        for (int d = 0; d < AHEAD; ++d)
#pragma unroll
            for (int u = 0; u < SU; ++u) nbu[d][u] = __ldg(vin + (size_t)u * Vh + nbr[d]);
#pragma unroll
        for (int k = 0; k < LF::GROUP_UNITS; ++k) lgu[0][k] = __ldcs(P.links + (size_t)k * Vh + h);

#pragma unroll
        for (int grp = 0; grp < 8 / LF::G; ++grp) {
            uint4 lu[LF::GROUP_UNITS];
#pragma unroll
            for (int k = 0; k < LF::GROUP_UNITS; ++k) lu[k] = lgu[grp & 1][k];
            if (grp + 1 < 8 / LF::G) {
#pragma unroll
                for (int k = 0; k < LF::GROUP_UNITS; ++k)
                    lgu[(grp + 1) & 1][k] = __ldcs(P.links + (size_t)((grp + 1) * LF::GROUP_UNITS + k) * Vh + h);
            }
#pragma unroll
            for (int j = 0; j < LF::G; ++j) {
                const int d = grp * LF::G + j;
                const int mu = d >> 1;
                const bool fwd = (d & 1) == 0;
                uint4 cur[SU];
#pragma unroll
                for (int u = 0; u < SU; ++u) cur[u] = nbu[d % NB][u];
                if (d + AHEAD < 8) {
#pragma unroll
                    for (int u = 0; u < SU; ++u)
                        nbu[(d + AHEAD) % NB][u] = __ldg(vin + (size_t)u * Vh + nbr[d + AHEAD]);
                }
                __half2 hs[6], chi[6];
                project16(mu, fwd, cur, hs);
                link_mul16<R, LF::GROUP_UNITS>(lu, j, hs, chi);
                const unsigned fb = (mu == 3 ? c_two : c_one) ^ ((((wm >> d) & 1u) && g.bc[mu] < 0) ? 0x80008000u : 0u);
                reconstruct16(mu, fwd, fb, chi, acc);
            }
        }

        if (EPI == EPI_H && RED == RED_NONE && !MAT && P.a == 1.0) {   // the plain hop: undo 2^k in FP16 and store
            const __half2 up = as_h2(h2_pow2(-ke));                      // k = -3 here: (8, 8), exact
#pragma unroll
            for (int i = 0; i < 12; ++i) acc[i] = __hmul2(acc[i], up);
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                uint4 w = make_uint4(as_w(acc[4 * u]), as_w(acc[4 * u + 1]), as_w(acc[4 * u + 2]), as_w(acc[4 * u + 3]));
                if (ftz) w = Unit<__half>::flush(w);
                vout[(size_t)u * Vh + h] = w;
            }
        } else if constexpr (MAT) {
            float a32[24];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                a32[2 * i] = __low2float(acc[i]) * unscale;
                a32[2 * i + 1] = __high2float(acc[i]) * unscale;
            }
            hop_epilogue<__half, EPI, RED, MAT>(P, vout, vy, vz, vrs, h, a32, part, ftz);
        } else {
            epilogue16x2<EPI, RED>(P, vout, vy, vz, vrs, h, acc, unscale, part, ftz);
        }
    }

    if constexpr (RED != RED_NONE) grid_reduce<NS, RedStage<RED>::HINT>(part, P.rc, sl);
}

}  // namespace wd
