// Hopping term for FP16 / BF16 / FP32 storage with FP32 arithmetic, two
// output sites per thread.
//
// Same operator and layouts as hop_impl.cuh. The two sites of a thread are
// h and h + V/4 (site B sits Lt/2 time slices after site A, at the same x, y,
// z up to the parity bit of x), and every FP32 value is held as a float2 pair
// (site A, site B), so all arithmetic runs as packed FP32x2 instructions.
//
// FP16 values are widened with integer bit operations instead of conversion
// instructions: moving the 15 magnitude bits of a half up by 13 bits and
// keeping its sign gives, bit for bit, the float equal to the half times
// 2^-112 (normal and subnormal halves alike). The factor 2^112 is folded into
// the projection coefficients (spinor operands) and the epilogue
// coefficients, so the widened values are never rescaled separately. Links
// are widened with conversion instructions (exact).
#pragma once

#include "hop_impl.cuh"
#include "kernels.h"

namespace wd {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Storage traits for the paired path: widen the element i (0..N-1) of a
// 16-byte unit; `SCALE` is the factor the widened value must be multiplied by.
template <typename T> struct Wide;

template <> struct Wide<__half> {
    static constexpr int N = 8;
    static constexpr float SCALE = 5.192296858534828e33f;   // 2^112
    __device__ __forceinline__ static float get(const uint4& u, int i) {
        const unsigned w = word_of(u, i >> 1);
        const unsigned b = (i & 1) ? (((w >> 3) & 0x0fffe000u) | (w & 0x80000000u))
                                   : (((w & 0x7fffu) << 13) | ((w & 0x8000u) << 16));
        return __uint_as_float(b);
    }
};

template <> struct Wide<__nv_bfloat16> {
    static constexpr int N = 8;
    static constexpr float SCALE = 1.0f;
    __device__ __forceinline__ static float get(const uint4& u, int i) {
        const unsigned w = word_of(u, i >> 1);
        return __uint_as_float((i & 1) ? (w & 0xffff0000u) : (w << 16));
    }
};

template <> struct Wide<float> {
    static constexpr int N = 4;
    static constexpr float SCALE = 1.0f;
    __device__ __forceinline__ static float get(const uint4& u, int i) { return __uint_as_float(word_of(u, i)); }
};

// 24 reals of sites a and b as pairs; values are scaled by 1/SCALE.
template <typename T>
__device__ __forceinline__ void load_pair(const uint4* __restrict__ v, int stride, int a, int b, float2 (&s)[24]) {
    constexpr int N = Wide<T>::N;
#pragma unroll
    for (int u = 0; u < 24 / N; ++u) {
        const uint4 wa = __ldg(v + (size_t)u * stride + a);
        const uint4 wb = __ldg(v + (size_t)u * stride + b);
#pragma unroll
        for (int i = 0; i < N; ++i) s[u * N + i] = f2(Wide<T>::get(wa, i), Wide<T>::get(wb, i));
    }
}

// Round pairs to storage and write both sites; s is replaced by the stored values.
template <typename T>
__device__ __forceinline__ void store_pair(uint4* v, int stride, int a, int b, float2 (&s)[24], bool ftz) {
    constexpr int N = Unit<T>::N;
    typedef typename Unit<T>::C C;
#pragma unroll
    for (int u = 0; u < 24 / N; ++u) {
        C va[N], vb[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            va[i] = s[u * N + i].x;
            vb[i] = s[u * N + i].y;
        }
        uint4 wa = Unit<T>::put(va), wb = Unit<T>::put(vb);
        if (ftz) {
            wa = Unit<T>::flush(wa);
            wb = Unit<T>::flush(wb);
        }
        v[(size_t)u * stride + a] = wa;
        v[(size_t)u * stride + b] = wb;
#pragma unroll
        for (int i = 0; i < N; ++i) s[u * N + i] = f2(Unit<T>::get(wa, i), Unit<T>::get(wb, i));
    }
}

#define PRE(s, c) (2 * (3 * (s) + (c)))
#define PIM(s, c) (2 * (3 * (s) + (c)) + 1)

// Projected half spinor H[k][c][re,im] (k = 0, 1) of direction mu, scaled by S.
__device__ __forceinline__ void project2(int mu, bool fwd, const float2 (&p)[24], float2 S, float2 (&h)[12]) {
    const float2 Sp = fwd ? S : neg2(S);   // s * S
    const float2 Sm = neg2(Sp);            // -s * S
    const float2 S2 = add2(S, S);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float2 h0r, h0i, h1r, h1i;
        if (mu == 0) {          // h0 = p0 + s i p3, h1 = p1 + s i p2
            h0r = fma2(p[PIM(3, c)], Sm, mul2(p[PRE(0, c)], S));
            h0i = fma2(p[PRE(3, c)], Sp, mul2(p[PIM(0, c)], S));
            h1r = fma2(p[PIM(2, c)], Sm, mul2(p[PRE(1, c)], S));
            h1i = fma2(p[PRE(2, c)], Sp, mul2(p[PIM(1, c)], S));
        } else if (mu == 1) {   // h0 = p0 + s p3, h1 = p1 - s p2
            h0r = fma2(p[PRE(3, c)], Sp, mul2(p[PRE(0, c)], S));
            h0i = fma2(p[PIM(3, c)], Sp, mul2(p[PIM(0, c)], S));
            h1r = fma2(p[PRE(2, c)], Sm, mul2(p[PRE(1, c)], S));
            h1i = fma2(p[PIM(2, c)], Sm, mul2(p[PIM(1, c)], S));
        } else if (mu == 2) {   // h0 = p0 + s i p2, h1 = p1 - s i p3
            h0r = fma2(p[PIM(2, c)], Sm, mul2(p[PRE(0, c)], S));
            h0i = fma2(p[PRE(2, c)], Sp, mul2(p[PIM(0, c)], S));
            h1r = fma2(p[PIM(3, c)], Sp, mul2(p[PRE(1, c)], S));
            h1i = fma2(p[PRE(3, c)], Sm, mul2(p[PIM(1, c)], S));
        } else {                // fwd: (2 p2, 2 p3); bwd: (2 p0, 2 p1)
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            h0r = mul2(p[PRE(a0, c)], S2);
            h0i = mul2(p[PIM(a0, c)], S2);
            h1r = mul2(p[PRE(a1, c)], S2);
            h1i = mul2(p[PIM(a1, c)], S2);
        }
        h[2 * c] = h0r;
        h[2 * c + 1] = h0i;
        h[6 + 2 * c] = h1r;
        h[6 + 2 * c + 1] = h1i;
    }
}

__device__ __forceinline__ void reconstruct2(int mu, bool fwd, const float2 (&x)[12], float2 (&acc)[24]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 x0r = x[2 * c], x0i = x[2 * c + 1], x1r = x[6 + 2 * c], x1i = x[6 + 2 * c + 1];
        if (mu == 3) {
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            acc[PRE(a0, c)] = add2(acc[PRE(a0, c)], x0r);
            acc[PIM(a0, c)] = add2(acc[PIM(a0, c)], x0i);
            acc[PRE(a1, c)] = add2(acc[PRE(a1, c)], x1r);
            acc[PIM(a1, c)] = add2(acc[PIM(a1, c)], x1i);
            continue;
        }
        acc[PRE(0, c)] = add2(acc[PRE(0, c)], x0r);
        acc[PIM(0, c)] = add2(acc[PIM(0, c)], x0i);
        acc[PRE(1, c)] = add2(acc[PRE(1, c)], x1r);
        acc[PIM(1, c)] = add2(acc[PIM(1, c)], x1i);
        // +s or -s times a pair, as a packed add or subtract
        auto ps = [&](float2 a, float2 v) { return fwd ? add2(a, v) : add2(a, neg2(v)); };
        auto ms = [&](float2 a, float2 v) { return fwd ? add2(a, neg2(v)) : add2(a, v); };
        if (mu == 0) {          // comp2 = -s i chi1, comp3 = -s i chi0
            acc[PRE(2, c)] = ps(acc[PRE(2, c)], x1i);
            acc[PIM(2, c)] = ms(acc[PIM(2, c)], x1r);
            acc[PRE(3, c)] = ps(acc[PRE(3, c)], x0i);
            acc[PIM(3, c)] = ms(acc[PIM(3, c)], x0r);
        } else if (mu == 1) {   // comp2 = -s chi1, comp3 = s chi0
            acc[PRE(2, c)] = ms(acc[PRE(2, c)], x1r);
            acc[PIM(2, c)] = ms(acc[PIM(2, c)], x1i);
            acc[PRE(3, c)] = ps(acc[PRE(3, c)], x0r);
            acc[PIM(3, c)] = ps(acc[PIM(3, c)], x0i);
        } else {                // comp2 = -s i chi0, comp3 = s i chi1
            acc[PRE(2, c)] = ps(acc[PRE(2, c)], x0i);
            acc[PIM(2, c)] = ms(acc[PIM(2, c)], x0r);
            acc[PRE(3, c)] = ms(acc[PRE(3, c)], x1i);
            acc[PIM(3, c)] = ps(acc[PIM(3, c)], x1r);
        }
    }
}

// chi_k = M h_k for the link at element offset `off` of both sites' link units.
template <typename T, int R>
__device__ __forceinline__ void link_mul2(const uint4 (&ua)[LinkFmt<T, R>::GROUP_UNITS],
                                          const uint4 (&ub)[LinkFmt<T, R>::GROUP_UNITS], int off,
                                          const float2 (&h)[12], float2 (&x)[12]) {
    constexpr int N = Unit<T>::N;
    float2 m[18];
#pragma unroll
    for (int e = 0; e < R; ++e) m[e] = f2(Unit<T>::get(ua[(off + e) / N], (off + e) % N),
                                          Unit<T>::get(ub[(off + e) / N], (off + e) % N));
    if (R == 12) {   // row2 = conj(row0 x row1)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            const float2 ar = m[2 * b1], ai = m[2 * b1 + 1], br = m[6 + 2 * b2], bi = m[6 + 2 * b2 + 1];
            const float2 cr = m[2 * b2], ci = m[2 * b2 + 1], dr = m[6 + 2 * b1], di = m[6 + 2 * b1 + 1];
            // re = ar br - ai bi - cr dr + ci di ; im = ar bi + ai br - cr di - ci dr
            float2 re = fma2(ai, neg2(bi), mul2(ar, br));
            re = fma2(cr, neg2(dr), re);
            re = fma2(ci, di, re);
            float2 im = fma2(ai, br, mul2(ar, bi));
            im = fma2(cr, neg2(di), im);
            im = fma2(ci, neg2(dr), im);
            m[12 + 2 * b] = re;
            m[12 + 2 * b + 1] = neg2(im);
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 re = mul2(m[2 * (3 * a)], h[6 * k]);
            float2 im = mul2(m[2 * (3 * a)], h[6 * k + 1]);
            re = fma2(m[2 * (3 * a) + 1], neg2(h[6 * k + 1]), re);
            im = fma2(m[2 * (3 * a) + 1], h[6 * k], im);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                const float2 mr = m[2 * (3 * a + b)], mi = m[2 * (3 * a + b) + 1];
                const float2 hr = h[6 * k + 2 * b], hi = h[6 * k + 2 * b + 1];
                re = fma2(mr, hr, re);
                re = fma2(mi, neg2(hi), re);
                im = fma2(mr, hi, im);
                im = fma2(mi, hr, im);
            }
            x[6 * k + 2 * a] = re;
            x[6 * k + 2 * a + 1] = im;
        }
    }
}

template <typename T, int R, int EPI, int RED>
__global__ void __launch_bounds__(128) hop2_kernel(const HopParams P) {
    pdl_begin();
    typedef LinkFmt<T, R> LF;
    constexpr int NS = RedSums<RED>::N;
    constexpr float SC = Wide<T>::SCALE;
    const Slice sl = slice_of(P.nrhs);
    if (guarded(P.guard ? P.guard + sl.rhs : nullptr, P.guard_kind)) return;
    const long long ro = (long long)sl.rhs * P.vs;     // this right-hand side's vectors
    const uint4* __restrict__ vin = P.in + ro;
    uint4* vout = P.out + ro;
    const uint4* vy = P.y ? P.y + ro : nullptr;
    const uint4* vz = P.z ? P.z + ro : nullptr;
    const uint4* vrs = P.rstar ? P.rstar + ro : nullptr;

    const Geom& g = P.g;
    const int p = P.parity;
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3], Lxh = g.Lxh, Vh = g.Vh;
    const int half = Vh >> 1, Lth = Lt >> 1;
    const int sy = Lxh, sz = Lxh * Ly, st = Lxh * Ly * Lz;
    const float2 A2 = f2((float)P.a, (float)P.a);
    const float2 B2 = f2((float)P.b * SC, (float)P.b * SC);
    const float2 C2 = f2((float)P.c * SC, (float)P.c * SC);
    const float2 SC2 = f2(SC, SC);
    float part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0.f;

    for (int ha = sl.b * blockDim.x + threadIdx.x; ha < half; ha += sl.nb * blockDim.x) {
        const int hb = ha + half;
        const int row = ha / Lxh;
        const int xh = ha - row * Lxh;
        const int y = row % Ly;
        const int r2 = row / Ly;
        const int z = r2 % Lz;
        const int ta = r2 / Lz;
        const int tb = ta + Lth;
        const int xa = 2 * xh + ((p + y + z + ta) & 1);
        const int xb = 2 * xh + ((p + y + z + tb) & 1);
        const int rowb = row + Lth * Ly * Lz;

        float2 acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = f2(0.f, 0.f);

#pragma unroll
        for (int grp = 0; grp < 8 / LF::G; ++grp) {
            uint4 la[LF::GROUP_UNITS], lb[LF::GROUP_UNITS];
#pragma unroll
            for (int k = 0; k < LF::GROUP_UNITS; ++k) {
                la[k] = __ldcs(P.links + (size_t)(grp * LF::GROUP_UNITS + k) * Vh + ha);
                lb[k] = __ldcs(P.links + (size_t)(grp * LF::GROUP_UNITS + k) * Vh + hb);
            }
#pragma unroll
            for (int j = 0; j < LF::G; ++j) {
                const int d = grp * LF::G + j;
                const int mu = d >> 1;
                const bool fwd = (d & 1) == 0;
                int na, nb;
                bool wa, wb;
                if (mu == 0) {
                    wa = fwd ? (xa == Lx - 1) : (xa == 0);
                    wb = fwd ? (xb == Lx - 1) : (xb == 0);
                    const int xna = fwd ? (wa ? 0 : xa + 1) : (wa ? Lx - 1 : xa - 1);
                    const int xnb = fwd ? (wb ? 0 : xb + 1) : (wb ? Lx - 1 : xb - 1);
                    na = row * Lxh + (xna >> 1);
                    nb = rowb * Lxh + (xnb >> 1);
                } else if (mu == 1) {
                    wa = wb = fwd ? (y == Ly - 1) : (y == 0);
                    const int off = fwd ? (wa ? -(Ly - 1) * sy : sy) : (wa ? (Ly - 1) * sy : -sy);
                    na = ha + off;
                    nb = hb + off;
                } else if (mu == 2) {
                    wa = wb = fwd ? (z == Lz - 1) : (z == 0);
                    const int off = fwd ? (wa ? -(Lz - 1) * sz : sz) : (wa ? (Lz - 1) * sz : -sz);
                    na = ha + off;
                    nb = hb + off;
                } else {
                    wa = fwd ? (ta == Lt - 1) : (ta == 0);
                    wb = fwd ? (tb == Lt - 1) : (tb == 0);
                    na = fwd ? (wa ? ha - (Lt - 1) * st : ha + st) : (wa ? ha + (Lt - 1) * st : ha - st);
                    nb = fwd ? (wb ? hb - (Lt - 1) * st : hb + st) : (wb ? hb + (Lt - 1) * st : hb - st);
                }
                const float pha = (wa && g.bc[mu] < 0) ? -SC : SC;
                const float phb = (wb && g.bc[mu] < 0) ? -SC : SC;
                float2 nbp[24];
                load_pair<T>(vin, Vh, na, nb, nbp);
                float2 hs[12], chi[12];
                project2(mu, fwd, nbp, f2(pha, phb), hs);
                link_mul2<T, R>(la, lb, j * R, hs, chi);
                reconstruct2(mu, fwd, chi, acc);
            }
        }

        float2 o[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = mul2(A2, acc[i]);
        float2 yv[24];
        if constexpr (EPI >= EPI_Y) {
            load_pair<T>(vy, Vh, ha, hb, yv);
#pragma unroll
            for (int i = 0; i < 24; ++i) o[i] = fma2(B2, yv[i], o[i]);
        }
        if constexpr (EPI >= EPI_YZ) {
            float2 zv[24];
            load_pair<T>(vz, Vh, ha, hb, zv);
#pragma unroll
            for (int i = 0; i < 24; ++i) o[i] = fma2(C2, zv[i], o[i]);
        }
        store_pair<T>(vout, Vh, ha, hb, o, P.guard != nullptr && P.guard[sl.rhs].ftz);

        if constexpr (RED == RED_RSV) {
            float2 rs[24];
            load_pair<T>(vrs, Vh, ha, hb, rs);
#pragma unroll
            for (int i = 0; i < 12; ++i) {   // conj(rs) * o, both sites
                const float2 rr = mul2(rs[2 * i], SC2), ri = mul2(rs[2 * i + 1], SC2);
                const float2 re = fma2(ri, o[2 * i + 1], mul2(rr, o[2 * i]));
                const float2 im = fma2(neg2(ri), o[2 * i], mul2(rr, o[2 * i + 1]));
                part[0] += re.x + re.y;
                part[1] += im.x + im.y;
            }
        } else if constexpr (RED == RED_TS) {          // (o, q), (o, o), (q, q); q = rstar if given, else y
            if (vrs) load_pair<T>(vrs, Vh, ha, hb, yv);
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const float2 yr = mul2(yv[2 * i], SC2), yi = mul2(yv[2 * i + 1], SC2);
                const float2 re = fma2(o[2 * i + 1], yi, mul2(o[2 * i], yr));
                const float2 im = fma2(neg2(o[2 * i + 1]), yr, mul2(o[2 * i], yi));
                const float2 oo = fma2(o[2 * i + 1], o[2 * i + 1], mul2(o[2 * i], o[2 * i]));
                const float2 yy = fma2(yi, yi, mul2(yr, yr));
                part[0] += re.x + re.y;
                part[1] += im.x + im.y;
                part[2] += oo.x + oo.y;
                part[NS - 1] += yy.x + yy.y;
            }
        } else if constexpr (RED == RED_NORM) {
#pragma unroll
            for (int i = 0; i < 24; ++i) {
                const float2 oo = mul2(o[i], o[i]);
                part[0] += oo.x + oo.y;
            }
        }
    }

    if constexpr (RED != RED_NONE) {
        grid_reduce<NS, RedStage<RED>::HINT>(part, P.rc, sl);   // FP32 or FP64 partials, as the arithmetic
    }
}

#undef PRE
#undef PIM

}  // namespace wd
