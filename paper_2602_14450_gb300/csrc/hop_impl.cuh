// Hopping term of the Wilson matrix (Eq. 1) on one parity:
//   out(x) = a * sum_mu [ (1 - gamma_mu) U_mu(x) in(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ in(x-mu) ]
//            + b * y(x) + c * z(x)
// for the sites x of the output parity, with the fermion boundary phase on
// hops that wrap. The three steps of a hop follow Sec. 2: project the
// neighbour spinor to two spin components, multiply both by the SU(3)
// link, rebuild the four components and accumulate.
//
// Gathered links: for every output site the 8 links it uses are stored
// together, d = 2*mu for U_mu(x) and d = 2*mu+1 for U_mu(x-mu)^+ (already
// conjugated and transposed), each as R reals (R = 18: full matrix row
// major; R = 12: rows 0 and 1, row 2 = conj(row0 x row1)). A site's links are
// 8*R reals split into 16-byte units with the site index fastest, so each
// unit load of a warp is one contiguous 512-byte segment.
#pragma once

#include "kernels.h"

namespace wd {

template <typename T, int R> struct LinkFmt {
    static constexpr int N = Unit<T>::N;
    static constexpr int BYTES = R * (int)sizeof(T);
    static constexpr int G = (BYTES % 16 == 0) ? 1 : ((2 * BYTES) % 16 == 0) ? 2 : ((4 * BYTES) % 16 == 0) ? 4 : 8;
    static constexpr int GROUP_UNITS = G * BYTES / 16;   // units per group of G links
    static constexpr int UNITS = 8 * BYTES / 16;         // units per site
};

template <int RED> struct RedSums { static constexpr int N = 1; };
template <> struct RedSums<RED_RSV> { static constexpr int N = 2; };
template <> struct RedSums<RED_TS> { static constexpr int N = 4; };
template <> struct RedSums<RED_NORM> { static constexpr int N = 1; };

#define RE(s, c) (2 * (3 * (s) + (c)))
#define IM(s, c) (2 * (3 * (s) + (c)) + 1)

// Half spinor h[spin 0..1][colour][re,im] from the neighbour spinor p for
// direction mu: projector (1 - gamma_mu) when fwd, (1 + gamma_mu) otherwise.
template <typename C>
__device__ __forceinline__ void project(int mu, bool fwd, const C (&p)[24], C (&h)[12]) {
    const C s = fwd ? C(1) : C(-1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C h0r, h0i, h1r, h1i;
        if (mu == 0) {          // h0 = p0 + s i p3, h1 = p1 + s i p2
            h0r = p[RE(0, c)] - s * p[IM(3, c)];
            h0i = p[IM(0, c)] + s * p[RE(3, c)];
            h1r = p[RE(1, c)] - s * p[IM(2, c)];
            h1i = p[IM(1, c)] + s * p[RE(2, c)];
        } else if (mu == 1) {   // h0 = p0 + s p3, h1 = p1 - s p2
            h0r = p[RE(0, c)] + s * p[RE(3, c)];
            h0i = p[IM(0, c)] + s * p[IM(3, c)];
            h1r = p[RE(1, c)] - s * p[RE(2, c)];
            h1i = p[IM(1, c)] - s * p[IM(2, c)];
        } else if (mu == 2) {   // h0 = p0 + s i p2, h1 = p1 - s i p3
            h0r = p[RE(0, c)] - s * p[IM(2, c)];
            h0i = p[IM(0, c)] + s * p[RE(2, c)];
            h1r = p[RE(1, c)] + s * p[IM(3, c)];
            h1i = p[IM(1, c)] - s * p[RE(3, c)];
        } else {                // fwd: (2 p2, 2 p3); bwd: (2 p0, 2 p1)
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            h0r = p[RE(a0, c)] + p[RE(a0, c)];
            h0i = p[IM(a0, c)] + p[IM(a0, c)];
            h1r = p[RE(a1, c)] + p[RE(a1, c)];
            h1i = p[IM(a1, c)] + p[IM(a1, c)];
        }
        h[2 * c] = h0r;
        h[2 * c + 1] = h0i;
        h[6 + 2 * c] = h1r;
        h[6 + 2 * c + 1] = h1i;
    }
}

// Accumulate the rebuilt four-spinor of chi = U h into acc.
template <typename C>
__device__ __forceinline__ void reconstruct(int mu, bool fwd, const C (&x)[12], C (&acc)[24]) {
    const C s = fwd ? C(1) : C(-1);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C x0r = x[2 * c], x0i = x[2 * c + 1], x1r = x[6 + 2 * c], x1i = x[6 + 2 * c + 1];
        if (mu == 3) {
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            acc[RE(a0, c)] += x0r; acc[IM(a0, c)] += x0i;
            acc[RE(a1, c)] += x1r; acc[IM(a1, c)] += x1i;
            continue;
        }
        acc[RE(0, c)] += x0r; acc[IM(0, c)] += x0i;
        acc[RE(1, c)] += x1r; acc[IM(1, c)] += x1i;
        if (mu == 0) {          // comp2 = -s i chi1, comp3 = -s i chi0
            acc[RE(2, c)] += s * x1i; acc[IM(2, c)] -= s * x1r;
            acc[RE(3, c)] += s * x0i; acc[IM(3, c)] -= s * x0r;
        } else if (mu == 1) {   // comp2 = -s chi1, comp3 = s chi0
            acc[RE(2, c)] -= s * x1r; acc[IM(2, c)] -= s * x1i;
            acc[RE(3, c)] += s * x0r; acc[IM(3, c)] += s * x0i;
        } else {                // comp2 = -s i chi0, comp3 = s i chi1
            acc[RE(2, c)] += s * x0i; acc[IM(2, c)] -= s * x0r;
            acc[RE(3, c)] -= s * x1i; acc[IM(3, c)] += s * x1r;
        }
    }
}

// chi_k = M h_k (k = 0, 1) for the link stored at element offset `off` of the
// group's units.
template <typename T, int R>
__device__ __forceinline__ void link_mul(const uint4 (&u)[LinkFmt<T, R>::GROUP_UNITS], int off,
                                         const typename Unit<T>::C (&h)[12], typename Unit<T>::C (&x)[12]) {
    typedef typename Unit<T>::C C;
    constexpr int N = Unit<T>::N;
    C m[18];
#pragma unroll
    for (int e = 0; e < R; ++e) m[e] = Unit<T>::get(u[(off + e) / N], (off + e) % N);
    if (R == 12) {
        // row2 = conj(row0 x row1)
#define MR(a, b) m[2 * (3 * (a) + (b))]
#define MI(a, b) m[2 * (3 * (a) + (b)) + 1]
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            C re = MR(0, b1) * MR(1, b2) - MI(0, b1) * MI(1, b2) - (MR(0, b2) * MR(1, b1) - MI(0, b2) * MI(1, b1));
            C im = MR(0, b1) * MI(1, b2) + MI(0, b1) * MR(1, b2) - (MR(0, b2) * MI(1, b1) + MI(0, b2) * MR(1, b1));
            m[12 + 2 * b] = re;
            m[12 + 2 * b + 1] = -im;
        }
#undef MR
#undef MI
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C re = 0, im = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const C mr = m[2 * (3 * a + b)], mi = m[2 * (3 * a + b) + 1];
                const C hr = h[6 * k + 2 * b], hi = h[6 * k + 2 * b + 1];
                re += mr * hr - mi * hi;
                im += mr * hi + mi * hr;
            }
            x[6 * k + 2 * a] = re;
            x[6 * k + 2 * a + 1] = im;
        }
    }
}

template <typename T, int R, int EPI, int RED, bool PF>
__global__ void __launch_bounds__(256) hop_kernel(const HopParams P) {
    typedef typename Unit<T>::C C;
    typedef LinkFmt<T, R> LF;
    constexpr int NS = RedSums<RED>::N;
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
    const int sy = Lxh, sz = Lxh * Ly, st = Lxh * Ly * Lz;
    const C ca = (C)P.a, cb = (C)P.b, cc = (C)P.c;
    C part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0;

    for (int h = sl.b * blockDim.x + threadIdx.x; h < Vh; h += sl.nb * blockDim.x) {
        const int row = h / Lxh;
        const int xh = h - row * Lxh;
        const int y = row % Ly;
        const int r2 = row / Ly;
        const int z = r2 % Lz;
        const int t = r2 / Lz;
        const int x = 2 * xh + ((p + y + z + t) & 1);

        C acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0;

        // neighbour site and wrap flag of each direction d = 2 mu (+mu), 2 mu + 1 (-mu)
        int hnb[8];
        bool wrp[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int mu = d >> 1;
            const bool fwd = (d & 1) == 0;
            if (mu == 0) {
                wrp[d] = fwd ? (x == Lx - 1) : (x == 0);
                const int xn = fwd ? (wrp[d] ? 0 : x + 1) : (wrp[d] ? Lx - 1 : x - 1);
                hnb[d] = row * Lxh + (xn >> 1);
            } else if (mu == 1) {
                wrp[d] = fwd ? (y == Ly - 1) : (y == 0);
                hnb[d] = fwd ? (wrp[d] ? h - (Ly - 1) * sy : h + sy) : (wrp[d] ? h + (Ly - 1) * sy : h - sy);
            } else if (mu == 2) {
                wrp[d] = fwd ? (z == Lz - 1) : (z == 0);
                hnb[d] = fwd ? (wrp[d] ? h - (Lz - 1) * sz : h + sz) : (wrp[d] ? h + (Lz - 1) * sz : h - sz);
            } else {
                wrp[d] = fwd ? (t == Lt - 1) : (t == 0);
                hnb[d] = fwd ? (wrp[d] ? h - (Lt - 1) * st : h + st) : (wrp[d] ? h + (Lt - 1) * st : h - st);
            }
        }
        // PF: the raw units of the next direction's neighbour and the next link
        // group are loaded before the current direction is computed.
        constexpr int SU = Spinor<T>::UNITS;
        uint4 nbu[2][SU];
        uint4 lgu[2][LF::GROUP_UNITS];
        if (PF) {
#pragma unroll
            for (int u = 0; u < SU; ++u) nbu[0][u] = __ldg(vin + (size_t)u * Vh + hnb[0]);
#pragma unroll
            for (int k = 0; k < LF::GROUP_UNITS; ++k) lgu[0][k] = __ldcs(P.links + (size_t)k * Vh + h);
        }

#pragma unroll
        for (int grp = 0; grp < 8 / LF::G; ++grp) {
            uint4 lu[LF::GROUP_UNITS];
            if (PF) {
#pragma unroll
                for (int k = 0; k < LF::GROUP_UNITS; ++k) lu[k] = lgu[grp & 1][k];
                if (grp + 1 < 8 / LF::G) {
#pragma unroll
                    for (int k = 0; k < LF::GROUP_UNITS; ++k)
                        lgu[(grp + 1) & 1][k] = __ldcs(P.links + (size_t)((grp + 1) * LF::GROUP_UNITS + k) * Vh + h);
                }
            } else {
#pragma unroll
                for (int k = 0; k < LF::GROUP_UNITS; ++k)
                    lu[k] = __ldcs(P.links + (size_t)(grp * LF::GROUP_UNITS + k) * Vh + h);
            }
#pragma unroll
            for (int j = 0; j < LF::G; ++j) {
                const int d = grp * LF::G + j;
                const int mu = d >> 1;
                const bool fwd = (d & 1) == 0;
                const bool wrap = wrp[d];
                C nb[24];
                if (PF) {
                    uint4 cur[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) cur[u] = nbu[d & 1][u];
                    if (d + 1 < 8) {
#pragma unroll
                        for (int u = 0; u < SU; ++u) nbu[(d + 1) & 1][u] = __ldg(vin + (size_t)u * Vh + hnb[d + 1]);
                    }
#pragma unroll
                    for (int u = 0; u < SU; ++u)
#pragma unroll
                        for (int i = 0; i < Unit<T>::N; ++i) nb[u * Unit<T>::N + i] = Unit<T>::get(cur[u], i);
                } else {
                    load_spinor<T>(vin, Vh, hnb[d], nb);
                }
                C hs[12], chi[12];
                project<C>(mu, fwd, nb, hs);
                if (g.bc[mu] < 0) {      // uniform: only antiperiodic directions pay for the phase
                    const C ph = wrap ? C(-1) : C(1);
#pragma unroll
                    for (int i = 0; i < 12; ++i) hs[i] *= ph;
                }
                link_mul<T, R>(lu, j * R, hs, chi);
                reconstruct<C>(mu, fwd, chi, acc);
            }
        }

        // epilogue: out = a * acc + b * y + c * z
        C o[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = ca * acc[i];
        C yv[24];
        if constexpr (EPI >= EPI_Y) {
            load_spinor<T>(vy, Vh, h, yv);
#pragma unroll
            for (int i = 0; i < 24; ++i) o[i] += cb * yv[i];
        }
        if constexpr (EPI >= EPI_YZ) {
            C zv[24];
            load_spinor<T>(vz, Vh, h, zv);
#pragma unroll
            for (int i = 0; i < 24; ++i) o[i] += cc * zv[i];
        }
        store_spinor<T>(vout, Vh, h, o);

        if constexpr (RED == RED_RSV) {
            C rs[24];
            load_spinor<T>(vrs, Vh, h, rs);
#pragma unroll
            for (int i = 0; i < 12; ++i) {   // conj(rs) * o
                part[0] += rs[2 * i] * o[2 * i] + rs[2 * i + 1] * o[2 * i + 1];
                part[1] += rs[2 * i] * o[2 * i + 1] - rs[2 * i + 1] * o[2 * i];
            }
        } else if constexpr (RED == RED_TS) {          // (o, q), (o, o), (q, q); q = rstar if given, else y
            C qv[24];
            if (vrs) {
                load_spinor<T>(vrs, Vh, h, qv);
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) qv[i] = yv[i];
            }
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                part[0] += o[2 * i] * qv[2 * i] + o[2 * i + 1] * qv[2 * i + 1];
                part[1] += o[2 * i] * qv[2 * i + 1] - o[2 * i + 1] * qv[2 * i];
                part[2] += o[2 * i] * o[2 * i] + o[2 * i + 1] * o[2 * i + 1];
                part[NS - 1] += qv[2 * i] * qv[2 * i] + qv[2 * i + 1] * qv[2 * i + 1];
            }
        } else if constexpr (RED == RED_NORM) {
#pragma unroll
            for (int i = 0; i < 24; ++i) part[0] += o[i] * o[i];
        }
    }

    if constexpr (RED != RED_NONE) {
        double v[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) v[k] = (double)part[k];
        grid_reduce<NS>(v, P.rc, sl);
    }
}

#undef RE
#undef IM

}  // namespace wd
