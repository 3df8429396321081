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

#include <type_traits>

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
// The scalar stage a reducing hop runs at its end in the solvers.
template <int RED> struct RedStage {
    static constexpr int HINT = RED == RED_RSV ? ST_ALPHA : RED == RED_TS ? ST_OMEGA : RED == RED_NORM ? ST_OUTER : ST_NONE;
};

#define RE(s, c) (2 * (3 * (s) + (c)))
#define IM(s, c) (2 * (3 * (s) + (c)) + 1)

template <typename C> __device__ __forceinline__ C fmac(C a, C b, C c);
template <> __device__ __forceinline__ float fmac<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fmac<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// Half spinor h[spin 0..1][colour][re,im] from the neighbour spinor p for
// direction mu: projector (1 - gamma_mu) when fwd, (1 + gamma_mu) otherwise.
// For mu = 3 the projector is 2 P with P a spin selection; the factor 2 is
// left to reconstruct() (scaling by 2 is exact, so the result is the same).
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
        } else {                // fwd: (p2, p3); bwd: (p0, p1), times 2 later
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            h0r = p[RE(a0, c)];
            h0i = p[IM(a0, c)];
            h1r = p[RE(a1, c)];
            h1i = p[IM(a1, c)];
        }
        h[2 * c] = h0r;
        h[2 * c + 1] = h0i;
        h[6 + 2 * c] = h1r;
        h[6 + 2 * c + 1] = h1i;
    }
}

// The same projection for an FP16 neighbour spinor, on the stored values:
// each colour's (re, im) pair is one half2 word, so the projector's sums are
// one rounded half2 add (or fused add of the swapped pair times +-1) per
// complex number, and only the 12 projected reals are widened to FP32.
__device__ __forceinline__ __half2 cword(const uint4 (&u)[3], int q) {
    unsigned w = word_of(u[q >> 2], q & 3);
    return *reinterpret_cast<__half2*>(&w);
}
__device__ __forceinline__ void project_half2(int mu, bool fwd, const uint4 (&u)[3], float (&h)[12]) {
    const __half2 pm = fwd ? __floats2half2_rn(-1.f, 1.f) : __floats2half2_rn(1.f, -1.f);   // (-s, s)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const __half2 p0 = cword(u, c), p1 = cword(u, 3 + c), p2 = cword(u, 6 + c), p3 = cword(u, 9 + c);
        __half2 a0, a1;
        if (mu == 0) {          // h0 = p0 + s i p3, h1 = p1 + s i p2
            a0 = __hfma2(__lowhigh2highlow(p3), pm, p0);
            a1 = __hfma2(__lowhigh2highlow(p2), pm, p1);
        } else if (mu == 1) {   // h0 = p0 + s p3, h1 = p1 - s p2
            a0 = fwd ? __hadd2(p0, p3) : __hsub2(p0, p3);
            a1 = fwd ? __hsub2(p1, p2) : __hadd2(p1, p2);
        } else if (mu == 2) {   // h0 = p0 + s i p2, h1 = p1 - s i p3
            a0 = __hfma2(__lowhigh2highlow(p2), pm, p0);
            a1 = __hfma2(__lowhigh2highlow(p3), __hneg2(pm), p1);
        } else {                // fwd: (p2, p3); bwd: (p0, p1), times 2 later
            a0 = fwd ? p2 : p0;
            a1 = fwd ? p3 : p1;
        }
        h[2 * c] = __low2float(a0);
        h[2 * c + 1] = __high2float(a0);
        h[6 + 2 * c] = __low2float(a1);
        h[6 + 2 * c + 1] = __high2float(a1);
    }
}

// acc += f * (rebuilt four-spinor of chi = U h); f carries the boundary
// phase of the hop and, for mu = 3, the projector's factor 2. Every term is
// one fused multiply-add.
template <typename C>
__device__ __forceinline__ void reconstruct(int mu, bool fwd, C f, const C (&x)[12], C (&acc)[24]) {
    const C sf = fwd ? f : -f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C x0r = x[2 * c], x0i = x[2 * c + 1], x1r = x[6 + 2 * c], x1i = x[6 + 2 * c + 1];
        if (mu == 3) {
            const int a0 = fwd ? 2 : 0, a1 = fwd ? 3 : 1;
            acc[RE(a0, c)] = fmac(f, x0r, acc[RE(a0, c)]);
            acc[IM(a0, c)] = fmac(f, x0i, acc[IM(a0, c)]);
            acc[RE(a1, c)] = fmac(f, x1r, acc[RE(a1, c)]);
            acc[IM(a1, c)] = fmac(f, x1i, acc[IM(a1, c)]);
            continue;
        }
        acc[RE(0, c)] = fmac(f, x0r, acc[RE(0, c)]);
        acc[IM(0, c)] = fmac(f, x0i, acc[IM(0, c)]);
        acc[RE(1, c)] = fmac(f, x1r, acc[RE(1, c)]);
        acc[IM(1, c)] = fmac(f, x1i, acc[IM(1, c)]);
        if (mu == 0) {          // comp2 = -s i chi1, comp3 = -s i chi0
            acc[RE(2, c)] = fmac(sf, x1i, acc[RE(2, c)]);
            acc[IM(2, c)] = fmac(-sf, x1r, acc[IM(2, c)]);
            acc[RE(3, c)] = fmac(sf, x0i, acc[RE(3, c)]);
            acc[IM(3, c)] = fmac(-sf, x0r, acc[IM(3, c)]);
        } else if (mu == 1) {   // comp2 = -s chi1, comp3 = s chi0
            acc[RE(2, c)] = fmac(-sf, x1r, acc[RE(2, c)]);
            acc[IM(2, c)] = fmac(-sf, x1i, acc[IM(2, c)]);
            acc[RE(3, c)] = fmac(sf, x0r, acc[RE(3, c)]);
            acc[IM(3, c)] = fmac(sf, x0i, acc[IM(3, c)]);
        } else {                // comp2 = -s i chi0, comp3 = s i chi1
            acc[RE(2, c)] = fmac(sf, x0i, acc[RE(2, c)]);
            acc[IM(2, c)] = fmac(-sf, x0r, acc[IM(2, c)]);
            acc[RE(3, c)] = fmac(-sf, x1i, acc[RE(3, c)]);
            acc[IM(3, c)] = fmac(sf, x1r, acc[IM(3, c)]);
        }
    }
}

// chi_k = M h_k (k = 0, 1) for the link stored at element offset `off` of the
// group's units. Each output is one multiply and a chain of fused
// multiply-adds (no separate adds).
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
            C re = MI(0, b2) * MI(1, b1);
            re = fmac(-MR(0, b2), MR(1, b1), re);
            re = fmac(-MI(0, b1), MI(1, b2), re);
            re = fmac(MR(0, b1), MR(1, b2), re);
            C nim = MR(0, b2) * MI(1, b1);
            nim = fmac(MI(0, b2), MR(1, b1), nim);
            nim = fmac(-MR(0, b1), MI(1, b2), nim);
            nim = fmac(-MI(0, b1), MR(1, b2), nim);
            m[12 + 2 * b] = re;
            m[12 + 2 * b + 1] = nim;
        }
#undef MR
#undef MI
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const C* mr = &m[6 * a];
            const C* hk = &h[6 * k];
            C re = mr[0] * hk[0];
            re = fmac(-mr[1], hk[1], re);
            re = fmac(mr[2], hk[2], re);
            re = fmac(-mr[3], hk[3], re);
            re = fmac(mr[4], hk[4], re);
            re = fmac(-mr[5], hk[5], re);
            C im = mr[0] * hk[1];
            im = fmac(mr[1], hk[0], im);
            im = fmac(mr[2], hk[3], im);
            im = fmac(mr[3], hk[2], im);
            im = fmac(mr[4], hk[5], im);
            im = fmac(mr[5], hk[4], im);
            x[6 * k + 2 * a] = re;
            x[6 * k + 2 * a + 1] = im;
        }
    }
}

// Epilogue of one output site: out = a * acc + b * y + c * z, rounded to
// storage and written, and this thread's share of the fused dot products.
template <typename T, int EPI, int RED, bool MAT = false>
__device__ __forceinline__ void hop_epilogue(const HopParams& P, uint4* vout, const uint4* vy, const uint4* vz,
                                             const uint4* vrs, int h, typename Unit<T>::C (&acc)[24],
                                             typename Unit<T>::C (&part)[RedSums<RED>::N], bool ftz) {
    typedef typename Unit<T>::C C;
    constexpr int NS = RedSums<RED>::N;
    const int Vh = P.g.Vh;
    const C ca = (C)P.a, cb = (C)P.b, cc = (C)P.c;
    if constexpr (MAT) {   // the site-local block (clover C^-1, Eqs. 4-5, chiral packing) applied to the hop
        C t[24];
        mat_mul_chiral<T>(P.mat, Vh, h, acc, t);
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = t[i];
    }
    C o[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) o[i] = (EPI == EPI_H && P.a == 1.0) ? acc[i] : ca * acc[i];
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
    store_spinor<T>(vout, Vh, h, o, ftz);

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

// link_mul with FP32 arithmetic on packed pairs: the two half-spinor columns
// k = 0, 1 share every link element, so each complex multiply-add of a row is
// four FP32x2 fused multiply-adds on (column 0, column 1) pairs.
template <typename T, int R>
__device__ __forceinline__ void link_mul_pair(const uint4 (&u)[LinkFmt<T, R>::GROUP_UNITS], int off,
                                              const float (&h)[12], float (&x)[12]) {
    constexpr int N = Unit<T>::N;
    float m[18];
#pragma unroll
    for (int e = 0; e < R; ++e) m[e] = Unit<T>::get(u[(off + e) / N], (off + e) % N);
    if (R == 12) {
#define MR(a, b) m[2 * (3 * (a) + (b))]
#define MI(a, b) m[2 * (3 * (a) + (b)) + 1]
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            float re = MI(0, b2) * MI(1, b1);
            re = __fmaf_rn(-MR(0, b2), MR(1, b1), re);
            re = __fmaf_rn(-MI(0, b1), MI(1, b2), re);
            re = __fmaf_rn(MR(0, b1), MR(1, b2), re);
            float nim = MR(0, b2) * MI(1, b1);
            nim = __fmaf_rn(MI(0, b2), MR(1, b1), nim);
            nim = __fmaf_rn(-MR(0, b1), MI(1, b2), nim);
            nim = __fmaf_rn(-MI(0, b1), MR(1, b2), nim);
            m[12 + 2 * b] = re;
            m[12 + 2 * b + 1] = nim;
        }
#undef MR
#undef MI
    }
    float2 hr[3], hi[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        hr[b] = make_float2(h[2 * b], h[6 + 2 * b]);
        hi[b] = make_float2(h[2 * b + 1], h[6 + 2 * b + 1]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float* mr = &m[6 * a];
        float2 re = __fmul2_rn(make_float2(mr[0], mr[0]), hr[0]);
        re = __ffma2_rn(make_float2(-mr[1], -mr[1]), hi[0], re);
        re = __ffma2_rn(make_float2(mr[2], mr[2]), hr[1], re);
        re = __ffma2_rn(make_float2(-mr[3], -mr[3]), hi[1], re);
        re = __ffma2_rn(make_float2(mr[4], mr[4]), hr[2], re);
        re = __ffma2_rn(make_float2(-mr[5], -mr[5]), hi[2], re);
        float2 im = __fmul2_rn(make_float2(mr[0], mr[0]), hi[0]);
        im = __ffma2_rn(make_float2(mr[1], mr[1]), hr[0], im);
        im = __ffma2_rn(make_float2(mr[2], mr[2]), hi[1], im);
        im = __ffma2_rn(make_float2(mr[3], mr[3]), hr[1], im);
        im = __ffma2_rn(make_float2(mr[4], mr[4]), hi[2], im);
        im = __ffma2_rn(make_float2(mr[5], mr[5]), hr[2], im);
        x[2 * a] = re.x;
        x[6 + 2 * a] = re.y;
        x[2 * a + 1] = im.x;
        x[6 + 2 * a + 1] = im.y;
    }
}

// Launch bounds of hop_kernel: the FP16 look-ahead kernels without a fused
// reduction fit 72 registers (7 blocks of 128 threads per SM; measured 3%
// faster, while BF16 there is 6% slower), the other 16-bit kernels keep 80
// (3 blocks of 256); FP32 128 and FP64 255 registers.
template <typename T, int RED, bool PF, bool MAT = false> struct HopBounds {
    static constexpr bool LEAN = std::is_same<T, __half>::value && PF && RED == RED_NONE && !MAT;
    static constexpr int THREADS = LEAN ? 128 : 256;
    static constexpr int MIN_BLOCKS = LEAN ? 7 : sizeof(T) == 2 ? (PF ? 3 : 2) : sizeof(T) == 4 ? 2 : 1;
};

template <typename T, int R, int EPI, int RED, bool PF, bool PAIR = false, bool MAT = false>
__global__ void __launch_bounds__(HopBounds<T, RED, PF, MAT>::THREADS, HopBounds<T, RED, PF, MAT>::MIN_BLOCKS)
    hop_kernel(const HopParams P) {
    [[maybe_unused]] constexpr unsigned wd_tl_tag = RED;   // timeline records: the reduction
    pdl_begin();
    typedef typename Unit<T>::C C;
    typedef LinkFmt<T, R> LF;
    constexpr int NS = RedSums<RED>::N;
    const Slice sl = slice_of(P.nrhs);
    if (guarded(P.guard ? P.guard + sl.rhs : nullptr, P.guard_kind)) return;
    const bool ftz = P.guard != nullptr && P.guard[sl.rhs].ftz;
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
    C part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0;

    for (int h = sl.b * blockDim.x + threadIdx.x; h < Vh; h += sl.nb * blockDim.x) {
        const int row = g.fxh.div(h);
        const int xh = h - row * Lxh;
        const int r2 = g.fy.div(row);
        const int y = row - r2 * Ly;
        const int t = g.fz.div(r2);
        const int z = r2 - t * Lz;
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
                C hs[12], chi[12];
                if (PF) {
                    uint4 cur[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) cur[u] = nbu[d & 1][u];
                    if (d + 1 < 8) {
#pragma unroll
                        for (int u = 0; u < SU; ++u) nbu[(d + 1) & 1][u] = __ldg(vin + (size_t)u * Vh + hnb[d + 1]);
                    }
                    if constexpr (std::is_same<T, __half>::value) {
                        project_half2(mu, fwd, cur, hs);
                    } else {
                        C nb[24];
#pragma unroll
                        for (int u = 0; u < SU; ++u)
#pragma unroll
                            for (int i = 0; i < Unit<T>::N; ++i) nb[u * Unit<T>::N + i] = Unit<T>::get(cur[u], i);
                        project<C>(mu, fwd, nb, hs);
                    }
                } else {
                    C nb[24];
                    load_spinor<T>(vin, Vh, hnb[d], nb);
                    project<C>(mu, fwd, nb, hs);
                }
                if constexpr (PAIR) {
                    link_mul_pair<T, R>(lu, j * R, hs, chi);
                } else {
                    link_mul<T, R>(lu, j * R, hs, chi);
                }
                const C f = (mu == 3 ? C(2) : C(1)) * ((wrap && g.bc[mu] < 0) ? C(-1) : C(1));
                reconstruct<C>(mu, fwd, f, chi, acc);
            }
        }

        hop_epilogue<T, EPI, RED, MAT>(P, vout, vy, vz, vrs, h, acc, part, ftz);
    }

    if constexpr (RED != RED_NONE) {
        grid_reduce<NS, RedStage<RED>::HINT>(part, P.rc, sl);   // FP32 or FP64 partials, as the arithmetic
    }
}

// ------------------------------------------------ shared-memory ring form ---
//
// The same hop with every thread streaming its operands through a private
// two-slot ring in shared memory: while the directions of one link group are
// computed from one slot, the asynchronous copies (cp.async, 16 bytes per
// thread and instruction) of the next group -- or of the first group of the
// thread's next site -- fill the other. The copies hold no registers, so the
// prefetch distance grows without lowering occupancy, and the grid-stride loop
// carries the pipeline across sites. Each thread reads only what it copied
// itself, so the only synchronisation is cp.async.wait_group.

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Whether unit u (N reals) of a neighbour spinor enters the hop in direction
// d: the t hops project onto two spin components only (+t: spins 2, 3;
// -t: spins 0, 1), so a unit holding none of those reals is not copied.
template <int N> __host__ __device__ constexpr bool unit_needed(int d, int u) {
    return (d >> 1) != 3 || (u * N < ((d & 1) ? 12 : 24) && (u + 1) * N > ((d & 1) ? 0 : 12));
}

// Copy the operands of link group `grp` of output site h into the ring slot
// that starts at `dst` (element u of the slot at dst[u * nt]).
template <typename T, int R>
__device__ __forceinline__ void issue_group(const uint4* vin, const uint4* links, int Vh, int h, int grp,
                                            const int (&nbr)[8], uint4* dst, int nt) {
    typedef LinkFmt<T, R> LF;
    constexpr int SU = Spinor<T>::UNITS;
#pragma unroll
    for (int j = 0; j < LF::G; ++j) {
        const int d = grp * LF::G + j;
#pragma unroll
        for (int u = 0; u < SU; ++u)
            if (unit_needed<Unit<T>::N>(d, u)) cp_async16(dst + (j * SU + u) * nt, vin + (size_t)u * Vh + nbr[d]);
    }
#pragma unroll
    for (int k = 0; k < LF::GROUP_UNITS; ++k)
        cp_async16(dst + (LF::G * SU + k) * nt, links + (size_t)(grp * LF::GROUP_UNITS + k) * Vh + h);
    cp_async_commit();
}

// Units of 16 bytes per thread and ring slot; the ring kernel runs with a
// fixed block size so that every shared-memory offset is a constant.
template <typename T, int R> struct RingFmt {
    static constexpr int BLOCK = 128;
    static constexpr int SLOT = LinkFmt<T, R>::G * Spinor<T>::UNITS + LinkFmt<T, R>::GROUP_UNITS;
    static constexpr int GROUPS = 8 / LinkFmt<T, R>::G;
    static constexpr size_t SMEM = (size_t)2 * SLOT * 16 * BLOCK;
};

template <typename T, int R, int EPI, int RED>
__global__ void __launch_bounds__(RingFmt<T, R>::BLOCK, 6) hop_ring_kernel(const HopParams P) {
    pdl_begin();
    typedef typename Unit<T>::C C;
    typedef LinkFmt<T, R> LF;
    typedef RingFmt<T, R> RF;
    constexpr int NS = RedSums<RED>::N;
    constexpr int SU = Spinor<T>::UNITS;
    constexpr int N = Unit<T>::N;
    static_assert(RF::GROUPS % 2 == 0, "a site's groups alternate between the two slots");
    extern __shared__ uint4 ring[];
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
    constexpr int nt = RF::BLOCK;
    const int Vh = g.Vh, p = P.parity;
    uint4* mine = ring + threadIdx.x;
    C part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0;

    const int stride = sl.nb * nt;
    int h = sl.b * nt + threadIdx.x;
    int nbr[8];
    unsigned wm = 0;
    if (h < Vh) {
        wm = site_neighbours(g, p, h, nbr);
        issue_group<T, R>(vin, P.links, Vh, h, 0, nbr, mine, nt);
    }
    while (h < Vh) {
        C acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0;
        const int hn = h + stride;
        int nbn[8];
        unsigned wmn = 0;
#pragma unroll
        for (int grp = 0; grp < RF::GROUPS; ++grp) {
            uint4* nxt = mine + ((grp + 1) & 1) * RF::SLOT * nt;
            if (grp + 1 < RF::GROUPS) {
                issue_group<T, R>(vin, P.links, Vh, h, grp + 1, nbr, nxt, nt);
            } else if (hn < Vh) {
                wmn = site_neighbours(g, p, hn, nbn);
                issue_group<T, R>(vin, P.links, Vh, hn, 0, nbn, nxt, nt);
            } else {
                cp_async_commit();          // empty group: the wait below counts the same way
            }
            cp_async_wait<1>();
            const uint4* cur = mine + (grp & 1) * RF::SLOT * nt;
            uint4 lu[LF::GROUP_UNITS];
#pragma unroll
            for (int k = 0; k < LF::GROUP_UNITS; ++k) lu[k] = cur[(LF::G * SU + k) * nt];
#pragma unroll
            for (int j = 0; j < LF::G; ++j) {
                const int d = grp * LF::G + j;
                const int mu = d >> 1;
                const bool fwd = (d & 1) == 0;
                C nb[24];
#pragma unroll
                for (int u = 0; u < SU; ++u) {
                    if (unit_needed<N>(d, u)) {
                        const uint4 w = cur[(j * SU + u) * nt];
#pragma unroll
                        for (int i = 0; i < N; ++i) nb[u * N + i] = Unit<T>::get(w, i);
                    } else {
#pragma unroll
                        for (int i = 0; i < N; ++i) nb[u * N + i] = 0;
                    }
                }
                C hs[12], chi[12];
                project<C>(mu, fwd, nb, hs);
                link_mul<T, R>(lu, j * R, hs, chi);
                const C f = (mu == 3 ? C(2) : C(1)) * ((((wm >> d) & 1u) && g.bc[mu] < 0) ? C(-1) : C(1));
                reconstruct<C>(mu, fwd, f, chi, acc);
            }
        }
        hop_epilogue<T, EPI, RED>(P, vout, vy, vz, vrs, h, acc, part, ftz);
        h = hn;
        wm = wmn;
#pragma unroll
        for (int d = 0; d < 8; ++d) nbr[d] = nbn[d];
    }
    cp_async_wait<0>();

    if constexpr (RED != RED_NONE) {
        grid_reduce<NS, RedStage<RED>::HINT>(part, P.rc, sl);   // FP32 or FP64 partials, as the arithmetic
    }
}

#undef RE
#undef IM

}  // namespace wd
