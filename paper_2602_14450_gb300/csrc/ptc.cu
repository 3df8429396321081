// Learned right preconditioner M: a linear, gauge-equivariant parallel-transport
// convolution network with channels 1 -> 12 -> 1, no activation (so M is linear).
//
//   layer: out[c](x) = sum_{k=0..8} sum_{c'} W[k, c, c'] (T_k in[c'])(x)
//   T_0 = 1, T_{1+d} with d = 2 mu: U_mu(x) f(x+mu); d = 2 mu + 1: U_mu(x-mu)^+ f(x-mu)
//
// The transport of site x in direction d uses exactly the gathered link d of
// the hop kernels (hop_impl.cuh) and the same boundary phases. W[k, c, c'] is
// a complex 4x4 matrix on spin. M maps an even-site vector to an even-site
// vector: layer 1 fans the single input channel out to 12 hidden channels on
// all sites, layer 2 folds them back onto the even sites.
//
// Weights (flat float layout shared with the C ABI): W1[k][c][s][t][re,im]
// then W2[k][c][s][t][re,im], 9 * 12 * 16 complex each. The kernels read them
// as given (the library stores BF16-rounded values for the solver).
//
// Training kernels compute, for L = sum |M v - y|^2/|y|^2 + mu |A M v - v|^2/|v|^2,
// the weight gradients dL/dRe W + i dL/dIm W by the adjoint network.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "blas_impl.cuh"
#include "handle.h"

namespace wd {

constexpr int PTC_C = 12;                 // hidden channels
constexpr int PTC_LAYER = 9 * PTC_C * 16; // complex weights per layer
constexpr int PTC_FLOATS = 2 * PTC_LAYER * 2;

// Link d of site h (gathered layout, R reals of LT) as 18 floats (row 2 rebuilt for R = 12).
template <typename LT, int R>
__device__ __forceinline__ void load_link(const uint4* __restrict__ links, int Vh, int h, int d, float (&m)[18]) {
    constexpr int N = Unit<LT>::N;
#pragma unroll
    for (int e = 0; e < R; ++e) {
        const int el = d * R + e;
        const uint4 w = __ldg(links + (size_t)(el / N) * Vh + h);
        m[e] = (float)Unit<LT>::get(w, el % N);
    }
    if (R == 12) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            const float ar = m[2 * b1], ai = m[2 * b1 + 1], br = m[6 + 2 * b2], bi = m[6 + 2 * b2 + 1];
            const float cr = m[2 * b2], ci = m[2 * b2 + 1], dr = m[6 + 2 * b1], di = m[6 + 2 * b1 + 1];
            m[12 + 2 * b] = ar * br - ai * bi - cr * dr + ci * di;
            m[12 + 2 * b + 1] = -(ar * bi + ai * br - cr * di - ci * dr);
        }
    }
}

// phi = m f on colour for each of the 4 spins (f, phi: [spin][colour][re,im]);
// each output is one multiply and a chain of fused multiply-adds.
__device__ __forceinline__ void colour_mul(const float (&m)[18], const float (&f)[24], float (&phi)[24]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float* mr = &m[6 * a];
            const float* fs = &f[6 * s];
            float re = mr[0] * fs[0];
            re = __fmaf_rn(-mr[1], fs[1], re);
            re = __fmaf_rn(mr[2], fs[2], re);
            re = __fmaf_rn(-mr[3], fs[3], re);
            re = __fmaf_rn(mr[4], fs[4], re);
            re = __fmaf_rn(-mr[5], fs[5], re);
            float im = mr[0] * fs[1];
            im = __fmaf_rn(mr[1], fs[0], im);
            im = __fmaf_rn(mr[2], fs[3], im);
            im = __fmaf_rn(mr[3], fs[2], im);
            im = __fmaf_rn(mr[4], fs[5], im);
            im = __fmaf_rn(mr[5], fs[4], im);
            phi[2 * (3 * s + a)] = re;
            phi[2 * (3 * s + a) + 1] = im;
        }
}

// acc += w phi on spin (w: 16 complex [s][t] as float2 in shared memory).
__device__ __forceinline__ void spin_mul_add_p(const float2* w, const float* phi, float (&acc)[24]) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float fr = phi[2 * (3 * t + a)], fi = phi[2 * (3 * t + a) + 1];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const float2 c = w[4 * s + t];
                acc[2 * (3 * s + a)] = __fmaf_rn(-c.y, fi, __fmaf_rn(c.x, fr, acc[2 * (3 * s + a)]));
                acc[2 * (3 * s + a) + 1] = __fmaf_rn(c.y, fr, __fmaf_rn(c.x, fi, acc[2 * (3 * s + a) + 1]));
            }
        }
}
__device__ __forceinline__ void spin_mul_add(const float2* w, const float (&phi)[24], float (&acc)[24]) {
    spin_mul_add_p(w, phi, acc);
}

// T_k f at site h of parity p, f read from the parity its support lives on.
// Returns false when that source parity holds no data.
template <typename TF, typename LT, int R>
__device__ __forceinline__ bool transported(const Geom& g, int p, int h, const Coord& c, int k, const uint4* f_same,
                                            const uint4* f_other, const uint4* links_p, float (&phi)[24]) {
    if (k == 0) {
        if (!f_same) return false;
        load_spinor<TF>(f_same, g.Vh, h, phi);
        return true;
    }
    if (!f_other) return false;
    const int d = k - 1;
    bool wrap;
    const int hn = neighbour(g, h, c, d, &wrap);
    float f[24], m[18];
    load_spinor<TF>(f_other, g.Vh, hn, f);
    if (wrap && g.bc[d >> 1] < 0) {
#pragma unroll
        for (int i = 0; i < 24; ++i) f[i] = -f[i];
    }
    load_link<LT, R>(links_p, g.Vh, h, d, m);
    colour_mul(m, f, phi);
    return true;
}

__device__ __forceinline__ const uint4* H_channel(const uint4* H, long long hvs, int c, int p) {
    return H + (size_t)(2 * c + p) * hvs;
}

// Fan-out layer: one input channel (per-parity pointers, null = zero) to
// channel blockIdx.y of H on parity blockIdx.z. H layout: [c][parity][units][Vh].
template <typename TIN, typename TH, typename LT, int R>
__global__ void __launch_bounds__(128) k_ptc_fanout(Geom g, const uint4* in_e, const uint4* in_o, uint4* H,
                                                    long long hvs, const uint4* links_e, const uint4* links_o,
                                                    const float* w, const SolverState* guard) {
    if (guarded(guard, GUARD_INNER)) return;
    __shared__ float2 ws[9 * 16];
    const int c = blockIdx.y, p = blockIdx.z;
    for (int i = threadIdx.x; i < 9 * 16; i += blockDim.x) {
        const int k = i / 16, e = i % 16;
        ws[i] = make_float2(w[2 * ((k * PTC_C + c) * 16 + e)], w[2 * ((k * PTC_C + c) * 16 + e) + 1]);
    }
    __syncthreads();
    const uint4* same = p == 0 ? in_e : in_o;
    const uint4* other = p == 0 ? in_o : in_e;
    const uint4* links = p == 0 ? links_e : links_o;
    uint4* out = H + (size_t)(2 * c + p) * hvs;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        const Coord co = coord_of(g, p, h);
        float acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int k = 0; k < 9; ++k) {
            float phi[24];
            if (transported<TIN, LT, R>(g, p, h, co, k, same, other, links, phi)) spin_mul_add(&ws[16 * k], phi, acc);
        }
        store_spinor<TH>(out, g.Vh, h, acc);
    }
}

// Fan-in layer: the 12 channels of H to one output channel on the even sites.
template <typename TH, typename TOUT, typename LT, int R>
__global__ void __launch_bounds__(128) k_ptc_fanin(Geom g, const uint4* H, long long hvs, uint4* out_e,
                                                   const uint4* links_e, const float* w, const SolverState* guard) {
    if (guarded(guard, GUARD_INNER)) return;
    __shared__ float2 ws[9 * PTC_C * 16];
    for (int i = threadIdx.x; i < 9 * PTC_C * 16; i += blockDim.x) ws[i] = make_float2(w[2 * i], w[2 * i + 1]);
    __syncthreads();
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        const Coord co = coord_of(g, 0, h);
        float acc[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int k = 0; k < 9; ++k) {
            float m[18];
            int hn = h;
            bool wrap = false;
            if (k > 0) {
                hn = neighbour(g, h, co, k - 1, &wrap);
                load_link<LT, R>(links_e, g.Vh, h, k - 1, m);
            }
            const float ph = (wrap && g.bc[(k - 1) >> 1] < 0) ? -1.f : 1.f;
#pragma unroll 1
            for (int c = 0; c < PTC_C; ++c) {
                const uint4* src = H + (size_t)(2 * c + (k == 0 ? 0 : 1)) * hvs;
                float f[24], phi[24];
                load_spinor<TH>(src, g.Vh, hn, f);
                if (k == 0) {
#pragma unroll
                    for (int i = 0; i < 24; ++i) phi[i] = f[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 24; ++i) f[i] *= ph;
                    colour_mul(m, f, phi);
                }
                spin_mul_add(&ws[16 * (k * PTC_C + c)], phi, acc);
            }
        }
        store_spinor<TOUT>(out_e, g.Vh, h, acc);
    }
}

// ---------------------------------------------------------- collapsed M ---
//
// The network has no nonlinearity and its spin weights commute with the
// colour transports, so its two layers collapse exactly:
//   M psi = sum_{k2} T_{k2} phi_{k2},  phi_{k2} = sum_{k1} V[k2][k1] T_{k1} psi,
//   V[k2][k1] = sum_c W2[k2][c] W1[k1][c]   (4x4 spin matrix products).
// For an even-site input (odd sites zero) only phi_0 = V[0][0] psi on the
// even sites and phi_{1+d} (d = 0..7) on the odd sites are nonzero, so M is
// two stencil passes with eight odd-site intermediate fields instead of the
// twelve hidden channels on both parities. The layered kernels above stay for
// training, which needs the hidden activations.

// V[k2][k1][s][t] from the BF16-rounded weights (double accumulation).
__global__ void k_ptc_collapse(const float* w, float2* V) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 81 * 16; i += gridDim.x * blockDim.x) {
        const int k2 = i / 144, k1 = (i / 16) % 9, s = (i / 4) % 4, t = i % 4;
        double re = 0.0, im = 0.0;
        for (int c = 0; c < PTC_C; ++c)
            for (int u = 0; u < 4; ++u) {
                const float* a = w + 2 * PTC_LAYER + 2 * ((k2 * PTC_C + c) * 16 + 4 * s + u);
                const float* b = w + 2 * ((k1 * PTC_C + c) * 16 + 4 * u + t);
                re += (double)a[0] * b[0] - (double)a[1] * b[1];
                im += (double)a[0] * b[1] + (double)a[1] * b[0];
            }
        V[i] = make_float2((float)re, (float)im);
    }
}

constexpr int S1_SITES = 32;                // sites per block of the first pass
constexpr int S1_STRIDE = 8 * 24 + 1;       // floats per site of its transport tile (padded)
constexpr int S1_VROW = 8 * 16 + 1;         // float2 per k2 row of its V tile (padded)

// First pass on the odd sites y: the eight transports T_{1+d} psi(y) (warp mu
// computes directions 2 mu and 2 mu + 1 for the block's 32 sites) go to shared
// memory; then warp mu forms phi_{1+d}(y) = sum_{k1} V[1+d][k1] T_{k1} psi(y)
// for its two directions and stores them.
template <typename TIN, typename TPHI, typename LT, int R>
__global__ void __launch_bounds__(128) k_ptc_s1(Geom g, const uint4* in_e, uint4* phi, long long pvs,
                                                const uint4* links_o, const float2* V, const SolverState* guard) {
    if (guarded(guard, GUARD_INNER)) return;
    __shared__ float ts[S1_SITES * S1_STRIDE];
    __shared__ float2 vs[8 * S1_VROW];
    for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
        const int a = i / 128, b = i % 128;     // a = k2 - 1, b = 16 (k1 - 1) + e
        vs[a * S1_VROW + b] = V[((1 + a) * 9 + 1 + b / 16) * 16 + b % 16];
    }
    __syncthreads();
    const int mu = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* mine = ts + lane * S1_STRIDE;
    for (int base = blockIdx.x * S1_SITES; base < g.Vh; base += gridDim.x * S1_SITES) {
        const int h = base + lane;
        const bool ok = h < g.Vh;
        if (ok) {
            const Coord co = coord_of(g, 1, h);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int d = 2 * mu + j;
                bool wrap;
                const int hn = neighbour(g, h, co, d, &wrap);
                float f[24], m[18], t[24];
                load_spinor<TIN>(in_e, g.Vh, hn, f);
                if (wrap && g.bc[mu] < 0) {
#pragma unroll
                    for (int i = 0; i < 24; ++i) f[i] = -f[i];
                }
                load_link<LT, R>(links_o, g.Vh, h, d, m);
                colour_mul(m, f, t);
#pragma unroll
                for (int i = 0; i < 24; ++i) mine[d * 24 + i] = t[i];
            }
        }
        __syncthreads();
        if (ok) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int d2 = 2 * mu + j;
                float acc[24];
#pragma unroll
                for (int i = 0; i < 24; ++i) acc[i] = 0.f;
#pragma unroll 1
                for (int k1 = 0; k1 < 8; ++k1) spin_mul_add_p(&vs[d2 * S1_VROW + 16 * k1], mine + 24 * k1, acc);
                store_spinor<TPHI>(phi + (size_t)d2 * pvs, g.Vh, h, acc);
            }
        }
        __syncthreads();
    }
}

// The 2 units of gathered-link storage that hold link d of a site (12 halves
// of an FP16 12-real link start at element 12 d), and the link rebuilt from them.
template <typename LT> __device__ __forceinline__ void load_link_units(const uint4* __restrict__ links, int Vh, int h,
                                                                       int d, uint4 (&u)[2]) {
    const int base = (12 * d) / Unit<LT>::N;
    u[0] = __ldg(links + (size_t)base * Vh + h);
    u[1] = __ldg(links + (size_t)(base + 1) * Vh + h);
}
template <typename LT> __device__ __forceinline__ void link_from_units(const uint4 (&u)[2], int d, float (&m)[18]) {
    constexpr int N = Unit<LT>::N;
    const int base = (12 * d) / N;
#pragma unroll
    for (int e = 0; e < 12; ++e) {
        const int el = 12 * d + e;
        m[e] = (float)Unit<LT>::get(u[el / N - base], el % N);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {   // row 2 = conj(row 0 x row 1)
        const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
        float re = m[2 * b2 + 1] * m[6 + 2 * b1 + 1];
        re = __fmaf_rn(-m[2 * b2], m[6 + 2 * b1], re);
        re = __fmaf_rn(-m[2 * b1 + 1], m[6 + 2 * b2 + 1], re);
        re = __fmaf_rn(m[2 * b1], m[6 + 2 * b2], re);
        float nim = m[2 * b2] * m[6 + 2 * b1 + 1];
        nim = __fmaf_rn(m[2 * b2 + 1], m[6 + 2 * b1], nim);
        nim = __fmaf_rn(-m[2 * b1], m[6 + 2 * b2 + 1], nim);
        nim = __fmaf_rn(-m[2 * b1 + 1], m[6 + 2 * b2], nim);
        m[12 + 2 * b] = re;
        m[12 + 2 * b + 1] = nim;
    }
}

// Second pass of the FP16 path with colour-major phi (as the tensor-core first
// pass writes it): every direction's phi units and link units are loaded one
// direction ahead of the arithmetic that uses them.
template <typename TIN, typename TPHI, typename TOUT, typename LT>
__global__ void __launch_bounds__(128, 5) k_ptc_s2_pf(Geom g, const uint4* in_e, const uint4* phi, long long pvs,
                                                      uint4* out_e, const uint4* links_e, const float2* V,
                                                      const SolverState* guard) {
    if (guarded(guard, GUARD_INNER)) return;
    __shared__ float2 v00[16];
    if (threadIdx.x < 16) v00[threadIdx.x] = V[threadIdx.x];
    __syncthreads();
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        int nbr[8];
        const unsigned wm = site_neighbours(g, 0, h, nbr);
        uint4 fu[2][3], lu[2][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) fu[0][a] = __ldg(phi + (size_t)a * g.Vh + nbr[0]);
        load_link_units<LT>(links_e, g.Vh, h, 0, lu[0]);
        float acc[24], f[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0.f;
        load_spinor<TIN>(in_e, g.Vh, h, f);
        spin_mul_add(v00, f, acc);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            if (d + 1 < 8) {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    fu[(d + 1) & 1][a] = __ldg(phi + (size_t)(d + 1) * pvs + (size_t)a * g.Vh + nbr[d + 1]);
                load_link_units<LT>(links_e, g.Vh, h, d + 1, lu[(d + 1) & 1]);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int e = 0; e < 8; ++e) f[2 * (3 * (e >> 1) + a) + (e & 1)] = Unit<TPHI>::get(fu[d & 1][a], e);
            float m[18], t[24];
            link_from_units<LT>(lu[d & 1], d, m);
            colour_mul(m, f, t);
            const float ph = (((wm >> d) & 1u) && g.bc[d >> 1] < 0) ? -1.f : 1.f;
#pragma unroll
            for (int i = 0; i < 24; ++i) acc[i] = __fmaf_rn(ph, t[i], acc[i]);
        }
        store_spinor<TOUT>(out_e, g.Vh, h, acc);
    }
}

// Second pass on the even sites x: M psi(x) = V[0][0] psi(x) + sum_d T_{1+d} phi_{1+d}(x).
// CMAJOR: phi units are colour-major (unit a = spins 0..3 of colour a, as the
// tensor-core first pass writes them); otherwise the spinor order of load_spinor.
template <typename TIN, typename TPHI, typename TOUT, typename LT, int R, bool CMAJOR>
__global__ void __launch_bounds__(128) k_ptc_s2(Geom g, const uint4* in_e, const uint4* phi, long long pvs,
                                                uint4* out_e, const uint4* links_e, const float2* V,
                                                const SolverState* guard) {
    if (guarded(guard, GUARD_INNER)) return;
    __shared__ float2 v00[16];
    if (threadIdx.x < 16) v00[threadIdx.x] = V[threadIdx.x];
    __syncthreads();
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
        const Coord co = coord_of(g, 0, h);
        float acc[24], f[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = 0.f;
        load_spinor<TIN>(in_e, g.Vh, h, f);
        spin_mul_add(v00, f, acc);
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            bool wrap;
            const int hn = neighbour(g, h, co, d, &wrap);
            float m[18], t[24];
            if constexpr (CMAJOR) {
                constexpr int NU = Unit<TPHI>::N;
                static_assert(NU == 8, "colour-major phi holds 8 reals per unit");
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uint4 w = __ldg(phi + (size_t)d * pvs + (size_t)a * g.Vh + hn);
#pragma unroll
                    for (int e = 0; e < 8; ++e) f[2 * (3 * (e >> 1) + a) + (e & 1)] = Unit<TPHI>::get(w, e);
                }
            } else {
                load_spinor<TPHI>(phi + (size_t)d * pvs, g.Vh, hn, f);
            }
            load_link<LT, R>(links_e, g.Vh, h, d, m);
            colour_mul(m, f, t);
            const float ph = (wrap && g.bc[d >> 1] < 0) ? -1.f : 1.f;
#pragma unroll
            for (int i = 0; i < 24; ++i) acc[i] = __fmaf_rn(ph, t[i], acc[i]);
        }
        store_spinor<TOUT>(out_e, g.Vh, h, acc);
    }
}

}  // namespace wd

#include "ptc_tc.cuh"

namespace wd {

// Weight gradient: dW[k][c] += sum_x sum_colour G_c(x) (x) conj(T_k F_c(x)), summed into
// grad (float, [k][c][s][t][re,im]). Mode 0 (layer 2): G = one even channel,
// F = the channels of H. Mode 1 (layer 1): G = the channels of H-shaped g_H,
// F = one even channel. One block row per (k, c) = (blockIdx.y, blockIdx.z).
template <typename LT, int R>
__global__ void __launch_bounds__(128) k_ptc_wgrad(Geom g, int mode, const uint4* G, const uint4* F, long long hvs,
                                                   const uint4* links_e, const uint4* links_o, float* part) {
    const int k = blockIdx.y, c = blockIdx.z;
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    for (int p = 0; p < 2; ++p) {
        if (mode == 0 && p == 1) break;      // layer-2 output lives on even sites only
        const uint4* links = p == 0 ? links_e : links_o;
        const uint4* gsrc = mode == 0 ? G : G + (size_t)(2 * c + p) * hvs;
        const uint4 *f_same, *f_other;
        if (mode == 0) {
            f_same = H_channel(F, hvs, c, p);
            f_other = H_channel(F, hvs, c, 1 - p);
        } else {
            f_same = p == 0 ? F : nullptr;
            f_other = p == 0 ? nullptr : F;
        }
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x) {
            const Coord co = coord_of(g, p, h);
            float phi[24];
            if (!transported<float, LT, R>(g, p, h, co, k, f_same, f_other, links, phi)) continue;
            float gv[24];
            load_spinor<float>(gsrc, g.Vh, h, gv);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {   // g_{s,a} conj(phi_{t,a})
                        const float gr = gv[2 * (3 * s + a)], gi = gv[2 * (3 * s + a) + 1];
                        const float fr = phi[2 * (3 * t + a)], fi = phi[2 * (3 * t + a) + 1];
                        acc[2 * (4 * s + t)] += gr * fr + gi * fi;
                        acc[2 * (4 * s + t) + 1] += gi * fr - gr * fi;
                    }
        }
    }
    // block sum of the 32 accumulators into this block's partial-sum slots (summed in block order later)
    __shared__ float sh[32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float v = acc[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
        part[((size_t)(k * PTC_C + c) * gridDim.x + blockIdx.x) * 32 + threadIdx.x] = v;
    }
}

// grad[(k, c)][32] += sum over the nb blocks of k_ptc_wgrad's partial sums, in block order (deterministic).
__global__ void k_ptc_wgrad_sum(int nb, const float* part, float* grad) {
    const int kc = blockIdx.x;   // k * PTC_C + c
    float v = 0.f;
    for (int b = 0; b < nb; ++b) v += part[((size_t)kc * nb + b) * 32 + threadIdx.x];
    grad[2 * (kc * 16) + threadIdx.x] += v;
}

}  // namespace wd

namespace wd {

// ------------------------------------------------------------ small kernels ---

// z = a x + b y over n floats (y may be null)
__global__ void k_f32_lincomb(long long n, float a, const float* x, float b, const float* y, float* z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = a * x[i] + (y ? b * y[i] : 0.f);
}

// part[block] = this block's share of sum x_i y_i (double accumulation)
__global__ void k_f32_dot(long long n, const float* x, const float* y, double* part) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    double v[1] = {s};
    block_sum<1>(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

// *out = sum of nb partial sums in block order (deterministic)
__global__ void k_sum_partials(int nb, const double* part, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *out = s;
    }
}

// gamma5 of the Dirac representation: (g5 f)_s = -f_{s xor 2}
__global__ void k_gamma5_f32(int Vh, const uint4* in, uint4* out) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        float f[24], o[24];
        load_spinor_cg<float>(in, Vh, h, f);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int j = 0; j < 6; ++j) o[6 * s + j] = -f[6 * (s ^ 2) + j];
        store_spinor<float>(out, Vh, h, o);
    }
}

// Fan-out weights of the adjoint of layer 2: Wa[k'][c] = W2[k][c]^+, k' the opposite hop of k.
__global__ void k_ptc_adjoint_weights(const float* w2, float* wa) {
    for (int i = threadIdx.x; i < PTC_LAYER; i += blockDim.x) {
        const int k = i / (PTC_C * 16), c = (i / 16) % PTC_C, s = (i / 4) % 4, t = i % 4;
        const int ka = k == 0 ? 0 : 1 + ((k - 1) ^ 1);
        const int src = (k * PTC_C + c) * 16 + 4 * t + s;   // transpose
        const int dst = (ka * PTC_C + c) * 16 + 4 * s + t;
        wa[2 * dst] = w2[2 * src];
        wa[2 * dst + 1] = -w2[2 * src + 1];                 // conjugate
    }
}

// Adam on the master weights, then the BF16-rounded copy used by the kernels.
__global__ void k_adam(int n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2, float* weff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        m[i] = b1 * m[i] + (1.f - b1) * gi;
        v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
        w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
        weff[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
    }
}

__global__ void k_round_bf16(int n, const float* w, float* weff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        weff[i] = __bfloat162float(__float2bfloat16_rn(w[i]));
}

// ------------------------------------------------------------------- host ---

static int grid_for(int n, int block) {
    int g = (n + block - 1) / block;
    const int cap = num_sms() * 8;
    return g < 1 ? 1 : (g > cap ? cap : g);
}

struct PtcBufs {
    float *w, *weff, *m, *v, *grad, *wadj;
    float2* V;      // collapsed spin weights V[k2][k1][s][t] of weff
};

static int ptc_bufs(wd_handle* h, PtcBufs* b) {
    const size_t nb = sizeof(float) * PTC_FLOATS;
    b->w = (float*)workspace(h, "ptc.w", nb);
    b->weff = (float*)workspace(h, "ptc.weff", nb);
    b->m = (float*)workspace(h, "ptc.m", nb);
    b->v = (float*)workspace(h, "ptc.v", nb);
    b->grad = (float*)workspace(h, "ptc.grad", nb);
    b->wadj = (float*)workspace(h, "ptc.wadj", nb / 2);
    b->V = (float2*)workspace(h, "ptc.V", sizeof(float2) * 81 * 16);
    if (!b->w || !b->weff || !b->m || !b->v || !b->grad || !b->wadj || !b->V)
        return fail(h, WD_ERR_CUDA, "out of device memory");
    return WD_OK;
}

// Hidden buffer of 12 channels x 2 parities in storage type of `prec`.
static uint4* ptc_hidden(wd_handle* h, int prec, const char* name) {
    return (uint4*)workspace(h, name, vec_bytes(h, prec) * 2 * PTC_C);
}

// M in = out: FP32 path (FP32 hidden, FP32 18-real links) or FP16 path
// (BF16 hidden, FP16 12-real links), weights from `w` (device, flat layout).
int* ptc_err(wd_handle* h);

// Whether M (its first pass, and in training the fan-out layers) mixes channels
// on the tensor cores (environment WD_PTC_TC=0 selects the FP32-core kernels).
static bool ptc_tensor_cores() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("WD_PTC_TC");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Training fan-out (FP32 input on the even sites, FP32 18-real links) into the
// 12 hidden channels of H on both parities: the even sites (hop 0 only) on the
// FP32 cores, the odd sites (the eight transports) on the tensor cores.
static cudaError_t ptc_fanout_f32(wd_handle* h, const uint4* in_e, uint4* H, long long hvs, const uint4* le,
                                  const uint4* lo, const float* w, cudaStream_t s, int* err) {
    const Geom& g = h->g;
    const int gx = grid_for(g.Vh, 128);
    if (!ptc_tensor_cores()) {
        k_ptc_fanout<float, float, float, 18><<<dim3(gx, PTC_C, 2), 128, 0, s>>>(g, in_e, nullptr, H, hvs, le, lo, w,
                                                                               nullptr);
        return cudaGetLastError();
    }
    k_ptc_fanout<float, float, float, 18><<<dim3(gx, PTC_C, 1), 128, 0, s>>>(g, in_e, nullptr, H, hvs, le, lo, w,
                                                                           nullptr);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_ptc_fanout_odd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tcf::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long tiles = ((long long)g.Vh + tc::TILE_M - 1) / tc::TILE_M;
    const long long tcap = (long long)num_sms() * 3;
    const int gt = (int)(tiles < tcap ? tiles : tcap);
    k_ptc_fanout_odd_tc<<<gt, 128, tcf::SMEM_BYTES, s>>>(g, in_e, H, hvs, lo, w, err, h->wait_rounds);
    return cudaGetLastError();
}

cudaError_t ptc_apply_raw(wd_handle* h, int prec, const uint4* in_e, uint4* out_e, uint4* H, const float* w,
                          const uint4* le, const uint4* lo, cudaStream_t s, const SolverState* guard) {
    const Geom& g = h->g;
    const int blk = 128, gx = grid_for(g.Vh, blk);
    if (prec == WD_FP32) {
        const long long hvs = (long long)spinor_units(WD_FP32) * g.Vh;
        cudaError_t e = ptc_fanout_f32(h, in_e, H, hvs, le, lo, w, s, ptc_err(h));
        if (e != cudaSuccess) return e;
        k_ptc_fanin<float, float, float, 18><<<gx, blk, 0, s>>>(g, H, hvs, out_e, le, w + 2 * PTC_LAYER, guard);
    } else {
        const long long hvs = (long long)spinor_units(WD_BF16) * g.Vh;
        k_ptc_fanout<__half, __nv_bfloat16, __half, 12><<<dim3(gx, PTC_C, 2), blk, 0, s>>>(g, in_e, nullptr, H, hvs,
                                                                                         le, lo, w, guard);
        k_ptc_fanin<__nv_bfloat16, __half, __half, 12><<<gx, blk, 0, s>>>(g, H, hvs, out_e, le, w + 2 * PTC_LAYER, guard);
    }
    return cudaGetLastError();
}

// Device flag raised by a kernel whose bounded wait gave up.
int* ptc_err(wd_handle* h) { return (int*)workspace(h, "ptc.err", sizeof(int)); }

// Intermediate fields phi_{1+d} of the collapsed M: 8 odd-site vectors in the
// storage type of `prec` (FP32 for WD_FP32, BF16 otherwise).
static uint4* ptc_phi(wd_handle* h, int prec) {
    return prec == WD_FP32 ? (uint4*)workspace(h, "ptc.phi32", vec_bytes(h, WD_FP32) * 8)
                           : (uint4*)workspace(h, "ptc.phi16", vec_bytes(h, WD_BF16) * 8);
}


cudaError_t ptc_apply_m(wd_handle* h, int prec, const uint4* in_e, uint4* out_e, uint4* PHI, const float2* V,
                        const uint4* le, const uint4* lo, cudaStream_t s, const SolverState* guard, int* err) {
    const Geom& g = h->g;
    long long groups = ((long long)g.Vh + S1_SITES - 1) / S1_SITES;
    const long long cap = (long long)num_sms() * 6;
    const int g1 = (int)(groups < cap ? groups : cap);
    const int g2 = grid_for(g.Vh, 128);
    if (prec == WD_FP32) {
        const long long pvs = (long long)spinor_units(WD_FP32) * g.Vh;
        k_ptc_s1<float, float, float, 18><<<g1, 128, 0, s>>>(g, in_e, PHI, pvs, lo, V, guard);
        k_ptc_s2<float, float, float, float, 18, false><<<g2, 128, 0, s>>>(g, in_e, PHI, pvs, out_e, le, V, guard);
    } else if (ptc_tensor_cores()) {
        const long long pvs = (long long)spinor_units(WD_BF16) * g.Vh;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_ptc_s1_tc<__half, __half, 12>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const long long tiles = ((long long)g.Vh + tc::TILE_M - 1) / tc::TILE_M;
        const long long tcap = (long long)num_sms() * 3;
        const int gt = (int)(tiles < tcap ? tiles : tcap);
        k_ptc_s1_tc<__half, __half, 12><<<gt, 128, tc::SMEM_BYTES, s>>>(g, in_e, PHI, pvs, lo, V, guard, err,
                                                                         h->wait_rounds);
        k_ptc_s2_pf<__half, __nv_bfloat16, __half, __half><<<g2, 128, 0, s>>>(g, in_e, PHI, pvs, out_e, le, V, guard);
    } else {
        const long long pvs = (long long)spinor_units(WD_BF16) * g.Vh;
        k_ptc_s1<__half, __nv_bfloat16, __half, 12><<<g1, 128, 0, s>>>(g, in_e, PHI, pvs, lo, V, guard);
        k_ptc_s2<__half, __nv_bfloat16, __half, __half, 12, false><<<g2, 128, 0, s>>>(g, in_e, PHI, pvs, out_e, le, V,
                                                                                        guard);
    }
    return cudaGetLastError();
}

// FP32 even-odd operator A (or A^+ = g5 A g5) on FP32 18-real links.
static cudaError_t apply_A_f32(wd_handle* h, const uint4* in, uint4* out, uint4* tmp, const uint4* le, const uint4* lo,
                               cudaStream_t s) {
    HopParams P{};
    P.g = h->g;
    P.nrhs = 1;
    P.parity = 1;
    P.links = lo;
    P.in = in;
    P.out = tmp;
    P.a = 1.0;
    cudaError_t e = Ops<float>::hop(18, EPI_H, RED_NONE, P, s);
    if (e != cudaSuccess) return e;
    P.parity = 0;
    P.links = le;
    P.in = tmp;
    P.out = out;
    P.y = in;
    P.a = -h->kappa * h->kappa;
    P.b = 1.0;
    return Ops<float>::hop(18, EPI_Y, RED_NONE, P, s);
}

int ptc_grad(wd_handle* h, int n, const float* v, const float* y, double mu, double* loss, cudaStream_t s) {
    PtcBufs B;
    int rc = ptc_bufs(h, &B);
    if (rc != WD_OK) return rc;
    const uint4 *le, *lo;
    if ((rc = ensure_links(h, WD_FP32, 18, &le, &lo)) != WD_OK) return rc;
    const Geom& g = h->g;
    const size_t vb = vec_bytes(h, WD_FP32);
    const long long nf = (long long)g.Vh * 24;
    const long long hvs = (long long)spinor_units(WD_FP32) * g.Vh;
    uint4* H = ptc_hidden(h, WD_FP32, "ptc.h32");
    uint4* GH = ptc_hidden(h, WD_FP32, "ptc.gh32");
    float* m = (float*)workspace(h, "ptc.vm", vb);
    float* e1 = (float*)workspace(h, "ptc.ve1", vb);
    float* am = (float*)workspace(h, "ptc.vam", vb);
    float* t1 = (float*)workspace(h, "ptc.vt1", vb);
    float* t2 = (float*)workspace(h, "ptc.vt2", vb);
    float* gv = (float*)workspace(h, "ptc.vg", vb);
    double* dots = (double*)workspace(h, "ptc.dots", sizeof(double) * (4 * n + 4));
    const int blk = 256, gv1 = grid_for((int)std::min<long long>(nf, 1LL << 30), blk);
    const dim3 wgrid(std::max(1, num_sms() / 8), 9, PTC_C);
    // per-block partial sums of the dot products and of the weight gradients, summed in block order
    double* dpart = (double*)workspace(h, "ptc.dpart", sizeof(double) * gv1);
    float* wpart = (float*)workspace(h, "ptc.wpart", sizeof(float) * 32 * wgrid.x * 9 * PTC_C);
    if (!H || !GH || !m || !e1 || !am || !t1 || !t2 || !gv || !dots || !dpart || !wpart)
        return fail(h, WD_ERR_CUDA, "out of device memory");
    auto dot = [&](const float* a, const float* b, double* out) {
        k_f32_dot<<<gv1, blk, 0, s>>>(nf, a, b, dpart);
        k_sum_partials<<<1, 32, 0, s>>>(gv1, dpart, out);
    };
    int* err = ptc_err(h);
    if (!err) return fail(h, WD_ERR_CUDA, "out of device memory");
    WD_CUDA(h, cudaMemsetAsync(err, 0, sizeof(int), s));
    WD_CUDA(h, cudaMemsetAsync(dots, 0, sizeof(double) * (4 * n + 4), s));
    WD_CUDA(h, cudaMemsetAsync(B.grad, 0, sizeof(float) * PTC_FLOATS, s));
    // input norms first: the gradient coefficients need them
    for (int i = 0; i < n; ++i) {
        const float* vi = v + i * nf;
        const float* yi = y + i * nf;
        dot(vi, vi, dots + 4 * i);
        dot(yi, yi, dots + 4 * i + 1);
    }
    std::vector<double> hd(4 * n + 4);
    WD_CUDA(h, cudaMemcpyAsync(hd.data(), dots, sizeof(double) * (4 * n + 4), cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaStreamSynchronize(s));
    const int gx = grid_for(g.Vh, 128);
    k_ptc_adjoint_weights<<<1, 256, 0, s>>>(B.weff + 2 * PTC_LAYER, B.wadj);
    for (int i = 0; i < n; ++i) {
        const float* vi = v + i * nf;
        const float* yi = y + i * nf;
        const double nv = hd[4 * i], ny = hd[4 * i + 1];
        // forward: m = M v (hidden H kept for the weight gradient of layer 2)
        WD_CUDA(h, ptc_apply_raw(h, WD_FP32, (const uint4*)vi, (uint4*)m, H, B.weff, le, lo, s, nullptr));
        // e1 = m - y ; e2 = A m - v ; A^+ e2 = g5 A g5 e2
        k_f32_lincomb<<<gv1, blk, 0, s>>>(nf, 1.f, m, -1.f, yi, e1);
        WD_CUDA(h, apply_A_f32(h, (const uint4*)m, (uint4*)am, (uint4*)t1, le, lo, s));
        k_f32_lincomb<<<gv1, blk, 0, s>>>(nf, 1.f, am, -1.f, vi, am);
        dot(e1, e1, dots + 4 * i + 2);
        dot(am, am, dots + 4 * i + 3);
        k_gamma5_f32<<<gx, 128, 0, s>>>(g.Vh, (const uint4*)am, (uint4*)t2);
        WD_CUDA(h, apply_A_f32(h, (const uint4*)t2, (uint4*)gv, (uint4*)t1, le, lo, s));
        k_gamma5_f32<<<gx, 128, 0, s>>>(g.Vh, (const uint4*)gv, (uint4*)t2);
        // g = 2 e1 / |y|^2 + 2 mu A^+ e2 / |v|^2  (= 2 dL/dconj(m))
        k_f32_lincomb<<<gv1, blk, 0, s>>>(nf, (float)(2.0 / ny), e1, (float)(2.0 * mu / nv), t2, gv);
        // layer 2: dW2 += sum g (x) conj(T_k H_c) ; g_H = adjoint network of layer 2 applied to g
        k_ptc_wgrad<float, 18><<<wgrid, 128, 0, s>>>(g, 0, (const uint4*)gv, H, hvs, le, lo, wpart);
        k_ptc_wgrad_sum<<<9 * PTC_C, 32, 0, s>>>(wgrid.x, wpart, B.grad + 2 * PTC_LAYER);
        WD_CUDA(h, ptc_fanout_f32(h, (const uint4*)gv, GH, hvs, le, lo, B.wadj, s, err));
        // layer 1: dW1 += sum g_H,c (x) conj(T_k v)
        k_ptc_wgrad<float, 18><<<wgrid, 128, 0, s>>>(g, 1, GH, (const uint4*)vi, hvs, le, lo, wpart);
        k_ptc_wgrad_sum<<<9 * PTC_C, 32, 0, s>>>(wgrid.x, wpart, B.grad);
        WD_CUDA(h, cudaGetLastError());
    }
    WD_CUDA(h, cudaMemcpyAsync(hd.data(), dots, sizeof(double) * (4 * n + 4), cudaMemcpyDeviceToHost, s));
    int herr = 0;
    WD_CUDA(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, WD_ERR_TIMEOUT, "wd_precond_grad: a bounded tensor-core wait gave up");
    double L = 0.0;
    for (int i = 0; i < n; ++i) L += hd[4 * i + 2] / hd[4 * i + 1] + mu * hd[4 * i + 3] / hd[4 * i];
    if (loss) *loss = L;
    return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_precond_set(wd_handle* h, const float* w, int where) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!w || (where != WD_HOST && where != WD_DEVICE)) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_set: bad argument");
    PtcBufs B;
    int rc = ptc_bufs(h, &B);
    if (rc != WD_OK) return rc;
    const size_t nb = sizeof(float) * PTC_FLOATS;
    WD_CUDA(h, cudaMemcpy(B.w, w, nb, where == WD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    WD_CUDA(h, cudaMemset(B.m, 0, nb));
    WD_CUDA(h, cudaMemset(B.v, 0, nb));
    k_round_bf16<<<(PTC_FLOATS + 255) / 256, 256>>>(PTC_FLOATS, B.w, B.weff);
    k_ptc_collapse<<<6, 256>>>(B.weff, B.V);
    WD_CUDA(h, cudaGetLastError());
    WD_CUDA(h, cudaDeviceSynchronize());
    h->have_precond = true;
    h->adam_t = 0;
    return WD_OK;
}

extern "C" int wd_precond_get(wd_handle* h, float* w, int where) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!w || (where != WD_HOST && where != WD_DEVICE)) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_get: bad argument");
    if (!h->have_precond) return fail(h, WD_ERR_INVALID_ARG, "no preconditioner weights loaded");
    PtcBufs B;
    int rc = ptc_bufs(h, &B);
    if (rc != WD_OK) return rc;
    WD_CUDA(h, cudaMemcpy(w, B.w, sizeof(float) * PTC_FLOATS,
                          where == WD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice));
    return WD_OK;
}

extern "C" int wd_precond_apply(wd_handle* h, int prec, const void* in, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if ((prec != WD_FP32 && prec != WD_FP16) || !in || !out || in == out)
        return fail(h, WD_ERR_INVALID_ARG, "wd_precond_apply: bad argument");
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_apply: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    if (!h->have_precond) return fail(h, WD_ERR_INVALID_ARG, "no preconditioner weights loaded");
    PtcBufs B;
    int rc = ptc_bufs(h, &B);
    if (rc != WD_OK) return rc;
    const uint4 *le, *lo;
    if ((rc = ensure_links(h, prec, prec == WD_FP32 ? 18 : 12, &le, &lo)) != WD_OK) return rc;
    uint4* PHI = ptc_phi(h, prec);
    int* err = ptc_err(h);
    if (!PHI || !err) return fail(h, WD_ERR_CUDA, "out of device memory");
    cudaStream_t s = (cudaStream_t)stream;
    WD_CUDA(h, cudaMemsetAsync(err, 0, sizeof(int), s));
    WD_CUDA(h, ptc_apply_m(h, prec, (const uint4*)in, (uint4*)out, PHI, B.V, le, lo, s, nullptr, err));
    int herr = 0;
    WD_CUDA(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaStreamSynchronize(s));
    if (herr) return fail(h, WD_ERR_TIMEOUT, "wd_precond_apply: a bounded tensor-core wait gave up");
    return WD_OK;
}

extern "C" int wd_precond_grad(wd_handle* h, int n, const float* v, const float* y, double mu, float* grad,
                               double* loss, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (n < 1 || !v || !y || !(mu >= 0)) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_grad: bad argument");
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_grad: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    if (!h->have_precond) return fail(h, WD_ERR_INVALID_ARG, "no preconditioner weights loaded");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ptc_grad(h, n, v, y, mu, loss, s);
    if (rc != WD_OK) return rc;
    if (grad) {
        PtcBufs B;
        if ((rc = ptc_bufs(h, &B)) != WD_OK) return rc;
        WD_CUDA(h, cudaMemcpyAsync(grad, B.grad, sizeof(float) * PTC_FLOATS, cudaMemcpyDeviceToDevice, s));
        WD_CUDA(h, cudaStreamSynchronize(s));
    }
    return WD_OK;
}

extern "C" int wd_precond_train_step(wd_handle* h, int n, const float* v, const float* y, double mu, double lr,
                                     double* loss, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (n < 1 || !v || !y || !(mu >= 0) || !(lr > 0)) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_train_step: bad argument");
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_train_step: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    if (!h->have_precond) return fail(h, WD_ERR_INVALID_ARG, "no preconditioner weights loaded");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ptc_grad(h, n, v, y, mu, loss, s);
    if (rc != WD_OK) return rc;
    PtcBufs B;
    if ((rc = ptc_bufs(h, &B)) != WD_OK) return rc;
    h->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->adam_t), c2 = 1.f - std::pow(b2, (float)h->adam_t);
    k_adam<<<(PTC_FLOATS + 255) / 256, 256, 0, s>>>(PTC_FLOATS, B.w, B.grad, B.m, B.v, (float)lr, b1, b2, 1e-8f, c1,
                                                   c2, B.weff);
    k_ptc_collapse<<<6, 256, 0, s>>>(B.weff, B.V);
    WD_CUDA(h, cudaGetLastError());
    WD_CUDA(h, cudaStreamSynchronize(s));
    return WD_OK;
}

// The same weights given as BF16 values in host memory: each widened exactly to FP32 (the BF16 bits are the
// high half of the FP32 word) and loaded as the FP32 masters.
extern "C" int wd_precond_load(wd_handle* h, const void* weights_bf16, size_t n) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!weights_bf16 || n != (size_t)PTC_FLOATS)
        return fail(h, WD_ERR_INVALID_ARG, "wd_precond_load: n must be WD_PRECOND_FLOATS");
    const unsigned short* b = static_cast<const unsigned short*>(weights_bf16);
    std::vector<float> w(PTC_FLOATS);
    for (size_t i = 0; i < n; ++i) {
        const unsigned u = (unsigned)b[i] << 16;
        std::memcpy(&w[i], &u, sizeof u);
    }
    return wd_precond_set(h, w.data(), WD_HOST);
}

// `steps` Adam steps on the same samples; *loss receives the loss before the last step.
extern "C" int wd_precond_train(wd_handle* h, int steps, int n, const float* v, const float* y, double mu, double lr,
                                double* loss, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (steps < 1) return fail(h, WD_ERR_INVALID_ARG, "wd_precond_train: steps must be at least 1");
    double l = 0.0;
    for (int i = 0; i < steps; ++i) {
        const int rc = wd_precond_train_step(h, n, v, y, mu, lr, &l, stream);
        if (rc != WD_OK) return rc;
    }
    if (loss) *loss = l;
    return WD_OK;
}

namespace wd {
// Collapsed spin weights of the loaded network (device), or null when none are loaded.
const float2* ptc_collapsed(wd_handle* h) {
    if (!h->have_precond) return nullptr;
    PtcBufs B;
    if (ptc_bufs(h, &B) != WD_OK) return nullptr;
    return B.V;
}

// Intermediate fields of the collapsed M for the FP16 solve path.
uint4* ptc_phi16(wd_handle* h) { return ptc_phi(h, WD_FP16); }
}  // namespace wd
