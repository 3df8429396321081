// Fused vector kernels of the rescaled BiCGStab (Alg. 4/5) and of the
// refinement loop (Alg. 2/3), plus layout conversions. Every kernel streams
// packed parity vectors unit by unit; reductions keep per-thread partial
// sums in the arithmetic type (FP32 for low-precision storage, as in the
// paper's Fig. 3) and combine threads, blocks and the grid in FP64.
#pragma once

#include <cstring>

#include "kernels.h"

namespace wd {

// out = (a + ib) * v for one complex element pair
template <typename C>
__device__ __forceinline__ void cscale_add(C& or_, C& oi, C ar, C ai, C vr, C vi) {
    or_ += ar * vr - ai * vi;
    oi += ar * vi + ai * vr;
}

#define GRID_STRIDE(h, n) for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < (n); h += gridDim.x * blockDim.x)

// Per right-hand-side loop over the sites of a batched launch.
#define RHS_LOOP(h, n) for (int h = sl.b * blockDim.x + threadIdx.x; h < (n); h += sl.nb * blockDim.x)

// The streaming kernels below work unit by unit (a unit = 16 bytes: 8 halves,
// 4 floats or 2 doubles of one site) and issue every load of a chunk of units
// -- for FP16/BF16 storage the whole site, for two sites per thread -- before
// the first store, so that a thread keeps all its reads in flight at once
// (the vectors may alias as far as the compiler knows, so a load written after
// a store would wait for it). The arithmetic per element and the order of
// every per-thread sum are those of a site-by-site loop.
template <typename T> struct Stream {
    static constexpr int N = Unit<T>::N;                     // reals per unit
    static constexpr int SU = 24 / N;                        // units per site
    static constexpr int CH = SU < 3 ? SU : 3;               // units per chunk
    static constexpr int SITES = sizeof(T) == 2 ? 2 : 1;     // sites per thread and step
};

// Round the N values of one unit to storage, write it (flushing stored
// subnormals with ftz) and replace the values by the stored ones.
template <typename T>
__device__ __forceinline__ void store_unit(uint4* v, size_t off, typename Unit<T>::C (&c)[Unit<T>::N], bool ftz) {
    uint4 w = Unit<T>::put(c);
    if (ftz) w = Unit<T>::flush(w);
    v[off] = w;
#pragma unroll
    for (int i = 0; i < Unit<T>::N; ++i) c[i] = Unit<T>::get(w, i);
}

// Per right-hand-side loop over groups of S sites of a batched launch: sites h, h + step, ... h + (S-1) step.
#define RHS_LOOP_S(h, n, S) for (int h = sl.b * blockDim.x + threadIdx.x; h < (n); h += (S) * sl.nb * blockDim.x)

// p := r (first iteration) or cP p - cV v + r
template <typename T>
__global__ void __launch_bounds__(256) k_pupdate(int n, int nrhs, long long vs, uint4* p, const uint4* v,
                                                 const uint4* r, const SolverState* sts) {
    pdl_begin();
    typedef typename Unit<T>::C C;
    typedef Stream<T> ST;
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_INNER)) return;
    const long long ro = sl.rhs * vs;
    p += ro; v += ro; r += ro;
    const bool first = st->first, ftz = st->ftz;
    const C pr = (C)st->cP[0], pi = (C)st->cP[1], vr = (C)st->cV[0], vi = (C)st->cV[1];
    const int step = sl.nb * blockDim.x;
    RHS_LOOP_S(h0, n, ST::SITES) {
#pragma unroll
        for (int u0 = 0; u0 < ST::SU; u0 += ST::CH) {
            uint4 ur[ST::SITES][ST::CH], up[ST::SITES][ST::CH], uv[ST::SITES][ST::CH];
#pragma unroll
            for (int q = 0; q < ST::SITES; ++q) {
                const int h = h0 + q * step;
                if (h >= n) continue;
#pragma unroll
                for (int c = 0; c < ST::CH; ++c) {
                    const size_t off = (size_t)(u0 + c) * n + h;
                    ur[q][c] = __ldg(r + off);
                    if (!first) {
                        up[q][c] = __ldg(p + off);
                        uv[q][c] = __ldg(v + off);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < ST::SITES; ++q) {
                const int h = h0 + q * step;
                if (h >= n) continue;
#pragma unroll
                for (int c = 0; c < ST::CH; ++c) {
                    C o[ST::N];
#pragma unroll
                    for (int i = 0; i < ST::N / 2; ++i) {
                        C a = Unit<T>::get(ur[q][c], 2 * i), b = Unit<T>::get(ur[q][c], 2 * i + 1);
                        if (!first) {
                            cscale_add(a, b, pr, pi, Unit<T>::get(up[q][c], 2 * i), Unit<T>::get(up[q][c], 2 * i + 1));
                            cscale_add(a, b, -vr, -vi, Unit<T>::get(uv[q][c], 2 * i),
                                       Unit<T>::get(uv[q][c], 2 * i + 1));
                        }
                        o[2 * i] = a;
                        o[2 * i + 1] = b;
                    }
                    store_unit<T>(p, (size_t)(u0 + c) * n + h, o, ftz);
                }
            }
        }
    }
}

// r := r - alpha v
template <typename T>
__global__ void __launch_bounds__(256) k_supdate(int n, int nrhs, long long vs, uint4* r, const uint4* v,
                                                 const SolverState* sts) {
    pdl_begin();
    typedef typename Unit<T>::C C;
    typedef Stream<T> ST;
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_INNER)) return;
    const long long o = sl.rhs * vs;
    r += o; v += o;
    const bool ftz = st->ftz;
    const C ar = (C)-st->alpha[0], ai = (C)-st->alpha[1];
    const int step = sl.nb * blockDim.x;
    RHS_LOOP_S(h0, n, ST::SITES) {
#pragma unroll
        for (int u0 = 0; u0 < ST::SU; u0 += ST::CH) {
            uint4 ur[ST::SITES][ST::CH], uv[ST::SITES][ST::CH];
#pragma unroll
            for (int q = 0; q < ST::SITES; ++q) {
                const int h = h0 + q * step;
                if (h >= n) continue;
#pragma unroll
                for (int c = 0; c < ST::CH; ++c) {
                    const size_t off = (size_t)(u0 + c) * n + h;
                    ur[q][c] = __ldg(r + off);
                    uv[q][c] = __ldg(v + off);
                }
            }
#pragma unroll
            for (int q = 0; q < ST::SITES; ++q) {
                const int h = h0 + q * step;
                if (h >= n) continue;
#pragma unroll
                for (int c = 0; c < ST::CH; ++c) {
                    C rr[ST::N];
#pragma unroll
                    for (int i = 0; i < ST::N; ++i) rr[i] = Unit<T>::get(ur[q][c], i);
#pragma unroll
                    for (int i = 0; i < ST::N / 2; ++i)
                        cscale_add(rr[2 * i], rr[2 * i + 1], ar, ai, Unit<T>::get(uv[q][c], 2 * i),
                                   Unit<T>::get(uv[q][c], 2 * i + 1));
                    store_unit<T>(r, (size_t)(u0 + c) * n + h, rr, ftz);
                }
            }
        }
    }
}

// x := x + cXr r + cXp p  (x := cXr r + cXp p on the first iteration)
// r := r - omega t, and with XR_FUSED stored as c (r - omega t), c = sigma / g~
// the rescaling factor from the predicted norm (ST_OMEGA)
// sums: XR_PLAIN  |r|^2, |x|^2, (r*, r)
//       XR_NORMS  |r|^2, |x|^2            (a separate k_scale pass follows)
//       XR_FUSED  |r|^2 (before scaling), |r_stored|^2, (r*, r_stored)
// One site per thread and step: six vectors of a site are in flight at once.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_xr(int n, int nrhs, long long vs, uint4* x, uint4* r, const uint4* p,
                                            const uint4* t, const uint4* rstar, const uint4* xr_src,
                                            const uint4* xp_src, SolverState* sts, RedCtx rc) {
    pdl_begin();
    typedef typename Unit<T>::C C;
    typedef Stream<T> ST;
    constexpr bool WITH_RS = MODE != XR_NORMS;
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_INNER)) return;
    const long long o = sl.rhs * vs;
    x += o; r += o; p += o; t += o; rstar += o;
    // x-update sources: r and p, or M r and M p with a right preconditioner
    const uint4* xsr = xr_src ? xr_src + o : r;
    const uint4* xsp = xp_src ? xp_src + o : p;
    const bool first = st->first, ftz = st->ftz, pre = xr_src != nullptr;
    const C xr_r = (C)st->cXr[0], xr_i = (C)st->cXr[1], xp_r = (C)st->cXp[0], xp_i = (C)st->cXp[1];
    const C om_r = (C)-st->omega[0], om_i = (C)-st->omega[1];
    const C gs = MODE == XR_FUSED ? (C)st->gam_tmp : (C)1;
    C s_r2 = 0, s_x2 = 0, s_re = 0, s_im = 0;
    RHS_LOOP(h, n) {
#pragma unroll
        for (int u0 = 0; u0 < ST::SU; u0 += ST::CH) {
            uint4 ur[ST::CH], up[ST::CH], ux[ST::CH], ut[ST::CH], urs[ST::CH], urr[ST::CH];
#pragma unroll
            for (int c = 0; c < ST::CH; ++c) {
                const size_t off = (size_t)(u0 + c) * n + h;
                ur[c] = __ldg(xsr + off);
                up[c] = __ldg(xsp + off);
                if (!first) ux[c] = __ldg(x + off);
                ut[c] = __ldg(t + off);
                if (pre) urr[c] = __ldg(r + off);
                if constexpr (WITH_RS) urs[c] = __ldg(rstar + off);
            }
#pragma unroll
            for (int c = 0; c < ST::CH; ++c) {
                const size_t off = (size_t)(u0 + c) * n + h;
                C xx[ST::N], rr[ST::N];
#pragma unroll
                for (int i = 0; i < ST::N; ++i) {
                    xx[i] = first ? (C)0 : Unit<T>::get(ux[c], i);
                    rr[i] = Unit<T>::get(ur[c], i);
                }
#pragma unroll
                for (int i = 0; i < ST::N / 2; ++i) {
                    cscale_add(xx[2 * i], xx[2 * i + 1], xr_r, xr_i, rr[2 * i], rr[2 * i + 1]);
                    cscale_add(xx[2 * i], xx[2 * i + 1], xp_r, xp_i, Unit<T>::get(up[c], 2 * i),
                               Unit<T>::get(up[c], 2 * i + 1));
                }
                store_unit<T>(x, off, xx, ftz);
                if (pre) {
#pragma unroll
                    for (int i = 0; i < ST::N; ++i) rr[i] = Unit<T>::get(urr[c], i);
                }
#pragma unroll
                for (int i = 0; i < ST::N / 2; ++i)
                    cscale_add(rr[2 * i], rr[2 * i + 1], om_r, om_i, Unit<T>::get(ut[c], 2 * i),
                               Unit<T>::get(ut[c], 2 * i + 1));
#pragma unroll
                for (int i = 0; i < ST::N; ++i) s_r2 += rr[i] * rr[i];
                if constexpr (MODE == XR_FUSED) {
#pragma unroll
                    for (int i = 0; i < ST::N; ++i) rr[i] *= gs;
                }
                store_unit<T>(r, off, rr, ftz);
                if constexpr (MODE == XR_FUSED) {
#pragma unroll
                    for (int i = 0; i < ST::N; ++i) s_x2 += rr[i] * rr[i];      // |r_stored|^2
                } else {
#pragma unroll
                    for (int i = 0; i < ST::N; ++i) s_x2 += xx[i] * xx[i];
                }
                if constexpr (WITH_RS) {
#pragma unroll
                    for (int i = 0; i < ST::N / 2; ++i) {
                        const C rsr = Unit<T>::get(urs[c], 2 * i), rsi = Unit<T>::get(urs[c], 2 * i + 1);
                        s_re += rsr * rr[2 * i] + rsi * rr[2 * i + 1];
                        s_im += rsr * rr[2 * i + 1] - rsi * rr[2 * i];
                    }
                }
            }
        }
    }
    const C v[4] = {s_r2, s_x2, s_re, s_im};
    grid_reduce<4, ST_RFUSED>(v, rc, sl);
}

// r := (sigma / g) r, and x := lambda x when rescaling the solution (Alg. 5)
// sums: |r|^2, (r*, r)
template <typename T>
__global__ void __launch_bounds__(256) k_scale(int n, int nrhs, long long vs, uint4* r, uint4* x,
                                               const uint4* rstar, SolverState* sts, RedCtx rc) {
    pdl_begin();
    typedef typename Unit<T>::C C;
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_INNER)) return;
    const long long o = sl.rhs * vs;
    r += o; x += o; rstar += o;
    const C gs = (C)st->gam_tmp;
    const bool resx = st->rescale_x;
    const C lam = (C)st->lam;
    C s_r2 = 0, s_re = 0, s_im = 0;
    RHS_LOOP(h, n) {
        C rr[24], rs[24];
        load_spinor<T>(r, n, h, rr);
#pragma unroll
        for (int i = 0; i < 24; ++i) rr[i] *= gs;
        store_spinor<T>(r, n, h, rr, st->ftz);
        load_spinor<T>(rstar, n, h, rs);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            s_r2 += rr[2 * i] * rr[2 * i] + rr[2 * i + 1] * rr[2 * i + 1];
            s_re += rs[2 * i] * rr[2 * i] + rs[2 * i + 1] * rr[2 * i + 1];
            s_im += rs[2 * i] * rr[2 * i + 1] - rs[2 * i + 1] * rr[2 * i];
        }
        if (resx) {
            C xx[24];
            load_spinor<T>(x, n, h, xx);
#pragma unroll
            for (int i = 0; i < 24; ++i) xx[i] *= lam;
            store_spinor<T>(x, n, h, xx, st->ftz);
        }
    }
    const C v[3] = {s_r2, s_re, s_im};
    grid_reduce<3, ST_END>(v, rc, sl);
}

// Rescale the FP64 outer residual and demote it (Alg. 3, first lines):
// y~ = low_prec((s / |r|) r) written to r and r*; sums |single(y~)|^2 and the
// count of nonzero reals. The product is formed in FP64 and rounded once (round_f64).
// Round-to-nearest-even of an FP64 value to a binary format with MB fraction
// bits and EB exponent bits, from the IEEE-754 bit fields in integer
// arithmetic (the FP64 pipe of this GPU is ~70x narrower than the integer
// one): the fraction is cut after MB bits and rounded on the dropped bits (a
// carry into the exponent field is the correct result, up to infinity);
// below the normal range the significand is shifted to units of the smallest
// subnormal and rounded the same way; beyond it the result is infinity;
// infinities stay, NaNs become quiet NaNs. Returns the bit pattern.
template <int MB, int EB>
__host__ __device__ __forceinline__ unsigned round_f64(double x) {
    constexpr int BIAS = (1 << (EB - 1)) - 1, EMIN = 1 - BIAS;
    constexpr unsigned EXP_ALL = (1u << EB) - 1u;
#ifdef __CUDA_ARCH__
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    memcpy(&u, &x, sizeof u);
#endif
    const unsigned sign = (unsigned)(u >> 63) << (EB + MB);
    const int e = (int)((u >> 52) & 0x7FF);
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return sign | (EXP_ALL << MB) | (m ? (1u << (MB - 1)) : 0u);
    const int E = e - 1023;
    if (E > BIAS) return sign | (EXP_ALL << MB);
    unsigned long long q, r, half;
    unsigned v;
    if (E >= EMIN) {
        q = m >> (52 - MB);
        r = m & ((1ull << (52 - MB)) - 1);
        half = 1ull << (51 - MB);
        v = sign | ((unsigned)(E + BIAS) << MB) | (unsigned)q;
    } else {
        const int sh = 52 + EMIN - MB - E;   // value / (smallest subnormal) = significand >> sh
        if (sh > 53) return sign;             // below half the smallest subnormal
        const unsigned long long mf = (1ull << 52) | m;
        q = mf >> sh;
        r = mf & ((1ull << sh) - 1);
        half = 1ull << (sh - 1);
        v = sign | (unsigned)q;
    }
    if (r > half || (r == half && (q & 1ull))) v += 1u;
    return v;
}

template <typename T>
__device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __uint_as_float(round_f64<23, 8>(v)); }
template <> __device__ __forceinline__ __half from_double<__half>(double v) {
    return __ushort_as_half((unsigned short)round_f64<10, 5>(v));
}
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v) {
    return __ushort_as_bfloat16((unsigned short)round_f64<7, 8>(v));
}

// Exact widening of a storage value to the arithmetic type C of its unit.
template <typename T>
__device__ __forceinline__ typename Unit<T>::C widen(T v);
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }
template <> __device__ __forceinline__ float widen<float>(float v) { return v; }
template <> __device__ __forceinline__ float widen<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Exact float -> double from the IEEE-754 bit fields on the integer pipe (the
// FP64 pipe of this GPU is ~70x narrower than the FP32 and integer ones):
// sign kept, exponent rebased from 127 to 1023, mantissa shifted into the top
// of the 52-bit field; float subnormals are normalised, infinities and NaNs
// keep the all-ones exponent.
__host__ __device__ __forceinline__ double f32_to_f64(float a) {
#ifdef __CUDA_ARCH__
    const unsigned u = __float_as_uint(a);
#else
    unsigned u;
    memcpy(&u, &a, sizeof u);
#endif
    const unsigned sgn = u & 0x80000000u;
    unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned hi, lo;
    if (e == 0u && m == 0u) {
        hi = sgn;
        lo = 0u;
    } else {
        if (e == 0u) {   // subnormal: value = m 2^-149, normalised on its leading bit p
#ifdef __CUDA_ARCH__
            const int p = 31 - __clz((int)m);
#else
            const int p = 31 - __builtin_clz(m);
#endif
            m = (m << (23 - p)) & 0x7FFFFFu;
            e = (unsigned)(p - 149 + 1023);
        } else {
            e = e == 0xFFu ? 0x7FFu : e + (1023u - 127u);
        }
        hi = sgn | (e << 20) | (m >> 3);
        lo = m << 29;
    }
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const unsigned long long bits = ((unsigned long long)hi << 32) | lo;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
#endif
}

template <typename T>
__device__ __forceinline__ double to_double(T v);
template <> __device__ __forceinline__ double to_double<double>(double v) { return v; }
template <> __device__ __forceinline__ double to_double<float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double to_double<__half>(__half v) { return (double)__half2float(v); }
template <> __device__ __forceinline__ double to_double<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// Element e (0..23) of site h of a packed vector of T, as a typed pointer.
template <typename T>
__device__ __forceinline__ T* elem_ptr(uint4* base, int stride, int h, int e) {
    constexpr int N = Unit<T>::N;
    return reinterpret_cast<T*>(base + (size_t)(e / N) * stride + h) + (e % N);
}
template <typename T>
__device__ __forceinline__ const T* elem_ptr(const uint4* base, int stride, int h, int e) {
    constexpr int N = Unit<T>::N;
    return reinterpret_cast<const T*>(base + (size_t)(e / N) * stride + h) + (e % N);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rescale_in(int n, int nrhs, long long vs, long long vs64, const uint4* r64,
                                                    uint4* r, uint4* rstar, int ftz, SolverState* sts, RedCtx rc) {
    typedef typename Unit<T>::C C;
    constexpr int N = Unit<T>::N;
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_OUTER)) return;
    r64 += sl.rhs * vs64;
    r += sl.rhs * vs;
    rstar += sl.rhs * vs;
    const double f = st->s / st->rnorm;
    const C tiny = (C)(sizeof(T) == 2 ? 6.103515625e-05 : 1.1754943508222875e-38);   // flush threshold
    C s_n2 = 0;
    int nz = 0;
    RHS_LOOP(h, n) {
        double src[24];
        load_spinor<double>(r64, n, h, src);
        alignas(16) T y[24];
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            // the product in FP64, rounded once to T; the rest on the exact widened value in C (a 16-bit
            // value's square is exact in FP32, a float's is rounded once, as a double square cast to float)
            T v = from_double<T>(f * src[i]);
            C dv = widen<T>(v);
            if (ftz && fabs(dv) < tiny) {
                v = from_double<T>(0.0);
                dv = 0;
            }
            y[i] = v;
            s_n2 += dv * dv;
            nz += dv != (C)0 ? 1 : 0;
        }
#pragma unroll
        for (int u = 0; u < 24 / N; ++u) {
            uint4 w = *reinterpret_cast<const uint4*>(&y[u * N]);
            r[(size_t)u * n + h] = w;
            rstar[(size_t)u * n + h] = w;
        }
    }
    const C v[2] = {s_n2, (C)nz};   // a per-thread count (at most 24 per site) is exact in FP32
    grid_reduce<2, ST_INIT>(v, rc, sl);
}

// out = M in site by site (M: 12 x 12 complex blocks of one parity, shared by all right-hand sides)
template <typename T>
__global__ void __launch_bounds__(256) k_apply_mat(int n, int nrhs, long long vs, const uint4* mat, const uint4* in,
                                                   uint4* out) {
    typedef typename Unit<T>::C C;
    const Slice sl = slice_of(nrhs);
    in += sl.rhs * vs;
    out += sl.rhs * vs;
    RHS_LOOP(h, n) {
        C v[24], o[24];
        load_spinor<T>(in, n, h, v);
        mat_mul<T>(mat, n, h, v, o);
        store_spinor<T>(out, n, h, o);
    }
}

// Blocks of storage T from FP64 blocks: 288 reals per site, element e of site h
// in unit e / N of the block array (units n apart), as for spinors.
template <typename T>
__global__ void __launch_bounds__(256) k_mat_from64(int n, const uint4* src, uint4* dst) {
    typedef typename Unit<T>::C C;
    constexpr int N = Unit<T>::N;
    GRID_STRIDE(h, n) {
#pragma unroll 1
        for (int u = 0; u < 288 / N; ++u) {
            C v[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int e = u * N + i;
                const uint4 w = src[(size_t)(e / 2) * n + h];
                v[i] = (C)Unit<double>::get(w, e % 2);
            }
            dst[(size_t)u * n + h] = Unit<T>::put(v);
        }
    }
}

// out = M in site by site with M in the chiral packing
template <typename T>
__global__ void __launch_bounds__(256) k_apply_chiral(int n, int nrhs, long long vs, const uint4* mat,
                                                      const uint4* in, uint4* out) {
    typedef typename Unit<T>::C C;
    const Slice sl = slice_of(nrhs);
    in += sl.rhs * vs;
    out += sl.rhs * vs;
    RHS_LOOP(h, n) {
        C v[24], o[24];
        load_spinor<T>(in, n, h, v);
        mat_mul_chiral<T>(mat, n, h, v, o);
        store_spinor<T>(out, n, h, o);
    }
}

// Chiral packing of full FP64 blocks M (144 complex per site, element (i, j)
// in unit 12 i + j): S_-/+ (k a, k' b) = (M[k a][k' b] -/+ M[k a][k'+2 b]
// -/+ M[k+2 a][k' b] + M[k+2 a][k'+2 b]) / 4 with spin-colour index 3 s + a,
// stored as described at mat_mul_chiral (block + first).
template <typename T>
__global__ void __launch_bounds__(128) k_chiral_from64(int n, const uint4* src, uint4* dst) {
    typedef typename Unit<T>::C C;
    constexpr int N = Unit<T>::N;
    GRID_STRIDE(h, n) {
        for (int c = 0; c < 2; ++c) {
            const double sg = c == 0 ? -1.0 : 1.0;
            double blk[40];
            for (int i = 0; i < 40; ++i) blk[i] = 0.0;
            int q = 6;
            for (int i = 0; i < 6; ++i)
                for (int j = i; j < 6; ++j) {
                    const int k = i / 3, a = i % 3, kk = j / 3, b = j % 3;
                    const int r0 = 3 * k + a, r2 = 3 * (k + 2) + a, c0 = 3 * kk + b, c2 = 3 * (kk + 2) + b;
                    double re = 0.0, im = 0.0;
                    const int idx[4] = {12 * r0 + c0, 12 * r0 + c2, 12 * r2 + c0, 12 * r2 + c2};
                    const double f[4] = {1.0, sg, sg, 1.0};
                    for (int t = 0; t < 4; ++t) {
                        const uint4 w = src[(size_t)idx[t] * n + h];
                        re += f[t] * Unit<double>::get(w, 0);
                        im += f[t] * Unit<double>::get(w, 1);
                    }
                    if (i == j) {
                        blk[i] = 0.25 * re;
                    } else {
                        blk[q] = 0.25 * re;
                        blk[q + 1] = 0.25 * im;
                        q += 2;
                    }
                }
            for (int u = 0; u < 40 / N; ++u) {
                C v[N];
                for (int e = 0; e < N; ++e) v[e] = (C)blk[u * N + e];
                dst[(size_t)(c * (40 / N) + u) * n + h] = Unit<T>::put(v);
            }
        }
    }
}

// x64 += (|r| / s^) * double(t~) / lambda'   (Alg. 3 correction; Alg. 2: s^ -> s)
template <typename T>
__global__ void __launch_bounds__(256) k_correct(int n, int nrhs, long long vs, long long vs64, uint4* x64,
                                                 const uint4* xt, const SolverState* sts) {
    const Slice sl = slice_of(nrhs);
    const SolverState* st = sts + sl.rhs;
    if (guarded(st, GUARD_OUTER)) return;
    x64 += sl.rhs * vs64;
    xt += sl.rhs * vs;
    const double f = st->rnorm / (st->use_shat ? st->shat : st->s) / st->lambda_p;
    RHS_LOOP(h, n) {
#pragma unroll
        for (int e = 0; e < 24; ++e) {
            double* xp = elem_ptr<double>(x64, n, h, e);
            if constexpr (sizeof(T) == 8)
                *xp += f * to_double<T>(*elem_ptr<T>(xt, n, h, e));
            else   // the FP32 widening of a 16- or 32-bit value, made double on the integer pipe
                *xp += f * f32_to_f64((float)widen<T>(*elem_ptr<T>(xt, n, h, e)));
        }
    }
}

// sum |v|^2 over a packed vector; stage as given (ST_ACC / ST_ACC_SET / ST_OUTER)
template <typename T>
__global__ void __launch_bounds__(256) k_norm2(int n, int nrhs, long long vs, const uint4* v, RedCtx rc, int gk) {
    typedef typename Unit<T>::C C;
    const Slice sl = slice_of(nrhs);
    if (guarded(rc.st ? rc.st + sl.rhs : nullptr, gk)) return;
    v += sl.rhs * vs;
    C s = 0;
    RHS_LOOP(h, n) {
        C a[24];
        load_spinor<T>(v, n, h, a);
#pragma unroll
        for (int i = 0; i < 24; ++i) s += a[i] * a[i];
    }
    const C d[1] = {s};
    grid_reduce<1>(d, rc, sl);
}

// Eq. 5 and the odd half of the true residual from one odd hop t = H_oe xi_e:
//   xi_o = eta_o + kappa t,   sum over sites of |eta_o - xi_o + kappa t|^2
// (the stage as given). The residual's own H_oe xi_e is this t: the same
// kernel on the same input gives the same bits, so it is not recomputed.
template <typename T>
__global__ void __launch_bounds__(256) k_odd_reconstruct(int n, int nrhs, long long vs, double kappa, const uint4* eta,
                                                         const uint4* t, uint4* xo, RedCtx rc) {
    typedef typename Unit<T>::C C;
    const Slice sl = slice_of(nrhs);
    eta += sl.rhs * vs;
    t += sl.rhs * vs;
    xo += sl.rhs * vs;
    const C k = (C)kappa;
    C s2 = 0;
    RHS_LOOP(h, n) {
        C e[24], tv[24], o[24];
        load_spinor<T>(eta, n, h, e);
        load_spinor<T>(t, n, h, tv);
#pragma unroll
        for (int i = 0; i < 24; ++i) o[i] = fma(k, tv[i], e[i]);
        store_spinor<T>(xo, n, h, o, false);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            const C r = fma(k, tv[i], e[i] - o[i]);
            s2 += r * r;
        }
    }
    const C d[1] = {s2};
    grid_reduce<1>(d, rc, sl);
}

// lex FP64 (24 doubles per site) -> packed parity vector of T
template <typename T>
__global__ void k_pack(Geom g, int parity, const double* lex, uint4* out) {
    GRID_STRIDE(h, g.Vh) {
        const int s = lex_of(g, parity, h);
#pragma unroll
        for (int e = 0; e < 24; ++e) *elem_ptr<T>(out, g.Vh, h, e) = from_double<T>(lex[(size_t)s * 24 + e]);
    }
}

template <typename T>
__global__ void k_unpack(Geom g, int parity, const uint4* in, double* lex) {
    GRID_STRIDE(h, g.Vh) {
        const int s = lex_of(g, parity, h);
#pragma unroll
        for (int e = 0; e < 24; ++e) {
            const T v = *elem_ptr<T>(in, g.Vh, h, e);
            if constexpr (sizeof(T) == 8)
                lex[(size_t)s * 24 + e] = to_double<T>(v);
            else
                lex[(size_t)s * 24 + e] = f32_to_f64((float)widen<T>(v));
        }
    }
}

// Gathered links of output parity p (see hop_impl.cuh) from FP64 lex links.
template <typename T, int R>
__global__ void k_build_links(Geom g, int parity, const double* U, uint4* out) {
    constexpr int N = Unit<T>::N;
    const int V = 2 * g.Vh;
    GRID_STRIDE(h, g.Vh) {
        const int s = lex_of(g, parity, h);
        int c[4];
        c[0] = s % g.L[0];
        c[1] = (s / g.L[0]) % g.L[1];
        c[2] = (s / (g.L[0] * g.L[1])) % g.L[2];
        c[3] = s / (g.L[0] * g.L[1] * g.L[2]);
        for (int mu = 0; mu < 4; ++mu) {
            int cm[4] = {c[0], c[1], c[2], c[3]};
            cm[mu] = (c[mu] + g.L[mu] - 1) % g.L[mu];
            const int sm = cm[0] + g.L[0] * (cm[1] + g.L[1] * (cm[2] + g.L[2] * cm[3]));
            const double* uf = U + ((size_t)mu * V + s) * 18;
            const double* ub = U + ((size_t)mu * V + sm) * 18;
            // a direction split across processes: the hops that leave the sub-lattice are
            // remote, and their links are stored as zeros (the face terms are added apart)
            const bool split = (g.part >> mu) & 1u;
            const bool zf = split && c[mu] == g.L[mu] - 1, zb = split && c[mu] == 0;
            for (int e = 0; e < R; ++e) {
                // forward: U_mu(x)[a][b]; backward: (U_mu(x-mu)^+)[a][b] = conj(U_mu(x-mu)[b][a])
                const int a = e / 6, b = (e % 6) / 2, im = e & 1;
                const double vf = zf ? 0.0 : uf[e];
                const double vb = zb ? 0.0 : (im ? -ub[2 * (3 * b + a) + 1] : ub[2 * (3 * b + a)]);
                const int ef = (2 * mu) * R + e, eb = (2 * mu + 1) * R + e;
                reinterpret_cast<T*>(out + (size_t)(ef / N) * g.Vh + h)[ef % N] = from_double<T>(vf);
                reinterpret_cast<T*>(out + (size_t)(eb / N) * g.Vh + h)[eb % N] = from_double<T>(vb);
            }
        }
    }
}

#undef GRID_STRIDE
#undef RHS_LOOP

}  // namespace wd
