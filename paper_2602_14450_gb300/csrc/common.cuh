// Shared device-side definitions of the Wilson-Dirac solver library.
//
// Storage: every packed field (spinor parity vector, gathered links) is an
// array of 16-byte units with the site index fastest: unit u of site h is at
// units[u * stride + h]. A unit holds 2 doubles, 4 floats, or 8 halves /
// bfloat16s. Arithmetic type C is float for FP32/FP16/BF16 storage and
// double for FP64 storage.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wd {

// ------------------------------------------------------------ timeline ---
//
// Timeline build (-DWD_TIMELINE, python -m paper_2602_14450_gb300.timeline):
// each block of a kernel that opens with pdl_begin() records its kernel site,
// grid size, SM, arrival, start (after the wait for the preceding kernel) and
// end on the global timer; the last block of each grid reduction records the
// times of its phases. The default build contains none of it.
#ifdef WD_TIMELINE
namespace tl {
static __device__ unsigned long long* blocks = nullptr;   // [0] records, then 4 words per block
static __device__ unsigned long long* phases = nullptr;   // [0] records, then 10 words per reduction
constexpr unsigned long long BLOCK_CAP = 1ull << 24, PHASE_CAP = 1ull << 20;
__device__ __forceinline__ unsigned long long now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned sm() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
// 16-bit hash of a source file's base name (the same function in timeline.py)
__host__ __device__ constexpr unsigned name_hash(const char* c, unsigned h = 7u) {
    return *c ? name_hash(c + 1, h * 31u + (unsigned char)*c) : (h & 0xFFFFu);
}
__host__ __device__ constexpr const char* base_name(const char* p, const char* last) {
    return *p ? base_name(p + 1, *p == '/' ? p + 1 : last) : last;
}
struct Scope {
    unsigned long long arrive, start;
    unsigned site;
    __device__ Scope(unsigned site_, unsigned long long arrive_) : arrive(arrive_), start(now()), site(site_) {}
    __device__ ~Scope() {
        if (threadIdx.x != 0 || !blocks) return;
        const unsigned long long end = now();
        const unsigned long long r = atomicAdd(blocks, 1ull);
        if (r >= BLOCK_CAP) return;
        unsigned long long* q = blocks + 1 + 4 * r;
        q[0] = ((unsigned long long)site << 32) | ((unsigned long long)gridDim.x << 8) | sm();
        q[1] = arrive;
        q[2] = start;
        q[3] = end;
    }
};
__device__ __forceinline__ void record_phases(int stage, int nsum, const unsigned long long (&t)[8]) {
    if (!phases) return;
    const unsigned long long end = now();
    const unsigned long long r = atomicAdd(phases, 1ull);
    if (r >= PHASE_CAP) return;
    unsigned long long* q = phases + 1 + 10 * r;
    q[0] = ((unsigned long long)stage << 32) | (unsigned)nsum;
    for (int i = 0; i < 8; ++i) q[1 + i] = t[i];
    q[9] = end;
}
// Points the recording buffers of this translation unit's kernels at b and p.
static int set_buffers(void* b, void* p) {
    if (cudaMemcpyToSymbol(blocks, &b, sizeof(b)) != cudaSuccess) return 1;
    return cudaMemcpyToSymbol(phases, &p, sizeof(p)) != cudaSuccess ? 1 : 0;
}
void register_unit(int (*setter)(void*, void*));   // api.cu: the setters of all translation units
static const int registered = (register_unit(set_buffers), 0);
}  // namespace tl
#define WD_TL_DECL unsigned long long wd_tl_t[8] = {};
#define WD_TL_T(i) wd_tl_t[i] = ::wd::tl::now();
#define WD_TL_PHASES(stage, nsum) ::wd::tl::record_phases(stage, nsum, wd_tl_t);
#else
#define WD_TL_DECL
#define WD_TL_T(i)
#define WD_TL_PHASES(stage, nsum)
#endif

// ---------------------------------------------------------------- storage ---

template <typename T> struct Unit;

template <> struct Unit<double> {
    typedef double C;
    static constexpr int N = 2;
    __device__ __forceinline__ static uint4 flush(const uint4& u) { return u; }   // FP64 storage is not flushed
    __device__ __forceinline__ static C get(const uint4& u, int i) {
        return i == 0 ? __hiloint2double((int)u.y, (int)u.x) : __hiloint2double((int)u.w, (int)u.z);
    }
    __device__ __forceinline__ static uint4 put(const C* v) {
        uint4 u;
        u.x = (unsigned)__double2loint(v[0]);
        u.y = (unsigned)__double2hiint(v[0]);
        u.z = (unsigned)__double2loint(v[1]);
        u.w = (unsigned)__double2hiint(v[1]);
        return u;
    }
};

template <> struct Unit<float> {
    typedef float C;
    static constexpr int N = 4;
    // Stored subnormals (exponent field 0) become +0.
    __device__ __forceinline__ static unsigned fw(unsigned w) { return (w & 0x7F800000u) ? w : 0u; }
    __device__ __forceinline__ static uint4 flush(const uint4& u) { return make_uint4(fw(u.x), fw(u.y), fw(u.z), fw(u.w)); }
    __device__ __forceinline__ static C get(const uint4& u, int i) {
        unsigned w = i == 0 ? u.x : i == 1 ? u.y : i == 2 ? u.z : u.w;
        return __uint_as_float(w);
    }
    __device__ __forceinline__ static uint4 put(const C* v) {
        return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
    }
};

__device__ __forceinline__ unsigned word_of(const uint4& u, int w) {
    return w == 0 ? u.x : w == 1 ? u.y : w == 2 ? u.z : u.w;
}

// Both 16-bit lanes of a word with subnormal values (exponent field 0) set to +0.
__device__ __forceinline__ unsigned flush16(unsigned w, unsigned emask) {
    return ((w & emask) ? (w & 0xFFFFu) : 0u) | ((w & (emask << 16)) ? (w & 0xFFFF0000u) : 0u);
}

template <> struct Unit<__half> {
    typedef float C;
    static constexpr int N = 8;
    __device__ __forceinline__ static uint4 flush(const uint4& u) {
        return make_uint4(flush16(u.x, 0x7C00u), flush16(u.y, 0x7C00u), flush16(u.z, 0x7C00u), flush16(u.w, 0x7C00u));
    }
    __device__ __forceinline__ static C get(const uint4& u, int i) {
        unsigned w = word_of(u, i >> 1);
        __half2 h = *reinterpret_cast<__half2*>(&w);
        return (i & 1) ? __high2float(h) : __low2float(h);
    }
    __device__ __forceinline__ static uint4 put(const C* v) {
        uint4 u;
        __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        __half2 c = __floats2half2_rn(v[4], v[5]), d = __floats2half2_rn(v[6], v[7]);
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        u.z = *reinterpret_cast<unsigned*>(&c);
        u.w = *reinterpret_cast<unsigned*>(&d);
        return u;
    }
};

template <> struct Unit<__nv_bfloat16> {
    typedef float C;
    static constexpr int N = 8;
    __device__ __forceinline__ static uint4 flush(const uint4& u) {
        return make_uint4(flush16(u.x, 0x7F80u), flush16(u.y, 0x7F80u), flush16(u.z, 0x7F80u), flush16(u.w, 0x7F80u));
    }
    __device__ __forceinline__ static C get(const uint4& u, int i) {
        unsigned w = word_of(u, i >> 1);
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
        return (i & 1) ? __high2float(h) : __low2float(h);
    }
    __device__ __forceinline__ static uint4 put(const C* v) {
        uint4 u;
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
        __nv_bfloat162 c = __floats2bfloat162_rn(v[4], v[5]), d = __floats2bfloat162_rn(v[6], v[7]);
        u.x = *reinterpret_cast<unsigned*>(&a);
        u.y = *reinterpret_cast<unsigned*>(&b);
        u.z = *reinterpret_cast<unsigned*>(&c);
        u.w = *reinterpret_cast<unsigned*>(&d);
        return u;
    }
};

// Units of one site of a spinor (24 reals).
template <typename T> struct Spinor {
    static constexpr int UNITS = 24 / Unit<T>::N;
};

// Load the 24 reals of site h (order: spin, colour, re/im).
template <typename T>
__device__ __forceinline__ void load_spinor(const uint4* __restrict__ v, int stride, int h,
                                            typename Unit<T>::C (&s)[24]) {
    constexpr int N = Unit<T>::N;
#pragma unroll
    for (int u = 0; u < 24 / N; ++u) {
        uint4 w = __ldg(v + (size_t)u * stride + h);
#pragma unroll
        for (int i = 0; i < N; ++i) s[u * N + i] = Unit<T>::get(w, i);
    }
}

// Load as stored by a previous kernel of the same launch chain (coherent load).
template <typename T>
__device__ __forceinline__ void load_spinor_cg(const uint4* v, int stride, int h, typename Unit<T>::C (&s)[24]) {
    constexpr int N = Unit<T>::N;
#pragma unroll
    for (int u = 0; u < 24 / N; ++u) {
        uint4 w = __ldcg(v + (size_t)u * stride + h);
#pragma unroll
        for (int i = 0; i < N; ++i) s[u * N + i] = Unit<T>::get(w, i);
    }
}

// Round to storage and write; `s` is overwritten with the stored values so
// that reductions see exactly what later kernels will read. With ftz, stored
// subnormal values are flushed to zero after the rounding.
template <typename T>
__device__ __forceinline__ void store_spinor(uint4* v, int stride, int h, typename Unit<T>::C (&s)[24],
                                             bool ftz = false) {
    constexpr int N = Unit<T>::N;
#pragma unroll
    for (int u = 0; u < 24 / N; ++u) {
        uint4 w = Unit<T>::put(&s[u * N]);
        if (ftz) w = Unit<T>::flush(w);
        v[(size_t)u * stride + h] = w;
#pragma unroll
        for (int i = 0; i < N; ++i) s[u * N + i] = Unit<T>::get(w, i);
    }
}

// out = M v for the site-local 12 x 12 complex matrix M of site h (row-major,
// spin-colour index 3 s + a, the layout of the clover blocks): row i is the
// 24 reals of units i * SU .. i * SU + SU - 1 (SU = units of a spinor).
template <typename T>
__device__ __forceinline__ void mat_mul(const uint4* __restrict__ mat, int stride, int h,
                                        const typename Unit<T>::C (&v)[24], typename Unit<T>::C (&out)[24]) {
    typedef typename Unit<T>::C C;
    constexpr int SU = 24 / Unit<T>::N;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        C row[24];
        load_spinor<T>(mat + (size_t)i * SU * stride, stride, h, row);
        C re = row[0] * v[0], im = row[0] * v[1];
        re = fma(-row[1], v[1], re);
        im = fma(row[1], v[0], im);
#pragma unroll
        for (int j = 1; j < 12; ++j) {
            re = fma(row[2 * j], v[2 * j], re);
            re = fma(-row[2 * j + 1], v[2 * j + 1], re);
            im = fma(row[2 * j], v[2 * j + 1], im);
            im = fma(row[2 * j + 1], v[2 * j], im);
        }
        out[2 * i] = re;
        out[2 * i + 1] = im;
    }
}

// Clover blocks commute with gamma_5 = -[[0, 1], [1, 0]] (spin blocks of this
// basis), so in the chiral combinations chi_+/- = psi_{0,1} -/+ psi_{2,3} of
// the spin pairs they split into two Hermitian 6 x 6 blocks S_+, S_-. Stored
// per site: for c = +, - the real diagonal (6 reals), the upper triangle
// (i < j, row by row: 15 complex) and 4 zeros, 40 reals per block and 80 per
// site (units of 16 bytes as for spinors). With S = T' M T'^T / 4 (T' the
// unnormalised chiral map), M v = T'^T S T' v:
//   out_{0,1} = o_+ + o_-,  out_{2,3} = o_- - o_+,  o_c = S_c chi_c.
template <typename T>
__device__ __forceinline__ void chiral_block_mul(const uint4* __restrict__ mat, int stride, int h, int unit0,
                                                 const typename Unit<T>::C (&x)[12], typename Unit<T>::C (&o)[12]) {
    typedef typename Unit<T>::C C;
    constexpr int N = Unit<T>::N;
    constexpr int UB = 40 / N;   // units per block
    C m[40];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const uint4 w = __ldg(mat + (size_t)(unit0 + u) * stride + h);
#pragma unroll
        for (int i = 0; i < N; ++i) m[u * N + i] = Unit<T>::get(w, i);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        o[2 * i] = m[i] * x[2 * i];
        o[2 * i + 1] = m[i] * x[2 * i + 1];
    }
    int q = 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
            const C br = m[q], bi = m[q + 1];
            q += 2;
            // o_i += b x_j ; o_j += conj(b) x_i
            o[2 * i] = fma(br, x[2 * j], fma(-bi, x[2 * j + 1], o[2 * i]));
            o[2 * i + 1] = fma(br, x[2 * j + 1], fma(bi, x[2 * j], o[2 * i + 1]));
            o[2 * j] = fma(br, x[2 * i], fma(bi, x[2 * i + 1], o[2 * j]));
            o[2 * j + 1] = fma(br, x[2 * i + 1], fma(-bi, x[2 * i], o[2 * j + 1]));
        }
}

template <typename T>
__device__ __forceinline__ void mat_mul_chiral(const uint4* __restrict__ mat, int stride, int h,
                                               const typename Unit<T>::C (&v)[24], typename Unit<T>::C (&out)[24]) {
    typedef typename Unit<T>::C C;
    constexpr int UB = 40 / Unit<T>::N;
    C xp[12], xm[12], op[12], om[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) {   // spin pair (k, k + 2), colour: reals 6 k + 2 a + re/im
        xp[i] = v[i] - v[12 + i];
        xm[i] = v[i] + v[12 + i];
    }
    chiral_block_mul<T>(mat, stride, h, 0, xp, op);
    chiral_block_mul<T>(mat, stride, h, UB, xm, om);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        out[i] = op[i] + om[i];
        out[12 + i] = om[i] - op[i];
    }
}

// --------------------------------------------------------------- geometry ---

// Division of a non-negative int below 2^31 by a fixed divisor d in
// [1, 2^31) with one high multiply, one add and one shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// Sec. 4): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> l; the sum stays below 2^32 for n < 2^31.
struct FastDiv {
    unsigned m;
    int l;
    int d;
    __host__ void init(int divisor) {
        d = divisor;
        l = 0;
        while ((1u << l) < (unsigned)d) ++l;
        m = (unsigned)((((unsigned long long)1 << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1);
    }
    __device__ __forceinline__ int div(int n) const { return (int)((__umulhi(m, (unsigned)n) + (unsigned)n) >> l); }
};

struct Geom {
    int L[4];    // Lx, Ly, Lz, Lt
    int Lxh;     // Lx / 2
    int Vh;      // V / 2 (sites per parity)
    int bc[4];   // boundary phases, +1 or -1
    FastDiv fxh, fy, fz;   // division by Lxh, Ly, Lz
    unsigned part;         // bit mu: direction mu is split across processes (its wrapping hops are remote)
};

// Lexicographic index of site h on parity p.
__device__ __forceinline__ int lex_of(const Geom& g, int p, int h) {
    int row = g.fxh.div(h);
    int xh = h - row * g.Lxh;
    int r2 = g.fy.div(row);
    int y = row - r2 * g.L[1];
    int t = g.fz.div(r2);
    int z = r2 - t * g.L[2];
    int x = 2 * xh + ((p + y + z + t) & 1);
    return x + g.L[0] * row;
}

// Coordinates of site h on parity p.
struct Coord {
    int x, y, z, t, row;
};
__device__ __forceinline__ Coord coord_of(const Geom& g, int p, int h) {
    Coord c;
    c.row = g.fxh.div(h);
    const int xh = h - c.row * g.Lxh;
    const int r2 = g.fy.div(c.row);
    c.y = c.row - r2 * g.L[1];
    c.t = g.fz.div(r2);
    c.z = r2 - c.t * g.L[2];
    c.x = 2 * xh + ((p + c.y + c.z + c.t) & 1);
    return c;
}

// Site index (on the other parity) of the neighbour of site h in direction
// d = 2 mu (+mu) or 2 mu + 1 (-mu); *wrap says whether the hop wraps.
__device__ __forceinline__ int neighbour(const Geom& g, int h, const Coord& c, int d, bool* wrap) {
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int Lxh = g.Lxh;
    if (mu == 0) {
        const bool w = fwd ? (c.x == g.L[0] - 1) : (c.x == 0);
        *wrap = w;
        const int xn = fwd ? (w ? 0 : c.x + 1) : (w ? g.L[0] - 1 : c.x - 1);
        return c.row * Lxh + (xn >> 1);
    }
    const int coordv = mu == 1 ? c.y : mu == 2 ? c.z : c.t;
    const int L = g.L[mu];
    const int s = mu == 1 ? Lxh : mu == 2 ? Lxh * g.L[1] : Lxh * g.L[1] * g.L[2];
    const bool w = fwd ? (coordv == L - 1) : (coordv == 0);
    *wrap = w;
    return fwd ? (w ? h - (L - 1) * s : h + s) : (w ? h + (L - 1) * s : h - s);
}

// Neighbour sites of output site h on parity p; returns the mask of the
// directions d whose hop wraps around the lattice.
__device__ __forceinline__ unsigned site_neighbours(const Geom& g, int p, int h, int (&nbr)[8]) {
    const int Lxh = g.Lxh, Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    const int row = g.fxh.div(h);
    const int xh = h - row * Lxh;
    const int r2 = g.fy.div(row);
    const int y = row - r2 * Ly;
    const int t = g.fz.div(r2);
    const int z = r2 - t * Lz;
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int sy = Lxh, sz = Lxh * Ly, st = Lxh * Ly * Lz;
    const bool w0 = x == g.L[0] - 1, w1 = x == 0, w2 = y == Ly - 1, w3 = y == 0;
    const bool w4 = z == Lz - 1, w5 = z == 0, w6 = t == Lt - 1, w7 = t == 0;
    nbr[0] = row * Lxh + ((w0 ? 0 : x + 1) >> 1);
    nbr[1] = row * Lxh + ((w1 ? g.L[0] - 1 : x - 1) >> 1);
    nbr[2] = w2 ? h - (Ly - 1) * sy : h + sy;
    nbr[3] = w3 ? h + (Ly - 1) * sy : h - sy;
    nbr[4] = w4 ? h - (Lz - 1) * sz : h + sz;
    nbr[5] = w5 ? h + (Lz - 1) * sz : h - sz;
    nbr[6] = w6 ? h - (Lt - 1) * st : h + st;
    nbr[7] = w7 ? h + (Lt - 1) * st : h - st;
    return (unsigned)w0 | (unsigned)w1 << 1 | (unsigned)w2 << 2 | (unsigned)w3 << 3 | (unsigned)w4 << 4 |
           (unsigned)w5 << 5 | (unsigned)w6 << 6 | (unsigned)w7 << 7;
}

// ---------------------------------------------------------------- complex ---

template <typename C> struct cpx {
    C re, im;
};
template <typename C> __device__ __forceinline__ cpx<C> mk(C a, C b) { cpx<C> z; z.re = a; z.im = b; return z; }

// -------------------------------------------------------- solver scalars ---

// FP64 scalar state of one right-hand side (Alg. 4/5 and the Alg. 2/3 loop).
// Complex scalars are (re, im) pairs.
struct SolverState {
    double rho[2], rho_p[2];        // (r*, r) and rho'
    double alpha[2], alpha_p[2];    // alpha, alpha'
    double omega[2], omega_p[2];    // omega, omega'
    double cP[2], cV[2];            // p := cP p - cV v + r   (beta*gamma, beta*gamma*omega')
    double cXr[2], cXp[2];          // x += cXr r + cXp p     (lambda'/gamma' * (omega, alpha))
    double gamma_p;                 // gamma'
    double lambda_p;                // lambda'
    double lam;                     // lambda of this iteration (Alg. 5)
    double g;                       // |r| before rescaling
    double gam_tmp;                 // sigma / g, the factor applied to r
    double bnorm;                   // |b| of the inner system
    double res;                     // |r| / gamma'
    double sigma, sigma_lambda, eps, omega0;
    int recalc, rescale_x, max_matvecs, scale_pass;
    int fused_scale;                // r is rescaled inside its update (k_xr, XR_FUSED) with the predicted norm
    int iter, matvecs, first, done, status;
    int skip;                       // right-hand side finished: every kernel leaves it alone
    int ftz;                        // flush subnormal values of every low-precision store
    double* hist;                   // optional device log: (matvecs, |r|/gamma') per inner iteration
    int hist_cap;                   // iterations the log holds
    // refinement (outer) scalars
    double rnorm;                   // |b^ - A x| of the FP64 outer residual
    double shat;                    // |single(y~)|
    double s;                       // target norm of y
    int use_shat;
    double acc;                     // accumulator for multi-kernel norms
    long long nonzeros;             // nonzero reals of the last rescaled input
};

enum Stage {
    ST_NONE = 0,
    ST_INIT = 1,     // sums: |y~|^2, nonzeros      -> start an inner solve
    ST_ALPHA = 2,    // sums: (r*, v)               -> alpha
    ST_OMEGA = 3,    // sums: (t,s), (t,t), (s,s)   -> omega (omega_0 prescription)
    ST_RNORM = 4,    // sums: |r|^2, |x|^2, (r*, r) -> g, sigma/g, lambda (or end of iteration)
    ST_END = 5,      // sums: |r_st|^2, (r*, r_st)  -> gamma, beta, convergence
    ST_OUTER = 6,    // sums: |r64|^2               -> outer residual norm
    ST_ACC = 7,      // sums: x                     -> acc += x
    ST_ACC_SET = 8,  // sums: x                     -> acc  = x
    ST_RFUSED = 9    // sums: |r|^2, |r_st|^2, (r*, r_st) -> gamma, beta, convergence (rescaling fused)
};

// Status codes (mirror enum wd_status of wd.h).
enum { S_OK = 0, S_NOT_CONVERGED = 4, S_BREAKDOWN = 5, S_NONFINITE = 6 };

__host__ __device__ __forceinline__ void stop(SolverState* st, int status) {
    st->done = 1;
    if (st->status == S_OK) st->status = status;
}

// The stages below run in one thread at the end of a reducing kernel, on
// the critical path between two kernels. FP64 is slow on this GPU (64 cycles
// for a dependent add or FMA, ~560 for a division or a square root), so each
// stage reads the state it needs into registers before any branch (one
// round trip to memory), divides once where a reciprocal serves several
// products, and stores only what it changes.

// 1 / sqrt(x): the device's reciprocal square root, the plain quotient in host builds of these stages.
__host__ __device__ __forceinline__ double rsqrt_d(double x) {
#ifdef __CUDA_ARCH__
    return rsqrt(x);
#else
    return 1.0 / sqrt(x);
#endif
}

// End of a BiCGStab iteration (Alg. 4 last lines): gamma known, r stored.
// rn2 = |r_stored|^2, rs = (r*, r_stored).
__host__ __device__ __forceinline__ void end_iteration(SolverState* st, double gamma, double rn2, const double* rs) {
    const double rho0 = st->rho[0], rho1 = st->rho[1];
    const double al0 = st->alpha[0], al1 = st->alpha[1], om0 = st->omega[0], om1 = st->omega[1];
    const double gp = st->gamma_p * gamma;
    const double lp = st->rescale_x ? st->lambda_p * st->lam : st->lambda_p;
    const int iter = st->iter + 1, matvecs = st->matvecs + 2, status = st->status;
    const double eps_b = st->eps * st->bnorm;
    const int max_mv = st->max_matvecs, hist_cap = st->hist_cap;
    double* hist = st->hist;
    // rho' = gamma * rho, gamma' *= gamma, alpha' = alpha, omega' = omega, rho = (r*, r)
    const double rp0 = gamma * rho0, rp1 = gamma * rho1;
    // beta = rho alpha' / (rho' omega'); the p-update folds the gamma of p and v: cP = gamma beta, cV = cP omega'.
    // With rho' = gamma rho_old, cP = rho alpha' / (rho_old omega'): formed without waiting for gamma.
    const double n0 = rs[0] * al0 - rs[1] * al1, n1 = rs[0] * al1 + rs[1] * al0;
    const double d0 = rho0 * om0 - rho1 * om1, d1 = rho0 * om1 + rho1 * om0;
    const double id = 1.0 / (d0 * d0 + d1 * d1);
    const double cp0 = (n0 * d0 + n1 * d1) * id, cp1 = (n1 * d0 - n0 * d1) * id;
    const double cv0 = cp0 * om0 - cp1 * om1, cv1 = cp0 * om1 + cp1 * om0;
    const double res = sqrt(rn2) / gp;
    st->rho_p[0] = rp0; st->rho_p[1] = rp1;
    st->gamma_p = gp;
    st->alpha_p[0] = al0; st->alpha_p[1] = al1;
    st->omega_p[0] = om0; st->omega_p[1] = om1;
    st->lambda_p = lp;
    st->rho[0] = rs[0]; st->rho[1] = rs[1];
    st->cP[0] = cp0; st->cP[1] = cp1;
    st->cV[0] = cv0; st->cV[1] = cv1;
    st->iter = iter;
    st->matvecs = matvecs;
    st->first = 0;
    st->res = res;
    if (hist && iter <= hist_cap) {
        hist[2 * (iter - 1)] = (double)matvecs;
        hist[2 * (iter - 1) + 1] = res;
    }
    int stop_with = -1;
    if (!(isfinite(res) && isfinite(cp0) && isfinite(cp1) && isfinite(cv0) && isfinite(cv1) && isfinite(gp)))
        stop_with = S_NONFINITE;
    else if (res <= eps_b)
        stop_with = S_OK;
    else if (matvecs >= max_mv)
        stop_with = S_NOT_CONVERGED;
    else if ((d0 == 0.0 && d1 == 0.0) || gamma == 0.0)   // rho' omega' = 0
        stop_with = S_BREAKDOWN;
    if (stop_with >= 0) {
        st->done = 1;
        if (status == S_OK) st->status = stop_with;
    }
}

// Scalar work done by the last block of a reducing kernel, one thread: one
// function per stage; a kernel inlines the stage it expects (its code then
// follows the final sum in instruction memory) and calls the shared
// out-of-line dispatcher for any other.
template <int STAGE> __host__ __device__ __forceinline__ void stage_fn(const double* s, SolverState* st) {}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_INIT>(const double* s, SolverState* st) {
    double n2 = s[0];
    st->shat = sqrt(n2);
    st->nonzeros = (long long)s[1];
    st->bnorm = st->use_shat ? st->shat : st->s;
    // Alg. 4 start: r = r* = y~, p = v = 0, rho' = |r|^2, omega' = alpha' = gamma' = 1
    st->rho[0] = n2; st->rho[1] = 0;
    st->rho_p[0] = n2; st->rho_p[1] = 0;
    st->alpha_p[0] = 1; st->alpha_p[1] = 0;
    st->omega_p[0] = 1; st->omega_p[1] = 0;
    st->cP[0] = st->cP[1] = st->cV[0] = st->cV[1] = 0;
    st->gamma_p = 1;
    st->lambda_p = 1;
    st->lam = 1;
    st->iter = 0;
    st->matvecs = 0;
    st->first = 1;
    st->done = 0;
    st->status = S_OK;
    st->res = st->shat;
    if (!(n2 > 0) || !isfinite(n2)) stop(st, isfinite(n2) ? S_OK : S_NONFINITE);
}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_ALPHA>(const double* s, SolverState* st) {   // alpha = rho / (r*, v)
    const double rho0 = st->rho[0], rho1 = st->rho[1];
    const double v0 = s[0], v1 = s[1];
    if (!(isfinite(v0) && isfinite(v1))) { stop(st, S_NONFINITE); return; }
    if (v0 == 0.0 && v1 == 0.0) { stop(st, S_BREAKDOWN); return; }
    const double id = 1.0 / (v0 * v0 + v1 * v1);
    st->alpha[0] = (rho0 * v0 + rho1 * v1) * id;
    st->alpha[1] = (rho1 * v0 - rho0 * v1) * id;
}

// omega = (t, s) / (t, t) with the omega_0 prescription; with fused rescaling also the factor for r
template <> __host__ __device__ __forceinline__ void stage_fn<ST_OMEGA>(const double* s, SolverState* st) {
    const double omega0 = st->omega0, sigma = st->sigma;
    const double c = st->lambda_p / st->gamma_p;
    const double al0 = st->alpha[0], al1 = st->alpha[1];
    const int fused = st->fused_scale;
    const double ts0 = s[0], ts1 = s[1], tt = s[2], ss = s[3];
    if (!(isfinite(tt) && isfinite(ss) && isfinite(ts0) && isfinite(ts1))) { stop(st, S_NONFINITE); return; }
    if (tt == 0.0) { stop(st, S_BREAKDOWN); return; }
    const double itt = 1.0 / tt;
    // |omega^| = |(t, s)| / (|t| |s|) below omega0: omega *= omega0 / |omega^| (compared squared; the factor
    // is formed alongside 1 / (t, t) and selected)
    const double a2 = ts0 * ts0 + ts1 * ts1, q = tt * ss;
    const double fs = omega0 * sqrt(q / a2);
    const double f = (omega0 > 0.0 && a2 > 0.0 && a2 < omega0 * omega0 * q) ? fs : 1.0;
    const double om0 = ts0 * itt * f, om1 = ts1 * itt * f;
    st->omega[0] = om0;
    st->omega[1] = om1;
    if (fused) {
        // |s - omega t|^2 = (s,s) - 2 Re(conj(omega) (t,s)) + |omega|^2 (t,t), floored against
        // cancellation; the factor sigma / g~ rescales r as it is stored
        double r2 = ss - 2.0 * (om0 * ts0 + om1 * ts1) + (om0 * om0 + om1 * om1) * tt;
        r2 = fmax(r2, 1e-12 * ss);
        const double gt = sigma * rsqrt_d(r2);
        st->gam_tmp = gt;
        if (!isfinite(gt)) { stop(st, S_NONFINITE); return; }
    }
    st->cXr[0] = c * om0;
    st->cXr[1] = c * om1;
    st->cXp[0] = c * al0;
    st->cXp[1] = c * al1;
}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_RNORM>(const double* s, SolverState* st) {
    double r2 = s[0], x2 = s[1];
    double rs[2] = {s[2], s[3]};
    st->g = sqrt(r2);
    if (st->rescale_x) st->lam = st->sigma_lambda / sqrt(x2);
    if (st->scale_pass) {
        st->gam_tmp = st->sigma > 0.0 ? st->sigma / st->g : 1.0;
        if (!isfinite(st->gam_tmp) || (st->rescale_x && !isfinite(st->lam))) stop(st, S_NONFINITE);
    } else {
        end_iteration(st, 1.0, r2, rs);
    }
}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_END>(const double* s, SolverState* st) {
    double rn2 = s[0];
    double rs[2] = {s[1], s[2]};
    double gamma = st->sigma > 0.0 ? (st->recalc ? sqrt(rn2) / st->g : st->gam_tmp) : 1.0;
    end_iteration(st, gamma, rn2, rs);
}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_RFUSED>(const double* s, SolverState* st) {
    const int recalc = st->recalc;
    const double gt = st->gam_tmp;
    const double r2 = s[0], rn2 = s[1];
    const double rs[2] = {s[2], s[3]};
    const double g = sqrt(r2);
    st->g = g;
    double gamma = recalc ? sqrt(rn2) / g : gt;
    if (r2 == 0.0) gamma = 1.0;   // r = 0 exactly: nothing was scaled, the solve has converged
    end_iteration(st, gamma, rn2, rs);
}

template <> __host__ __device__ __forceinline__ void stage_fn<ST_OUTER>(const double* s, SolverState* st) { st->rnorm = sqrt(s[0]); }

template <> __host__ __device__ __forceinline__ void stage_fn<ST_ACC>(const double* s, SolverState* st) { st->acc += s[0]; }

template <> __host__ __device__ __forceinline__ void stage_fn<ST_ACC_SET>(const double* s, SolverState* st) { st->acc = s[0]; }

static __host__ __device__ __noinline__ void run_stage(int stage, const double* s, SolverState* st) {
    switch (stage) {
    case ST_INIT: stage_fn<ST_INIT>(s, st); break;
    case ST_ALPHA: stage_fn<ST_ALPHA>(s, st); break;
    case ST_OMEGA: stage_fn<ST_OMEGA>(s, st); break;
    case ST_RNORM: stage_fn<ST_RNORM>(s, st); break;
    case ST_END: stage_fn<ST_END>(s, st); break;
    case ST_RFUSED: stage_fn<ST_RFUSED>(s, st); break;
    case ST_OUTER: stage_fn<ST_OUTER>(s, st); break;
    case ST_ACC: stage_fn<ST_ACC>(s, st); break;
    case ST_ACC_SET: stage_fn<ST_ACC_SET>(s, st); break;
    default: break;
    }
}

template <int HINT>
__device__ __forceinline__ void run_stage_hinted(int stage, const double* s, SolverState* st) {
    if (HINT != ST_NONE && stage == HINT)
        stage_fn<HINT>(s, st);
    else
        run_stage(stage, s, st);
}

// ----------------------------------------------------------- reductions ---

// Context of a reducing kernel: each block writes its partial sums; the
// last block to finish (ticket) adds them in block order (deterministic),
// runs the scalar stage and re-arms the ticket. Arrays are indexed by the
// right-hand side: partials[rhs][block][sum] (RED_STRIDE doubles per rhs),
// ticket[rhs], st[rhs].
struct RedCtx {
    double* partials;
    unsigned* ticket;    // zero between kernels
    SolverState* st;
    int stage;
};

// Partial-sum slots per right-hand side (blocks x sums).
constexpr int RED_STRIDE = 8192 * 4;

// A launch serves `nrhs` right-hand sides: block b works for rhs b % nrhs as
// its (b / nrhs)-th block, so blocks that run together share site blocks
// (and therefore links) across right-hand sides.
struct Slice {
    int rhs, b, nb;
};
__device__ __forceinline__ Slice slice_of(int nrhs) {
    Slice s;
    s.rhs = blockIdx.x % nrhs;
    s.b = blockIdx.x / nrhs;
    s.nb = gridDim.x / nrhs;
    return s;
}

template <int NSUM>
__device__ __forceinline__ void warp_sum(double (&v)[NSUM]) {
#pragma unroll
    for (int k = 0; k < NSUM; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
}

// Sum v over the block; the result is valid in thread 0. FP64 additions are
// slow on this GPU (64 cycles of latency each), so the second level adds the
// few warp sums one after the other instead of another five-step shuffle.
template <int NSUM>
__device__ __forceinline__ void block_sum(double (&v)[NSUM]) {
    __shared__ double sh[NSUM][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_sum<NSUM>(v);
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NSUM; ++k) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) v[k] += sh[k][w];
        }
    }
}

// The ticket of a grid reduction: an add with acquire-release semantics at GPU
// scope. Its release orders the block's partial-sum stores before it; its
// acquire, with the barrier that follows, orders the last block's loads of
// all partial sums (from L2) after every other block's release. The ticket is
// re-armed with a plain store: the next kernel sees it after this one ends.
__device__ __forceinline__ unsigned ticket_add(unsigned* t) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(t) : "memory");
    return old;
}

// Reduce v over the sl.nb blocks that serve right-hand side sl.rhs (HINT: the
// scalar stage the calling kernel expects to run). The last block adds the partial sums with all its threads (each thread loads its
// eight next partials before adding them, so the loads overlap), then sums
// over the block; FP64 arithmetic is shared by the SM's warps, so spreading it
// over the block's warps matters more than its latency.
template <int NSUM, int HINT = ST_NONE>
__device__ __forceinline__ void grid_reduce(const double (&vin)[NSUM], const RedCtx& rc, const Slice& sl) {
    __shared__ unsigned is_last;
    WD_TL_DECL
    WD_TL_T(0)
    double* part = rc.partials + (size_t)sl.rhs * RED_STRIDE;
    unsigned* ticket = rc.ticket + sl.rhs;
    double v[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; ++k) v[k] = vin[k];
    block_sum<NSUM>(v);
    WD_TL_T(1)
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NSUM; ++k) part[(size_t)sl.b * NSUM + k] = v[k];
        WD_TL_T(2)
        is_last = (ticket_add(ticket) == (unsigned)sl.nb - 1) ? 1u : 0u;
        WD_TL_T(3)
    }
    __syncthreads();
    if (!is_last) return;
    WD_TL_T(4)
    double acc[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; ++k) acc[k] = 0.0;
    const int nt = blockDim.x;
    for (int b0 = threadIdx.x; b0 < sl.nb; b0 += 8 * nt) {
        double t[8][NSUM];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int b = b0 + i * nt;
#pragma unroll
            for (int k = 0; k < NSUM; ++k) t[i][k] = b < sl.nb ? __ldcg(part + (size_t)b * NSUM + k) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 0; k < NSUM; ++k) acc[k] += t[i][k];
    }
    WD_TL_T(5)
    block_sum<NSUM>(acc);
    if (threadIdx.x == 0) {
        WD_TL_T(6)
        if (rc.st) run_stage_hinted<HINT>(rc.stage, acc, rc.st + sl.rhs);
        WD_TL_T(7)
        *ticket = 0u;
        WD_TL_PHASES(rc.stage, NSUM)
    }
}

// Double-float reduction of FP32 per-thread partial sums. The partial sums of
// the low-precision kernels are FP32; their block and grid sums are carried
// as pairs (hi, lo) of FP32 numbers whose exact sum is the value, with the
// error-free additions below, which run on the FP32 pipe (the FP64 pipe of this
// GPU takes ~19 cycles per warp instruction per SM, and FP64 shuffle trees over
// a block's warps made the reductions a visible share of every reducing
// kernel). A pair carries ~48 significant bits, more than the FP32 partials it
// adds; the order of the additions is fixed, so results are reproducible.
struct F2 {
    float hi, lo;
};
// Round-to-nearest FP32 add and subtract, never contracted or reassociated
// (host versions for the host-side tests of these sums).
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float s = a + b;
    return s;
#endif
}
__host__ __device__ __forceinline__ float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float s = a - b;
    return s;
#endif
}
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e == a + b exactly in round-to-nearest.
__host__ __device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = add_rn(a, b);
    const float bb = sub_rn(s, a);
    const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
    return {s, e};
}
// Fast2Sum (Dekker 1971): exact when |a| >= |b|.
__host__ __device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = add_rn(a, b);
    return {s, sub_rn(b, sub_rn(s, a))};
}
// x + y: the accurate double-word addition (sums of the high and of the low
// words by TwoSum, each followed by a renormalisation; Hida, Li and Bailey 2001).
__host__ __device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    F2 s = two_sum(x.hi, y.hi);
    const F2 t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, add_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, add_rn(s.lo, t.lo));
}

template <int NSUM>
__device__ __forceinline__ void warp_sum(F2 (&v)[NSUM]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < NSUM; ++k) {
            const F2 o = {__shfl_down_sync(0xffffffffu, v[k].hi, off), __shfl_down_sync(0xffffffffu, v[k].lo, off)};
            v[k] = f2_add(v[k], o);
        }
    }
}

// Sum of F2 values over the block, valid in thread 0.
template <int NSUM>
__device__ __forceinline__ void block_sum(F2 (&v)[NSUM]) {
    __shared__ float2 shf[NSUM][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_sum<NSUM>(v);
    __syncthreads();   // shf may still be read by a previous call
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NSUM; ++k) shf[k][warp] = make_float2(v[k].hi, v[k].lo);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) v[k] = f2_add(v[k], F2{shf[k][w].x, shf[k][w].y});
        }
    }
}

// grid_reduce for FP32 per-thread partial sums: block sums stored as FP32
// pairs in the partial-sum slots; the last block sums them with the same code
// that formed its own block sum (a second pass of one loop, so those
// instructions are already in its SM's instruction cache: code that only the
// last block runs costs instruction fetches from memory on the critical path)
// and widens the pair's exact value to FP64 for the scalar stage.
template <int NSUM, int HINT = ST_NONE>
__device__ __forceinline__ void grid_reduce(const float (&vf)[NSUM], const RedCtx& rc, const Slice& sl) {
    __shared__ unsigned is_last;
    WD_TL_DECL
    WD_TL_T(0)
    float2* part = reinterpret_cast<float2*>(rc.partials + (size_t)sl.rhs * RED_STRIDE);
    unsigned* ticket = rc.ticket + sl.rhs;
    F2 v[NSUM];
#pragma unroll
    for (int k = 0; k < NSUM; ++k) v[k] = F2{vf[k], 0.f};
#pragma unroll 1
    for (int pass = 0;; ++pass) {
        block_sum<NSUM>(v);
        if (pass == 1) break;
        WD_TL_T(1)
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NSUM; ++k) part[(size_t)sl.b * NSUM + k] = make_float2(v[k].hi, v[k].lo);
            WD_TL_T(2)
            is_last = (ticket_add(ticket) == (unsigned)sl.nb - 1) ? 1u : 0u;
            WD_TL_T(3)
        }
        __syncthreads();
        if (!is_last) return;
        WD_TL_T(4)
#pragma unroll
        for (int k = 0; k < NSUM; ++k) v[k] = F2{0.f, 0.f};
#pragma unroll 3
        for (int b = threadIdx.x; b < sl.nb; b += blockDim.x) {
            float2 t[NSUM];
#pragma unroll
            for (int k = 0; k < NSUM; ++k) t[k] = __ldcg(part + (size_t)b * NSUM + k);
#pragma unroll
            for (int k = 0; k < NSUM; ++k) v[k] = f2_add(v[k], F2{t[k].x, t[k].y});
        }
        WD_TL_T(5)
    }
    if (threadIdx.x == 0) {
        WD_TL_T(6)
        double a[NSUM];
#pragma unroll
        for (int k = 0; k < NSUM; ++k) a[k] = (double)v[k].hi + (double)v[k].lo;
        if (rc.st) run_stage_hinted<HINT>(rc.stage, a, rc.st + sl.rhs);
        WD_TL_T(7)
        *ticket = 0u;
        WD_TL_PHASES(rc.stage, NSUM)
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may become resident while its predecessor in the stream is
// still running. It first waits for that predecessor to complete and its
// writes to be visible, then lets its own successor start launching. Both
// instructions do nothing for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_begin_wait() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
// A kernel may declare a local wd_tl_tag (0-15) before pdl_begin() to tell
// its variants apart in the timeline records (the hops: their reduction).
constexpr unsigned wd_tl_tag = 0;
#ifdef WD_TIMELINE
#define pdl_begin()                                                                                           \
    const unsigned long long wd_tl_arrive = ::wd::tl::now();                                                  \
    pdl_begin_wait();                                                                                         \
    const ::wd::tl::Scope wd_tl_scope((unsigned)__LINE__ | (wd_tl_tag << 12) |                                 \
                                          (::wd::tl::name_hash(::wd::tl::base_name(__FILE__, __FILE__)) << 16), \
                                      wd_tl_arrive)
#else
#define pdl_begin() pdl_begin_wait()
#endif

// Guards: inner-loop kernels return once the inner solve of their right-hand
// side is done (or the right-hand side is finished); refinement kernels only
// skip finished right-hand sides.
enum GuardKind { GUARD_NONE = 0, GUARD_INNER = 1, GUARD_OUTER = 2 };
__device__ __forceinline__ bool guarded(const SolverState* st, int kind) {
    if (st == nullptr || kind == GUARD_NONE) return false;
    const volatile SolverState* v = st;
    return v->skip || (kind == GUARD_INNER && v->done);
}

}  // namespace wd
