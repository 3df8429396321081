// Domain decomposition of the hopping term (Eq. 1) over a 4-D grid of
// sub-lattices, one per process, and the FP64 dot products and vector updates
// a solver on those sub-lattices needs (the paper sums every global reduction
// in FP64 across processes, Sec. 5, Fig. 3; its runs use 64 MPI processes,
// Sec. 6).
//
// A sub-domain handle holds its local sub-lattice (all extents even, so a
// site's parity is the same in local and global coordinates). In a direction
// mu split across processes (grid[mu] > 1) the gathered links of the hops that
// leave the sub-lattice are stored as zeros, so the ordinary hop kernels
// compute the interior part exactly and unchanged. The missing terms travel
// as half spinors, 12 reals per face site in the storage precision:
//   face 2 mu     (lower face, x_mu = 0):      h = (1 - gamma_mu) psi, two spin
//                 rows, for the forward hop of the neighbour below;
//   face 2 mu + 1 (upper face, x_mu = L - 1):  chi = U_mu(x)^+ (1 + gamma_mu) psi,
//                 the link already applied (it lives here), for the backward
//                 hop of the neighbour above;
// each times the boundary phase when the hop wraps around the global lattice.
// The receiver multiplies the forward half spinors by its own U_mu(x), rebuilds
// the four spin components and adds a * (the result) to the interior output.
#include <cstring>

#include "handle.h"
#include "hop_impl.cuh"

namespace wd {

// Face site f (of Vh / L[mu]) with x_mu = cmu on parity q: its parity site index
// and its lexicographic index. The three other coordinates run
// lexicographically (lowest direction fastest); on a fixed parity the fastest
// of them alternates, so f is their lexicographic index halved.
__device__ __forceinline__ void face_site(const Geom& g, int mu, int cmu, int q, int f, int* h, int* lex) {
    int o[3], k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (i != mu) o[k++] = i;
    const int e0h = g.L[o[0]] >> 1, e1 = g.L[o[1]];
    const int kk = f % e0h, rest = f / e0h;
    int c[4];
    c[o[1]] = rest % e1;
    c[o[2]] = rest / e1;
    c[mu] = cmu;
    c[o[0]] = 2 * kk + ((q + cmu + c[o[1]] + c[o[2]]) & 1);
    const int s = c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
    *lex = s;
    *h = s >> 1;
}

// A stored FP64 link entry as the hop kernels see it: rounded to the storage type.
template <typename T> __device__ __forceinline__ typename Unit<T>::C link_val(double v);
template <> __device__ __forceinline__ double link_val<double>(double v) { return v; }
template <> __device__ __forceinline__ float link_val<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ float link_val<__half>(double v) { return __half2float(__double2half(v)); }
template <> __device__ __forceinline__ float link_val<__nv_bfloat16>(double v) {
    return __bfloat162float(__double2bfloat16(v));
}

template <typename T> __device__ __forceinline__ T to_store(typename Unit<T>::C v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename T> __device__ __forceinline__ typename Unit<T>::C from_store(T v);
template <> __device__ __forceinline__ double from_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_store<float>(float v) { return v; }
template <> __device__ __forceinline__ float from_store<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float from_store<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// x_k = M h_k (k = 0, 1) for a 3x3 complex M given as 18 reals, row-major; with
// dagger, M^+ is applied instead.
template <typename C>
__device__ __forceinline__ void mul3(const C (&m)[18], bool dagger, const C (&h)[12], C (&x)[12]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C re = 0, im = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int e = dagger ? 2 * (3 * b + a) : 2 * (3 * a + b);
                const C mr = m[e], mi = dagger ? -m[e + 1] : m[e + 1];
                const C hr = h[6 * k + 2 * b], hi = h[6 * k + 2 * b + 1];
                re = fmac(mr, hr, fmac(-mi, hi, re));
                im = fmac(mr, hi, fmac(mi, hr, im));
            }
            x[6 * k + 2 * a] = re;
            x[6 * k + 2 * a + 1] = im;
        }
}

template <typename T>
__device__ __forceinline__ void load_link(const double* U64, int V, int mu, int lex, typename Unit<T>::C (&m)[18]) {
    const double* u = U64 + ((size_t)mu * V + lex) * 18;
#pragma unroll
    for (int e = 0; e < 18; ++e) m[e] = link_val<T>(u[e]);
}

// Face `side` (0: lower, 1: upper) in direction mu of the input vector `in`
// (parity q), 12 reals per face site, real e of face site f at face[e * F + f].
template <typename T>
__global__ void __launch_bounds__(128) k_dd_pack(Geom g, int q, int mu, int side, const uint4* __restrict__ in,
                                                 const double* __restrict__ U64, double phase, T* __restrict__ face) {
    typedef typename Unit<T>::C C;
    const int F = g.Vh / g.L[mu];
    const int cmu = side == 0 ? 0 : g.L[mu] - 1;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
        int h, lex;
        face_site(g, mu, cmu, q, f, &h, &lex);
        C p[24];
        load_spinor<T>(in, g.Vh, h, p);
        C hs[12], x[12];
        project<C>(mu, side == 0, p, hs);   // side 0: (1 - gamma_mu), side 1: (1 + gamma_mu)
        if (side == 1) {
            C m[18];
            load_link<T>(U64, 2 * g.Vh, mu, lex, m);
            mul3<C>(m, true, hs, x);
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) x[i] = hs[i];
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) face[(size_t)i * F + f] = to_store<T>((C)phase * x[i]);
    }
}

// out += a * (hop terms of the received face `side` of direction mu) on the
// output sites of parity p: side 0 holds the lower face of the neighbour above
// (forward hops of this sub-lattice's upper face, x_mu = L - 1, times U_mu(x)
// here), side 1 the upper face of the neighbour below (backward hops of the
// lower face, x_mu = 0, link already applied).
template <typename T>
__global__ void __launch_bounds__(128) k_dd_face(Geom g, int p, int mu, int side, const T* __restrict__ face,
                                                 const double* __restrict__ U64, double a, uint4* out) {
    typedef typename Unit<T>::C C;
    const int F = g.Vh / g.L[mu];
    const int cmu = side == 0 ? g.L[mu] - 1 : 0;
    const bool fwd = side == 0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F; f += gridDim.x * blockDim.x) {
        int h, lex;
        face_site(g, mu, cmu, p, f, &h, &lex);
        C hs[12], x[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) hs[i] = from_store<T>(face[(size_t)i * F + f]);
        if (fwd) {
            C m[18];
            load_link<T>(U64, 2 * g.Vh, mu, lex, m);
            mul3<C>(m, false, hs, x);
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) x[i] = hs[i];
        }
        C acc[24];
        load_spinor_cg<T>(out, g.Vh, h, acc);
        reconstruct<C>(mu, fwd, (C)(mu == 3 ? 2.0 * a : a), x, acc);
        store_spinor<T>(out, g.Vh, h, acc);
    }
}

// Deterministic FP64 dot product sum_i conj(a_i) b_i over n sites of 24 reals:
// per-block partials, then one block sums them in block order.
constexpr int DOT_BLOCK = 256;
constexpr int DOT_MAX_BLOCKS = 1024;

template <typename T>
__global__ void __launch_bounds__(DOT_BLOCK) k_dot_partial(int n, const uint4* __restrict__ a,
                                                          const uint4* __restrict__ b, double* __restrict__ part) {
    typedef typename Unit<T>::C C;
    double re = 0.0, im = 0.0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        C x[24], y[24];
        load_spinor<T>(a, n, h, x);
        load_spinor<T>(b, n, h, y);
        C sr = 0, si = 0;
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            sr += x[2 * i] * y[2 * i] + x[2 * i + 1] * y[2 * i + 1];
            si += x[2 * i] * y[2 * i + 1] - x[2 * i + 1] * y[2 * i];
        }
        re += (double)sr;
        im += (double)si;
    }
    __shared__ double s_re[DOT_BLOCK / 32], s_im[DOT_BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_re[w] = re;
        s_im[w] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int i = 0; i < DOT_BLOCK / 32; ++i) {
            tr += s_re[i];
            ti += s_im[i];
        }
        part[2 * blockIdx.x] = tr;
        part[2 * blockIdx.x + 1] = ti;
    }
}

__global__ void k_dot_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int i = 0; i < nb; ++i) {
            tr += part[2 * i];
            ti += part[2 * i + 1];
        }
        out[0] = tr;
        out[1] = ti;
    }
}

// y = a x + b y (complex a, b) over n sites of 24 reals.
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(int n, double ar, double ai, const uint4* __restrict__ x, double br,
                                               double bi, uint4* y) {
    typedef typename Unit<T>::C C;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        C xv[24], yv[24], o[24];
        load_spinor<T>(x, n, h, xv);
        load_spinor_cg<T>(y, n, h, yv);
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const C xr = xv[2 * i], xi = xv[2 * i + 1], yr = yv[2 * i], yi = yv[2 * i + 1];
            o[2 * i] = (C)ar * xr - (C)ai * xi + (C)br * yr - (C)bi * yi;
            o[2 * i + 1] = (C)ar * xi + (C)ai * xr + (C)br * yi + (C)bi * yr;
        }
        store_spinor<T>(y, n, h, o);
    }
}

static int prec_size(int prec) { return prec == WD_FP64 ? 8 : prec == WD_FP32 ? 4 : 2; }

static int grid_of(long n, int block) {
    long g = (n + block - 1) / block;
    const long cap = (long)num_sms() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace wd

using namespace wd;

extern "C" {

int wd_dd_set_partition(wd_handle* h, const int grid[4], const int coords[4]) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!grid || !coords) return fail(h, WD_ERR_INVALID_ARG, "wd_dd_set_partition: null grid or coords");
    unsigned mask = 0;
    for (int mu = 0; mu < 4; ++mu) {
        if (grid[mu] < 1 || coords[mu] < 0 || coords[mu] >= grid[mu])
            return fail(h, WD_ERR_INVALID_ARG, "wd_dd_set_partition: grid[%d] = %d, coords[%d] = %d", mu, grid[mu], mu,
                        coords[mu]);
        if (grid[mu] > 1) mask |= 1u << mu;
    }
    if (mask && h->have_clover)
        return fail(h, WD_ERR_INVALID_ARG, "wd_dd_set_partition: a split lattice takes no clover term");
    h->g.part = mask;
    for (int mu = 0; mu < 4; ++mu) {
        h->dd_grid[mu] = grid[mu];
        h->dd_coords[mu] = coords[mu];
    }
    // the gathered links carry the split: rebuild them on next use
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                if (h->links[a][b][c]) {
                    cudaDeviceSynchronize();
                    cudaFree(h->links[a][b][c]);
                    h->links[a][b][c] = nullptr;
                }
    h->gen += 1;
    return WD_OK;
}

size_t wd_dd_face_bytes(const wd_handle* h, int prec, int mu) {
    if (!h || !valid_prec(prec) || mu < 0 || mu > 3) return 0;
    return (size_t)(h->g.Vh / h->g.L[mu]) * 12 * prec_size(prec);
}

int wd_dd_pack(wd_handle* h, int prec, int parity, const void* in, void* const send[8], void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || (parity != 0 && parity != 1) || !in || !send)
        return fail(h, WD_ERR_INVALID_ARG, "wd_dd_pack: bad argument");
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    for (int mu = 0; mu < 4; ++mu) {
        if (!((h->g.part >> mu) & 1)) continue;
        const int F = h->g.Vh / h->g.L[mu];
        for (int side = 0; side < 2; ++side) {
            void* dst = send[2 * mu + side];
            if (!dst) return fail(h, WD_ERR_INVALID_ARG, "wd_dd_pack: face buffer %d is null", 2 * mu + side);
            // the hop wraps around the global lattice between the first and the last process of the row
            const bool wraps = side == 0 ? h->dd_coords[mu] == 0 : h->dd_coords[mu] == h->dd_grid[mu] - 1;
            const double phase = wraps ? (double)h->g.bc[mu] : 1.0;
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                k_dd_pack<T><<<grid_of(F, 128), 128, 0, s>>>(h->g, 1 - parity, mu, side, (const uint4*)in, h->U64,
                                                              phase, (T*)dst);
                return cudaGetLastError();
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "wd_dd_pack");
        }
    }
    return WD_OK;
}

int wd_dd_hop_interior(wd_handle* h, int prec, int recon, int parity, const void* in, const void* y, double a,
                       double b, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || !valid_recon(recon) || (parity != 0 && parity != 1) || !in || !out ||
        (b != 0.0 && !y))
        return fail(h, WD_ERR_INVALID_ARG, "wd_dd_hop_interior: bad argument");
    if (in == out) return fail(h, WD_ERR_INVALID_ARG, "wd_dd_hop_interior: in and out must not overlap");
    const uint4 *le, *lo;
    int rc = ensure_links(h, prec, recon, &le, &lo);
    if (rc != WD_OK) return rc;
    HopParams P{};
    P.g = h->g;
    P.nrhs = 1;
    P.guard_kind = GUARD_NONE;
    apply_tuning(h, prec, recon, P);
    P.parity = parity;
    P.links = parity == 0 ? le : lo;
    P.in = (const uint4*)in;
    P.out = (uint4*)out;
    P.y = (const uint4*)y;
    P.a = a;
    P.b = b;
    const int epi = b == 0.0 ? EPI_H : EPI_Y;
    cudaError_t e = by_prec(prec, [&](auto tag) {
        typedef typename decltype(tag)::type T;
        return Ops<T>::hop(recon, epi, RED_NONE, P, (cudaStream_t)stream);
    });
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, "wd_dd_hop_interior");
}

int wd_dd_hop_faces(wd_handle* h, int prec, int parity, const void* const recv[8], double a, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || (parity != 0 && parity != 1) || !recv || !out)
        return fail(h, WD_ERR_INVALID_ARG, "wd_dd_hop_faces: bad argument");
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    cudaStream_t s = (cudaStream_t)stream;
    // one launch per face, in order: corner sites receive terms from several faces
    for (int mu = 0; mu < 4; ++mu) {
        if (!((h->g.part >> mu) & 1)) continue;
        const int F = h->g.Vh / h->g.L[mu];
        for (int side = 0; side < 2; ++side) {
            const void* src = recv[2 * mu + side];
            if (!src) return fail(h, WD_ERR_INVALID_ARG, "wd_dd_hop_faces: face buffer %d is null", 2 * mu + side);
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                k_dd_face<T><<<grid_of(F, 128), 128, 0, s>>>(h->g, parity, mu, side, (const T*)src, h->U64, a,
                                                              (uint4*)out);
                return cudaGetLastError();
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "wd_dd_hop_faces");
        }
    }
    return WD_OK;
}

int wd_vec_dot(wd_handle* h, int prec, const void* a, const void* b, double out[2], void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || !a || !b || !out) return fail(h, WD_ERR_INVALID_ARG, "wd_vec_dot: bad argument");
    double* part = (double*)workspace(h, "vec.dot", sizeof(double) * (2 * DOT_MAX_BLOCKS + 2));
    if (!part) return fail(h, WD_ERR_CUDA, "out of device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int nb = (h->g.Vh + DOT_BLOCK - 1) / DOT_BLOCK;
    if (nb > DOT_MAX_BLOCKS) nb = DOT_MAX_BLOCKS;
    cudaError_t e = by_prec(prec, [&](auto tag) {
        typedef typename decltype(tag)::type T;
        k_dot_partial<T><<<nb, DOT_BLOCK, 0, s>>>(h->g.Vh, (const uint4*)a, (const uint4*)b, part);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "wd_vec_dot");
    k_dot_final<<<1, 32, 0, s>>>(nb, part, part + 2 * DOT_MAX_BLOCKS);
    WD_CUDA(h, cudaGetLastError());
    WD_CUDA(h, cudaMemcpyAsync(out, part + 2 * DOT_MAX_BLOCKS, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    WD_CUDA(h, cudaStreamSynchronize(s));
    return WD_OK;
}

int wd_vec_axpby(wd_handle* h, int prec, const double a[2], const void* x, const double b[2], void* y, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || !a || !b || !x || !y) return fail(h, WD_ERR_INVALID_ARG, "wd_vec_axpby: bad argument");
    cudaError_t e = by_prec(prec, [&](auto tag) {
        typedef typename decltype(tag)::type T;
        k_axpby<T><<<grid_of(h->g.Vh, 256), 256, 0, (cudaStream_t)stream>>>(h->g.Vh, a[0], a[1], (const uint4*)x,
                                                                              b[0], b[1], (uint4*)y);
        return cudaGetLastError();
    });
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, "wd_vec_axpby");
}

}  // extern "C"
