// Clover (Sheikholeslami-Wohlert) blocks of the Wilson-clover matrix
// D_sw = C - kappa H, the diagonal blocks D_ee = C_ee, D_oo = C_oo of Eqs. 4-5:
//   C(x) = 1 - c_sw kappa sum_{mu<nu} sigma_mu_nu (x) Fh_mu_nu(x),
//   sigma_mu_nu = (i/2) [gamma_mu, gamma_nu],
//   Fh_mu_nu = traceless part of (Q_mu_nu - Q_mu_nu^+) / (8 i),
// Q_mu_nu(x) the four plaquettes of the mu-nu plane with a corner at x, each
// traversed mu-then-nu. Built once per gauge field in FP64, one thread per
// site: C and C^{-1} (Gauss-Jordan with partial pivoting) are written as
// 12 x 12 complex blocks (row-major, spin-colour index 3 s + a) per parity in
// the unit layout of the spinors. The operators use C^-1 in the chiral packing
// (two Hermitian 6 x 6 blocks, 80 reals per site; see mat_mul_chiral), made
// on first use per precision; C itself (full) serves the true residual.
#include <algorithm>
#include <cmath>
#include <string>

#include "handle.h"

namespace wd {

namespace {

struct Z {
    double r, i;
};
__device__ __forceinline__ Z zmul(Z a, Z b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Z zsub(Z a, Z b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Z zconj(Z a) { return {a.r, -a.i}; }

struct M3 {
    Z e[3][3];
};

__device__ M3 mul(const M3& a, const M3& b) {
    M3 c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Z s = {0, 0};
            for (int k = 0; k < 3; ++k) s = zadd(s, zmul(a.e[i][k], b.e[k][j]));
            c.e[i][j] = s;
        }
    return c;
}

__device__ M3 dag(const M3& a) {
    M3 c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.e[i][j] = zconj(a.e[j][i]);
    return c;
}

// Lexicographic index of the site at coordinates c shifted by (s0 mu-hat + s1 nu-hat), periodic.
__device__ long long shifted(const Geom& g, const int (&c)[4], int mu, int s0, int nu, int s1) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + s0 + g.L[mu]) % g.L[mu];
    d[nu] = (d[nu] + s1 + g.L[nu]) % g.L[nu];
    return d[0] + (long long)g.L[0] * (d[1] + (long long)g.L[1] * (d[2] + (long long)g.L[2] * d[3]));
}

__device__ M3 link(const double* U, long long V, int mu, long long site) {
    const double* p = U + ((size_t)mu * V + site) * 18;
    M3 m;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m.e[a][b] = {p[2 * (3 * a + b)], p[2 * (3 * a + b) + 1]};
    return m;
}

// gamma_mu[s][t] in the Dirac representation: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = diag(1, 1, -1, -1).
__device__ Z gamma_el(int mu, int s, int t) {
    if (mu == 3) return {(s == t) ? (s < 2 ? 1.0 : -1.0) : 0.0, 0.0};
    const bool upper = s < 2, tupper = t < 2;
    if (upper == tupper) return {0, 0};
    const int a = s & 1, b = t & 1;
    Z p;   // Pauli sigma_{mu+1}[a][b]
    if (mu == 0) p = {(a != b) ? 1.0 : 0.0, 0.0};
    else if (mu == 1) p = (a == b) ? Z{0, 0} : (a == 0 ? Z{0, -1} : Z{0, 1});
    else p = (a != b) ? Z{0, 0} : Z{a == 0 ? 1.0 : -1.0, 0.0};
    const Z f = upper ? Z{0, -1} : Z{0, 1};   // -i (upper right block) or +i (lower left block)
    return zmul(f, p);
}

// sigma_mu_nu[s][t] = (i/2) sum_u (gamma_mu[s][u] gamma_nu[u][t] - gamma_nu[s][u] gamma_mu[u][t])
__device__ Z sigma_el(int mu, int nu, int s, int t) {
    Z c = {0, 0};
    for (int u = 0; u < 4; ++u)
        c = zadd(c, zsub(zmul(gamma_el(mu, s, u), gamma_el(nu, u, t)), zmul(gamma_el(nu, s, u), gamma_el(mu, u, t))));
    return zmul(Z{0, 0.5}, c);
}

__device__ void store_block(uint4* dst, int Vh, int h, const Z (&m)[12][12]) {
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
            uint4 w;
            w.x = (unsigned)__double2loint(m[i][j].r);
            w.y = (unsigned)__double2hiint(m[i][j].r);
            w.z = (unsigned)__double2loint(m[i][j].i);
            w.w = (unsigned)__double2hiint(m[i][j].i);
            dst[(size_t)(12 * i + j) * Vh + h] = w;
        }
}

__global__ void __launch_bounds__(128) k_clover_build(Geom g, const double* U, double ck, uint4* fwd_e, uint4* fwd_o,
                                                      uint4* inv_e, uint4* inv_o, int* singular) {
    const long long V = 2LL * g.Vh;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V; s += (long long)gridDim.x * blockDim.x) {
        int c[4];
        long long r = s;
        c[0] = (int)(r % g.L[0]); r /= g.L[0];
        c[1] = (int)(r % g.L[1]); r /= g.L[1];
        c[2] = (int)(r % g.L[2]); r /= g.L[2];
        c[3] = (int)r;
        const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
        const int h = (int)(s / 2);
        Z a[12][12];
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) a[i][j] = {i == j ? 1.0 : 0.0, 0.0};
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const M3 um = link(U, V, mu, s), un = link(U, V, nu, s);
                M3 q = mul(mul(mul(um, link(U, V, nu, shifted(g, c, mu, 1, nu, 0))),
                               dag(link(U, V, mu, shifted(g, c, mu, 0, nu, 1)))),
                           dag(un));
                M3 l = mul(mul(mul(un, dag(link(U, V, mu, shifted(g, c, mu, -1, nu, 1)))),
                               dag(link(U, V, nu, shifted(g, c, mu, -1, nu, 0)))),
                           link(U, V, mu, shifted(g, c, mu, -1, nu, 0)));
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) q.e[i][j] = zadd(q.e[i][j], l.e[i][j]);
                l = mul(mul(mul(dag(link(U, V, mu, shifted(g, c, mu, -1, nu, 0))),
                                dag(link(U, V, nu, shifted(g, c, mu, -1, nu, -1)))),
                            link(U, V, mu, shifted(g, c, mu, -1, nu, -1))),
                        link(U, V, nu, shifted(g, c, mu, 0, nu, -1)));
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) q.e[i][j] = zadd(q.e[i][j], l.e[i][j]);
                l = mul(mul(mul(dag(link(U, V, nu, shifted(g, c, mu, 0, nu, -1))),
                                link(U, V, mu, shifted(g, c, mu, 0, nu, -1))),
                            link(U, V, nu, shifted(g, c, mu, 1, nu, -1))),
                        dag(um));
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) q.e[i][j] = zadd(q.e[i][j], l.e[i][j]);
                // F = (Q - Q^+) / (8 i), then its traceless part
                Z f[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        const Z d = zsub(q.e[i][j], zconj(q.e[j][i]));
                        f[i][j] = {d.i / 8.0, -d.r / 8.0};   // d / (8 i)
                    }
                const Z tr = {(f[0][0].r + f[1][1].r + f[2][2].r) / 3.0, (f[0][0].i + f[1][1].i + f[2][2].i) / 3.0};
                for (int i = 0; i < 3; ++i) f[i][i] = zsub(f[i][i], tr);
                for (int s1 = 0; s1 < 4; ++s1)
                    for (int t1 = 0; t1 < 4; ++t1) {
                        const Z sg = sigma_el(mu, nu, s1, t1);
                        if (sg.r == 0.0 && sg.i == 0.0) continue;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) {
                                const Z v = zmul(sg, f[i][j]);
                                a[3 * s1 + i][3 * t1 + j] = zsub(a[3 * s1 + i][3 * t1 + j], Z{ck * v.r, ck * v.i});
                            }
                    }
            }
        store_block(p == 0 ? fwd_e : fwd_o, g.Vh, h, a);
        // inverse by Gauss-Jordan elimination with partial pivoting
        Z inv[12][12];
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) inv[i][j] = {i == j ? 1.0 : 0.0, 0.0};
        bool ok = true;
        for (int col = 0; col < 12; ++col) {
            int piv = col;
            double best = -1.0;
            for (int i = col; i < 12; ++i) {
                const double m = a[i][col].r * a[i][col].r + a[i][col].i * a[i][col].i;
                if (m > best) { best = m; piv = i; }
            }
            if (!(best > 0.0)) { ok = false; break; }
            if (piv != col)
                for (int j = 0; j < 12; ++j) {
                    Z t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
                    t = inv[col][j]; inv[col][j] = inv[piv][j]; inv[piv][j] = t;
                }
            const Z d = a[col][col];
            const Z rd = {d.r / best, -d.i / best};   // 1 / d
            for (int j = 0; j < 12; ++j) {
                a[col][j] = zmul(a[col][j], rd);
                inv[col][j] = zmul(inv[col][j], rd);
            }
            for (int i = 0; i < 12; ++i) {
                if (i == col) continue;
                const Z fct = a[i][col];
                if (fct.r == 0.0 && fct.i == 0.0) continue;
                for (int j = 0; j < 12; ++j) {
                    a[i][j] = zsub(a[i][j], zmul(fct, a[col][j]));
                    inv[i][j] = zsub(inv[i][j], zmul(fct, inv[col][j]));
                }
            }
        }
        if (!ok) atomicExch(singular, 1);
        store_block(p == 0 ? inv_e : inv_o, g.Vh, h, inv);
    }
}

}  // namespace

// (Re)build the FP64 clover blocks of the handle's gauge field; lower-precision
// copies are dropped and rebuilt on first use.
int clover_build(wd_handle* h) {
    const size_t bytes = (size_t)h->g.Vh * 144 * 16;
    uint4* b[4];
    const char* names[4] = {"clov.fwd64.e", "clov.fwd64.o", "clov.inv64.e", "clov.inv64.o"};
    for (int i = 0; i < 4; ++i) {
        b[i] = (uint4*)workspace(h, names[i], bytes);
        if (!b[i]) return fail(h, WD_ERR_CUDA, "out of device memory (clover blocks)");
    }
    int* sing = (int*)workspace(h, "clov.singular", sizeof(int));
    if (!sing) return fail(h, WD_ERR_CUDA, "out of device memory");
    WD_CUDA(h, cudaMemset(sing, 0, sizeof(int)));
    const long long V = 2LL * h->g.Vh;
    const int grid = (int)std::min<long long>((V + 127) / 128, (long long)num_sms() * 16);
    k_clover_build<<<grid, 128>>>(h->g, h->U64, h->csw * h->kappa, b[0], b[1], b[2], b[3], sing);
    WD_CUDA(h, cudaGetLastError());
    int hs = 0;
    WD_CUDA(h, cudaMemcpy(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost));
    if (hs) return fail(h, WD_ERR_INVALID_ARG, "wd_set_clover: a clover block is singular");
    for (int k = 0; k < 2; ++k)
        for (int p = 0; p < 4; ++p) h->clov[k][p][0] = h->clov[k][p][1] = nullptr;
    h->clov_inv64[0] = b[2];
    h->clov_inv64[1] = b[3];
    h->clov[1][WD_FP64][0] = b[0];
    h->clov[1][WD_FP64][1] = b[1];
    h->gen += 1;
    return WD_OK;
}

// Clover blocks of kind 0 (C^{-1}) or 1 (C) in precision prec for both
// parities; null pointers when the handle has no clover term.
int ensure_clover(wd_handle* h, int prec, int kind, const uint4** even, const uint4** odd) {
    *even = *odd = nullptr;
    if (!h->have_clover) return WD_OK;
    for (int p = 0; p < 2; ++p) {
        if (!h->clov[kind][prec][p]) {
            // C^-1: chiral packing, 80 reals per site; C: full block, 288 reals per site
            const size_t per_unit = 16 / (prec == WD_FP64 ? 8 : prec == WD_FP32 ? 4 : 2);
            const size_t units = (kind == 0 ? 80 : 288) / per_unit;
            const std::string name = "clov.k" + std::to_string(kind) + ".p" + std::to_string(prec) + "." +
                                     std::to_string(p);
            uint4* dst = (uint4*)workspace(h, name, (size_t)h->g.Vh * units * 16);
            if (!dst) return fail(h, WD_ERR_CUDA, "out of device memory (clover blocks)");
            const uint4* src = kind == 0 ? h->clov_inv64[p] : h->clov[1][WD_FP64][p];
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                return kind == 0 ? Ops<T>::chiral_from64(h->g.Vh, src, dst, nullptr)
                                 : Ops<T>::mat_from64(h->g.Vh, src, dst, nullptr);
            });
            WD_CUDA(h, e);
            WD_CUDA(h, cudaDeviceSynchronize());
            h->clov[kind][prec][p] = dst;
        }
    }
    *even = h->clov[kind][prec][0];
    *odd = h->clov[kind][prec][1];
    return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_set_clover(wd_handle* h, double csw) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!std::isfinite(csw)) return fail(h, WD_ERR_INVALID_ARG, "wd_set_clover: c_sw must be finite");
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_clover: wd_set_gauge has not been called");
    if (h->g.part && csw != 0.0) return fail(h, WD_ERR_INVALID_ARG, "wd_set_clover: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    if (csw == 0.0) {
        h->have_clover = false;
        h->csw = 0.0;
        for (int k = 0; k < 2; ++k)
            for (int p = 0; p < 4; ++p) h->clov[k][p][0] = h->clov[k][p][1] = nullptr;
        h->clov_inv64[0] = h->clov_inv64[1] = nullptr;
        h->gen += 1;
        return WD_OK;
    }
    h->csw = csw;
    int rc = clover_build(h);
    if (rc != WD_OK) {
        h->have_clover = false;
        return rc;
    }
    h->have_clover = true;
    return WD_OK;
}
