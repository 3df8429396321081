// C ABI entry points: handle lifetime, gauge upload and link packing, vector
// packing, and operator application (wd.h).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <vector>

#include "handle.h"

namespace wd {

static int g_hop_block = 0;
// Default threads per block of the hop kernels: environment WD_HOP_BLOCK (64 or 128), else 128.
int hop_block() {
    if (g_hop_block == 0) {
        const char* e = std::getenv("WD_HOP_BLOCK");
        const int b = e ? std::atoi(e) : 0;
        g_hop_block = (b == 64 || b == 128) ? b : 128;
    }
    return g_hop_block;
}
void set_hop_block(int b) { g_hop_block = b; }

int hop_variant() {
    static int v = 0;
    if (v == 0) {
        const char* e = std::getenv("WD_HOP_KERNEL");
        v = (e && e[0] >= '1' && e[0] <= '6') ? e[0] - '0' : 4;
    }
    return v;
}

int hop16_ahead() {
    static int v = 0;
    if (v == 0) {
        const char* e = std::getenv("WD_HOP16_AHEAD");
        v = (e && e[0] == '1') ? 1 : 2;
    }
    return v;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

static int prec_bytes(int prec) { return prec == WD_FP64 ? 8 : prec == WD_FP32 ? 4 : 2; }
int link_units(int prec, int recon) { return 8 * recon * prec_bytes(prec) / 16; }
int spinor_units(int prec) { return 24 * prec_bytes(prec) / 16; }

int fail(wd_handle* h, int code, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(wd_handle* h, cudaError_t e, const char* what) {
    return fail(h, WD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t vec_bytes(const wd_handle* h, int prec) { return (size_t)h->g.Vh * spinor_units(prec) * 16; }

void* workspace(wd_handle* h, const std::string& name, size_t bytes) {
    Buffer& b = h->ws[name];
    if (b.p && b.bytes >= bytes) return b.p;
    if (b.p) {
        cudaDeviceSynchronize();
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        b.p = nullptr;
        return nullptr;
    }
    b.bytes = bytes;
    ++h->gen;
    return b.p;
}

RedCtx red_ctx(wd_handle* h, int stage) {
    RedCtx rc;
    rc.partials = h->partials;
    rc.ticket = h->ticket;
    rc.st = h->st;
    rc.stage = stage;
    return rc;
}

int ensure_solver_state(wd_handle* h, int nrhs) {
    if (!h->cap) {
        WD_CUDA(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) WD_CUDA(h, cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming));
        WD_CUDA(h, cudaEventCreate(&h->t0));
        WD_CUDA(h, cudaEventCreate(&h->t1));
        WD_CUDA(h, cudaHostAlloc((void**)&h->hflag, sizeof(int), cudaHostAllocMapped));
        WD_CUDA(h, cudaHostGetDevicePointer((void**)&h->dflag, h->hflag, 0));
    }
    if (h->cap_rhs >= nrhs) return WD_OK;
    WD_CUDA(h, cudaDeviceSynchronize());
    if (h->st) cudaFree(h->st);
    if (h->partials) cudaFree(h->partials);
    if (h->ticket) cudaFree(h->ticket);
    if (h->hst) cudaFreeHost(h->hst);
    h->st = nullptr;
    h->partials = nullptr;
    h->ticket = nullptr;
    h->hst = nullptr;
    h->cap_rhs = 0;
    WD_CUDA(h, cudaMalloc(&h->st, sizeof(SolverState) * nrhs));
    WD_CUDA(h, cudaMemset(h->st, 0, sizeof(SolverState) * nrhs));
    WD_CUDA(h, cudaMalloc(&h->partials, sizeof(double) * RED_STRIDE * nrhs));
    WD_CUDA(h, cudaMalloc(&h->ticket, sizeof(unsigned) * nrhs));
    WD_CUDA(h, cudaMemset(h->ticket, 0, sizeof(unsigned) * nrhs));
    WD_CUDA(h, cudaMallocHost(&h->hst, sizeof(SolverState) * nrhs));
    std::memset(h->hst, 0, sizeof(SolverState) * nrhs);
    h->cap_rhs = nrhs;
    ++h->gen;
    return WD_OK;
}

int ensure_links(wd_handle* h, int prec, int recon, const uint4** even, const uint4** odd) {
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    if (!valid_prec(prec) || !valid_recon(recon)) return fail(h, WD_ERR_INVALID_ARG, "bad precision %d or recon %d", prec, recon);
    const int ri = recon == 12 ? 0 : 1;
    if (!h->links[prec][ri][0]) {
        if (recon == 12 && (h->unit_dev > 1e-6 || h->det_dev > 1e-6))
            return fail(h, WD_ERR_NOT_SU3, "12-real links need SU(3) links: max |UU^+ - 1| = %g, max |det U - 1| = %g",
                        h->unit_dev, h->det_dev);
        const size_t bytes = (size_t)h->g.Vh * link_units(prec, recon) * 16;
        for (int p = 0; p < 2; ++p) {
            uint4* buf = nullptr;
            WD_CUDA(h, cudaMalloc(&buf, bytes));
            h->links[prec][ri][p] = buf;
            cudaError_t e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                return Ops<T>::build_links(recon, h->g, p, h->U64, buf, 0);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "build_links");
        }
        WD_CUDA(h, cudaDeviceSynchronize());
    }
    *even = h->links[prec][ri][0];
    *odd = h->links[prec][ri][1];
    return WD_OK;
}

// max |U U^+ - 1| and max |det U - 1| over links, as bit patterns of
// non-negative doubles (monotone as unsigned integers).
__global__ void k_unitarity(int nlinks, const double* U, unsigned long long* out) {
    double du = 0.0, dd = 0.0;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += gridDim.x * blockDim.x) {
        const double* m = U + (size_t)l * 18;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double re = 0, im = 0;
                for (int k = 0; k < 3; ++k) {   // sum_k U_ak conj(U_bk)
                    const double ar = m[2 * (3 * a + k)], ai = m[2 * (3 * a + k) + 1];
                    const double br = m[2 * (3 * b + k)], bi = m[2 * (3 * b + k) + 1];
                    re += ar * br + ai * bi;
                    im += ai * br - ar * bi;
                }
                if (a == b) re -= 1.0;
                du = fmax(du, sqrt(re * re + im * im));
            }
#define R_(a, b) m[2 * (3 * (a) + (b))]
#define I_(a, b) m[2 * (3 * (a) + (b)) + 1]
        double dr = 0, di = 0;
        for (int b = 0; b < 3; ++b) {
            const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            const double cr = R_(1, b1) * R_(2, b2) - I_(1, b1) * I_(2, b2) - (R_(1, b2) * R_(2, b1) - I_(1, b2) * I_(2, b1));
            const double ci = R_(1, b1) * I_(2, b2) + I_(1, b1) * R_(2, b2) - (R_(1, b2) * I_(2, b1) + I_(1, b2) * R_(2, b1));
            dr += R_(0, b) * cr - I_(0, b) * ci;
            di += R_(0, b) * ci + I_(0, b) * cr;
        }
#undef R_
#undef I_
        dd = fmax(dd, sqrt((dr - 1.0) * (dr - 1.0) + di * di));
    }
    for (int off = 16; off > 0; off >>= 1) {
        du = fmax(du, __shfl_down_sync(0xffffffffu, du, off));
        dd = fmax(dd, __shfl_down_sync(0xffffffffu, dd, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(du));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(dd));
    }
}

cudaError_t launch_unitarity(int nlinks, const double* U, unsigned long long* out, cudaStream_t s) {
    int grid = (nlinks + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_unitarity<<<grid, 256, 0, s>>>(nlinks, U, out);
    return cudaGetLastError();
}

}  // namespace wd

#ifdef WD_TIMELINE
namespace wd {
namespace tl {
static std::vector<int (*)(void*, void*)>& units() {
    static std::vector<int (*)(void*, void*)> u;
    return u;
}
void register_unit(int (*setter)(void*, void*)) { units().push_back(setter); }
}  // namespace tl
}  // namespace wd
#endif

using namespace wd;

extern "C" {

int wd_create(const int dims[4], double kappa, const int bc[4], wd_handle** out) {
    if (!out || !dims) return WD_ERR_INVALID_ARG;
    *out = nullptr;
    long long v = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2 || dims[i] % 2) return WD_ERR_INVALID_ARG;
        v *= dims[i];
    }
    if (v / 2 >= (1LL << 31) / 8) return WD_ERR_INVALID_ARG;   // site and unit indices stay in int range
    if (!std::isfinite(kappa)) return WD_ERR_INVALID_ARG;
    int b[4] = {1, 1, 1, -1};
    if (bc) {
        for (int i = 0; i < 4; ++i) {
            if (bc[i] != 1 && bc[i] != -1) return WD_ERR_INVALID_ARG;
            b[i] = bc[i];
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return WD_ERR_CUDA;
    wd_handle* h = new (std::nothrow) wd_handle();
    if (!h) return WD_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) {
        h->g.L[i] = dims[i];
        h->g.bc[i] = b[i];
    }
    h->g.Lxh = dims[0] / 2;
    h->g.Vh = (int)(v / 2);
    h->g.fxh.init(h->g.Lxh);
    h->g.fy.init(dims[1]);
    h->g.fz.init(dims[2]);
    h->kappa = kappa;
    cudaGetDevice(&h->device);
    *out = h;
    return WD_OK;
}

int wd_destroy(wd_handle* h) {
    if (!h) return WD_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : h->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                if (h->links[a][b][c]) cudaFree(h->links[a][b][c]);
    if (h->U64) cudaFree(h->U64);
    if (h->st) cudaFree(h->st);
    if (h->partials) cudaFree(h->partials);
    if (h->ticket) cudaFree(h->ticket);
    if (h->hst) cudaFreeHost(h->hst);
    if (h->hflag) cudaFreeHost(h->hflag);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (int i = 0; i < 2; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    if (h->t0) cudaEventDestroy(h->t0);
    if (h->t1) cudaEventDestroy(h->t1);
    delete h;
    return WD_OK;
}

int wd_set_gauge(wd_handle* h, const double* U, int where) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!U || (where != WD_HOST && where != WD_DEVICE)) return fail(h, WD_ERR_INVALID_ARG, "bad gauge pointer or location");
    const size_t nl = (size_t)8 * h->g.Vh;   // 4 V links
    const size_t bytes = nl * 18 * sizeof(double);
    if (!h->U64) WD_CUDA(h, cudaMalloc(&h->U64, bytes));
    WD_CUDA(h, cudaMemcpy(h->U64, U, bytes, where == WD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                if (h->links[a][b][c]) {
                    cudaFree(h->links[a][b][c]);
                    h->links[a][b][c] = nullptr;
                }
    unsigned long long* dev = (unsigned long long*)workspace(h, "unitarity", 2 * sizeof(unsigned long long));
    if (!dev) return fail(h, WD_ERR_CUDA, "out of device memory");
    WD_CUDA(h, cudaMemset(dev, 0, 2 * sizeof(unsigned long long)));
    WD_CUDA(h, launch_unitarity((int)nl, h->U64, dev, 0));
    unsigned long long host[2];
    WD_CUDA(h, cudaMemcpy(host, dev, sizeof host, cudaMemcpyDeviceToHost));
    std::memcpy(&h->unit_dev, &host[0], sizeof(double));
    std::memcpy(&h->det_dev, &host[1], sizeof(double));
    h->have_gauge = true;
    if (h->have_clover) return clover_build(h);   // the clover blocks follow the links
    return WD_OK;
}

int wd_gauge_unitarity(wd_handle* h, double* max_unitarity_dev, double* max_det_dev) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    if (max_unitarity_dev) *max_unitarity_dev = h->unit_dev;
    if (max_det_dev) *max_det_dev = h->det_dev;
    return WD_OK;
}

int wd_set_arith(wd_handle* h, int bits) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (bits != 16 && bits != 32) return fail(h, WD_ERR_INVALID_ARG, "wd_set_arith: bits must be 16 or 32, got %d", bits);
    const int a16 = bits == 16 ? 1 : 0;
    if (a16 != h->arith16) {
        h->arith16 = a16;
        h->gen += 1;   // captured solver graphs hold the other kernels
    }
    return WD_OK;
}

int wd_get_arith(const wd_handle* h) { return h ? (h->arith16 ? 16 : 32) : 0; }

int wd_timeline_set(void* blocks, void* phases) {
#ifdef WD_TIMELINE
    int bad = 0;
    for (auto f : wd::tl::units()) bad |= f(blocks, phases);
    return bad ? WD_ERR_CUDA : WD_OK;
#else
    (void)blocks;
    (void)phases;
    return WD_ERR_INVALID_ARG;
#endif
}

int wd_set_wait_limit(wd_handle* h, long long rounds) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (rounds >= (1LL << 31)) return fail(h, WD_ERR_INVALID_ARG, "wd_set_wait_limit: at most 2^31 - 1 rounds");
    const unsigned w = rounds < 0 ? 0u : (unsigned)rounds + 1u;
    if (w != h->wait_rounds) {
        h->wait_rounds = w;
        h->gen += 1;   // captured solver graphs hold the old limit
    }
    return WD_OK;
}

size_t wd_vector_bytes(const wd_handle* h, int prec) {
    if (!h || !valid_prec(prec)) return 0;
    return vec_bytes(h, prec);
}

int wd_pack(wd_handle* h, int prec, int parity, const double* lex, void* packed, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || (parity != 0 && parity != 1) || !lex || !packed)
        return fail(h, WD_ERR_INVALID_ARG, "wd_pack: bad argument");
    cudaError_t e = by_prec(prec, [&](auto tag) {
        typedef typename decltype(tag)::type T;
        return Ops<T>::pack(h->g, parity, lex, (uint4*)packed, (cudaStream_t)stream);
    });
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, "wd_pack");
}

int wd_unpack(wd_handle* h, int prec, int parity, const void* packed, double* lex, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || (parity != 0 && parity != 1) || !lex || !packed)
        return fail(h, WD_ERR_INVALID_ARG, "wd_unpack: bad argument");
    cudaError_t e = by_prec(prec, [&](auto tag) {
        typedef typename decltype(tag)::type T;
        return Ops<T>::unpack(h->g, parity, (const uint4*)packed, lex, (cudaStream_t)stream);
    });
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, "wd_unpack");
}

// The operators of wd_apply on nrhs packed vectors stored back to back.
static int apply_n(wd_handle* h, int prec, int recon, int op, int nrhs, const void* in, void* out, void* stream,
                   const char* who) {
    if (!valid_prec(prec) || !valid_recon(recon) || op < WD_OP_HOP_EO || op > WD_OP_FULL || !in || !out ||
        nrhs < 1)
        return fail(h, WD_ERR_INVALID_ARG, "%s: bad argument", who);
    if (in == out) return fail(h, WD_ERR_INVALID_ARG, "%s: in and out must not overlap", who);
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "%s: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators", who);
    const uint4 *le, *lo;
    int rc = ensure_links(h, prec, recon, &le, &lo);
    if (rc != WD_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t half = vec_bytes(h, prec);
    const long long vsu = (long long)spinor_units(prec) * h->g.Vh;   // units of one parity vector
    HopParams P{};
    P.g = h->g;
    P.rc.partials = nullptr;
    P.rc.ticket = nullptr;
    P.rc.st = nullptr;
    P.rc.stage = ST_NONE;
    P.nrhs = nrhs;
    P.vs = op == WD_OP_FULL ? 2 * vsu : vsu;
    P.guard = nullptr;
    P.guard_kind = GUARD_NONE;
    apply_tuning(h, prec, recon, P);
    const double k = h->kappa;
    const uint4 *ci_e = nullptr, *ci_o = nullptr, *cf_e = nullptr, *cf_o = nullptr;
    if (h->have_clover && (op == WD_OP_EO_A || op == WD_OP_FULL)) {
        if ((rc = ensure_clover(h, prec, op == WD_OP_EO_A ? 0 : 1, op == WD_OP_EO_A ? &ci_e : &cf_e,
                                op == WD_OP_EO_A ? &ci_o : &cf_o)) != WD_OK)
            return rc;
    }
    auto hop = [&](int parity, const void* src, void* dst, int epi, double a, double b, const void* y,
                   const uint4* mat = nullptr) {
        P.mat = mat;
        P.parity = parity;
        P.links = parity == 0 ? le : lo;
        P.in = (const uint4*)src;
        P.out = (uint4*)dst;
        P.y = (const uint4*)y;
        P.z = nullptr;
        P.a = a;
        P.b = b;
        P.c = 0.0;
        return by_prec(prec, [&](auto tag) {
            typedef typename decltype(tag)::type T;
            return Ops<T>::hop(recon, epi, RED_NONE, P, s);
        });
    };
    cudaError_t e = cudaSuccess;
    switch (op) {
    case WD_OP_HOP_EO: e = hop(0, in, out, EPI_H, 1.0, 0.0, nullptr); break;
    case WD_OP_HOP_OE: e = hop(1, in, out, EPI_H, 1.0, 0.0, nullptr); break;
    case WD_OP_EO_A: {   // with clover: in - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe in (Eq. 4)
        void* tmp = workspace(h, "apply.tmp." + std::to_string(prec), half * (size_t)nrhs);
        if (!tmp) return fail(h, WD_ERR_CUDA, "out of device memory");
        e = hop(1, in, tmp, EPI_H, 1.0, 0.0, nullptr, ci_o);
        if (e == cudaSuccess) e = hop(0, tmp, out, EPI_Y, -k * k, 1.0, in, ci_e);
        break;
    }
    case WD_OP_FULL: {   // with clover: C in - kappa H in on both parities
        const char* ie = (const char*)in;
        char* oe = (char*)out;
        const void* ye = ie;
        const void* yo = ie + half;
        if (cf_e) {   // out = C in first, then the hop adds to it in place
            e = by_prec(prec, [&](auto tag) {
                typedef typename decltype(tag)::type T;
                cudaError_t r2 = Ops<T>::apply_mat(h->g.Vh, nrhs, 2 * vsu, cf_e, (const uint4*)ie, (uint4*)oe, s);
                if (r2 == cudaSuccess)
                    r2 = Ops<T>::apply_mat(h->g.Vh, nrhs, 2 * vsu, cf_o, (const uint4*)(ie + half),
                                           (uint4*)(oe + half), s);
                return r2;
            });
            ye = oe;
            yo = oe + half;
        }
        if (e == cudaSuccess) e = hop(0, ie + half, oe, EPI_Y, -k, 1.0, ye);
        if (e == cudaSuccess) e = hop(1, ie, oe + half, EPI_Y, -k, 1.0, yo);
        break;
    }
    }
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, who);
}

int wd_apply(wd_handle* h, int prec, int recon, int op, const void* in, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    return apply_n(h, prec, recon, op, 1, in, out, stream, "wd_apply");
}

int wd_apply_batch(wd_handle* h, int prec, int recon, int op, int nrhs, const void* in, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (nrhs < 1 || nrhs > 1024) return fail(h, WD_ERR_INVALID_ARG, "wd_apply_batch: nrhs must be 1..1024");
    return apply_n(h, prec, recon, op, nrhs, in, out, stream, "wd_apply_batch");
}

int wd_set_rhs_per_thread(wd_handle* h, int recon, int k_plain, int k_reducing, int links_smem) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_recon(recon) || k_plain < 1 || k_plain > 12 || k_reducing < 1 || k_reducing > 12 ||
        (links_smem != 0 && links_smem != 1))
        return fail(h, WD_ERR_INVALID_ARG, "wd_set_rhs_per_thread: bad argument");
    const int ri = recon == 12 ? 0 : 1;
    h->tune_rhs[ri][0] = k_plain;
    h->tune_rhs[ri][1] = k_reducing;
    h->tune_rhs_smem[ri][0] = h->tune_rhs_smem[ri][1] = links_smem;
    h->gen += 1;   // captured solver graphs hold the old kernels
    return WD_OK;
}

const char* wd_status_string(int status) {
    switch (status) {
    case WD_OK: return "WD_OK";
    case WD_ERR_INVALID_ARG: return "WD_ERR_INVALID_ARG";
    case WD_ERR_CUDA: return "WD_ERR_CUDA";
    case WD_ERR_NOT_SU3: return "WD_ERR_NOT_SU3";
    case WD_ERR_NOT_CONVERGED: return "WD_ERR_NOT_CONVERGED";
    case WD_ERR_BREAKDOWN: return "WD_ERR_BREAKDOWN";
    case WD_ERR_NONFINITE: return "WD_ERR_NONFINITE";
    case WD_ERR_TIMEOUT: return "WD_ERR_TIMEOUT";
    case WD_ERR_NO_GAUGE: return "WD_ERR_NO_GAUGE";
    default: return "WD_ERR_UNKNOWN";
    }
}

const char* wd_last_error(const wd_handle* h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
