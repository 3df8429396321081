// wd_apply_eo_noalloc: the even-odd operator A of wd_apply(WD_OP_EO_A) for
// callers that must not allocate device memory.
//
// A p = p - kappa^2 H_eo H_oe p needs one odd-site intermediate vector. The
// ordinary entry point keeps that vector in a workspace it allocates with
// cudaMalloc on first use. Some callers cannot allow that: code that runs
// after its set-up phase under a framework's caching allocator that owns all
// device memory, or code whose streams must never see the implicit device
// synchronization that cudaMalloc / cudaFree can bring. This variant keeps the
// intermediate in a fixed array in the library's own device memory instead.
#include <mutex>

#include "handle.h"

namespace wd {

// Size limit of the intermediate: one odd-site vector of the chosen precision.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB

// The scratch array itself. Every GPU that loads the library holds it until
// the process exits; every call of wd_apply_eo_noalloc on a device shares it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the array per device. Host code must not pass the
// symbol itself to a kernel: on the host it names a stand-in, not device memory.
static void* scratch_address(int device, cudaError_t* err) {
    constexpr int MAX_DEV = 64;
    static std::mutex m;
    static void* addr[MAX_DEV] = {};
    *err = cudaSuccess;
    if (device < 0 || device >= MAX_DEV) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(m);
    if (!addr[device]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // the current device is `device`
        if (*err != cudaSuccess) return nullptr;
        addr[device] = p;
    }
    return addr[device];
}

}  // namespace wd

using namespace wd;

extern "C" int wd_apply_eo_noalloc(wd_handle* h, int prec, int recon, const void* in, void* out, void* stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!valid_prec(prec) || !valid_recon(recon) || !in || !out)
        return fail(h, WD_ERR_INVALID_ARG, "wd_apply_eo_noalloc: bad argument");
    if (in == out) return fail(h, WD_ERR_INVALID_ARG, "wd_apply_eo_noalloc: in and out must not overlap");
    if (!h->have_gauge) return fail(h, WD_ERR_NO_GAUGE, "wd_set_gauge has not been called");
    if (h->g.part) return fail(h, WD_ERR_INVALID_ARG, "wd_apply_eo_noalloc: a split lattice (wd_dd_set_partition) has only the wd_dd_* operators");
    const size_t need = vec_bytes(h, prec);
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(h, WD_ERR_INVALID_ARG,
                    "wd_apply_eo_noalloc: the odd-site intermediate needs %zu bytes, the fixed scratch holds %zu",
                    need, NOALLOC_SCRATCH_BYTES);
    const int ri = recon == 12 ? 0 : 1;
    const uint4* le = h->links[prec][ri][0];
    const uint4* lo = h->links[prec][ri][1];
    if (!le || !lo)
        return fail(h, WD_ERR_INVALID_ARG,
                    "wd_apply_eo_noalloc: links of this precision and format are not built yet (building them "
                    "allocates); call wd_apply or wd_solve with them once first");
    // With a clover term, A = 1 - kappa^2 C_ee^-1 H_eo C_oo^-1 H_oe (Eq. 4 with D_ee = C_ee, D_oo = C_oo): the
    // blocks C^-1 of this precision must exist already, since building them allocates.
    const uint4* ci_e = nullptr;
    const uint4* ci_o = nullptr;
    if (h->have_clover) {
        ci_e = h->clov[0][prec][0];
        ci_o = h->clov[0][prec][1];
        if (!ci_e || !ci_o)
            return fail(h, WD_ERR_INVALID_ARG,
                        "wd_apply_eo_noalloc: the clover blocks of this precision are not built yet (building them "
                        "allocates); call wd_apply(WD_OP_EO_A) or wd_solve with this precision once first");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    void* tmp = scratch_address(dev, &e);
    if (!tmp) return cuda_fail(h, e, "cudaGetSymbolAddress of the fixed scratch");

    HopParams P{};
    P.g = h->g;
    P.nrhs = 1;
    P.guard_kind = GUARD_NONE;
    apply_tuning(h, prec, recon, P);   // the kernel variant and block of wd_tune, and the FP16 arithmetic
    cudaStream_t s = (cudaStream_t)stream;
    const double k = h->kappa;
    auto hop = [&](int parity, const void* src, void* dst, int epi, double a, double b, const void* y,
                   const uint4* mat) {
        P.mat = mat;
        P.parity = parity;
        P.links = parity == 0 ? le : lo;
        P.in = (const uint4*)src;
        P.out = (uint4*)dst;
        P.y = (const uint4*)y;
        P.a = a;
        P.b = b;
        return by_prec(prec, [&](auto tag) {
            typedef typename decltype(tag)::type T;
            return Ops<T>::hop(recon, epi, RED_NONE, P, s);
        });
    };
    e = hop(1, in, tmp, EPI_H, 1.0, 0.0, nullptr, ci_o);                 // tmp = C_oo^-1 H_oe in (all of it)
    if (e == cudaSuccess) e = hop(0, tmp, out, EPI_Y, -k * k, 1.0, in, ci_e);  // out = in - kappa^2 C_ee^-1 H_eo tmp
    return e == cudaSuccess ? WD_OK : cuda_fail(h, e, "wd_apply_eo_noalloc");
}
