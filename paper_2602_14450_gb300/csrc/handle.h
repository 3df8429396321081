// Internal state behind the opaque wd_handle of the C ABI.
#pragma once

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/wd.h"
#include "kernels.h"

struct GraphKey {
    int prec, recon, scale_pass, iters, nrhs;
    long long gen;
    bool operator<(const GraphKey& o) const {
        if (prec != o.prec) return prec < o.prec;
        if (recon != o.recon) return recon < o.recon;
        if (scale_pass != o.scale_pass) return scale_pass < o.scale_pass;
        if (iters != o.iters) return iters < o.iters;
        if (nrhs != o.nrhs) return nrhs < o.nrhs;
        return gen < o.gen;
    }
};

struct Buffer {
    void* p = nullptr;
    size_t bytes = 0;
};

struct wd_handle {
    wd::Geom g{};
    double kappa = 0.0;
    int device = 0;
    std::string err;

    double* U64 = nullptr;             // FP64 links, host layout, on the device
    bool have_gauge = false;
    double unit_dev = -1.0, det_dev = -1.0;
    uint4* links[4][2][2] = {};        // [prec][recon 12 -> 0, 18 -> 1][output parity]

    std::map<std::string, Buffer> ws; // named device workspaces
    long long gen = 0;                 // bumped whenever a workspace moves
    int cap_rhs = 0;                   // right-hand sides the state arrays hold
    wd::SolverState* st = nullptr;     // device scalar state, one per right-hand side
    wd::SolverState* hst = nullptr;    // pinned host mirror
    int* hflag = nullptr;              // mapped pinned host word: "some right-hand side still iterating",
                                       // written by the last kernel of each inner-iteration graph launch
    int* dflag = nullptr;              // its device address
    double* partials = nullptr;        // reduction partials, RED_STRIDE per right-hand side
    unsigned* ticket = nullptr;        // reduction tickets, one per right-hand side
    cudaStream_t cap = nullptr;        // capture stream
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    std::map<GraphKey, cudaGraphExec_t> graphs;

    bool have_precond = false;         // weights of the learned preconditioner loaded
    long long adam_t = 0;              // Adam steps taken on those weights

    double csw = 0.0;                  // clover coefficient of wd_set_clover (0: plain Wilson)
    bool have_clover = false;
    uint4* clov[2][4][2] = {};         // clover blocks [C^-1 (chiral packing), C (full)][prec][parity], on first use
    uint4* clov_inv64[2] = {};         // full FP64 C^-1 per parity, the source of the chiral packings

    // hop kernel chosen by wd_tune per [prec][recon 12 -> 0, 18 -> 1][without / with fused reduction]; 0 = default
    int tune_variant[4][2][2] = {};
    int tune_block[4][2][2] = {};
    // FP16-arithmetic hop chosen by wd_tune: right-hand sides per thread and links in shared memory
    int tune_rhs[2][2] = {};
    int tune_rhs_smem[2][2] = {};
    int tune_spt[2] = {};              // ... sites per thread of the plain FP16-arithmetic hop

    int arith16 = 0;                   // wd_set_arith: FP16-storage hops sum in FP16 arithmetic

    unsigned wait_rounds = 0;          // wd_set_wait_limit: rounds of a bounded device wait + 1; 0 = the default

    int dd_grid[4] = {1, 1, 1, 1};     // wd_dd_set_partition: processes per direction
    int dd_coords[4] = {0, 0, 0, 0};   // ... and this sub-lattice's place among them
};

namespace wd {

int fail(wd_handle* h, int code, const char* fmt, ...);
int cuda_fail(wd_handle* h, cudaError_t e, const char* what);
// Device buffer `name` of at least `bytes` (reallocated, and gen bumped, when too small).
void* workspace(wd_handle* h, const std::string& name, size_t bytes);
// Scalar state, partials and tickets for `nrhs` right-hand sides.
int ensure_solver_state(wd_handle* h, int nrhs);
int ensure_links(wd_handle* h, int prec, int recon, const uint4** even, const uint4** odd);
size_t vec_bytes(const wd_handle* h, int prec);
RedCtx red_ctx(wd_handle* h, int stage);
// Clover blocks (clover.cu): rebuild from the gauge field; fetch kind 0 (C^-1)
// or 1 (C) in a precision (null pointers without a clover term).
int clover_build(wd_handle* h);
int ensure_clover(wd_handle* h, int prec, int kind, const uint4** even, const uint4** odd);
// 1 + 12 |c_sw| kappa bounds the norm of every clover block C.
inline double clover_bound(const wd_handle* h) { return h->have_clover ? 1.0 + 12.0 * std::fabs(h->csw) * h->kappa : 1.0; }
// Hop kernel configuration chosen by wd_tune for (prec, recon), if any, and
// the arithmetic of FP16 hops chosen by wd_set_arith.
inline void apply_tuning(const wd_handle* h, int prec, int recon, HopParams& P) {
    for (int f = 0; f < 2; ++f) {
        P.variant[f] = h->tune_variant[prec][recon == 12 ? 0 : 1][f];
        P.block[f] = h->tune_block[prec][recon == 12 ? 0 : 1][f];
    }
    P.arith16 = (prec == WD_FP16 && h->arith16) ? 1 : 0;
    P.wait_rounds = h->wait_rounds;
    for (int f = 0; f < 2; ++f) {
        P.rhs_group[f] = P.arith16 ? h->tune_rhs[recon == 12 ? 0 : 1][f] : 0;
        P.rhs_smem[f] = P.arith16 ? h->tune_rhs_smem[recon == 12 ? 0 : 1][f] : 0;
    }
    P.spt = P.arith16 ? h->tune_spt[recon == 12 ? 0 : 1] : 0;
}

}  // namespace wd

#define WD_CUDA(h, call)                                            \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return wd::cuda_fail((h), e_, #call); \
    } while (0)

namespace wd {

template <typename T> struct Tag { typedef T type; };

// Call f(Tag<storage type>) for a wd_prec value.
template <typename F>
cudaError_t by_prec(int prec, F&& f) {
    switch (prec) {
    case WD_FP64: return f(Tag<double>());
    case WD_FP32: return f(Tag<float>());
    case WD_FP16: return f(Tag<__half>());
    case WD_BF16: return f(Tag<__nv_bfloat16>());
    default: return cudaErrorInvalidValue;
    }
}

inline bool valid_prec(int p) { return p == WD_FP64 || p == WD_FP32 || p == WD_FP16 || p == WD_BF16; }
inline bool valid_recon(int r) { return r == 12 || r == 18; }

}  // namespace wd
