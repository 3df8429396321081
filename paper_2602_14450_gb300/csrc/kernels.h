// Host-side launchers of the device kernels, one instantiation per storage
// type (translation units ops_f64.cu, ops_f32.cu, ops_f16.cu, ops_bf16.cu).
//
// Every vector argument may hold a batch of `nrhs` right-hand sides stored
// back to back: right-hand side r of a packed parity vector starts `vs`
// 16-byte units after right-hand side r - 1 (vs = units per site * V/2 for a
// tightly packed batch). Scalar state, reduction partials and tickets are
// arrays over right-hand sides (see RedCtx).
#pragma once

#include "common.cuh"

namespace wd {

enum Epi { EPI_H = 0, EPI_Y = 1, EPI_YZ = 2 };
enum Red { RED_NONE = 0, RED_RSV = 1, RED_TS = 2, RED_NORM = 3 };
// Rescaling of r in the x/r-update kernel k_xr (Alg. 4): none, norms for a separate k_scale pass, or fused.
enum XrMode { XR_PLAIN = 0, XR_NORMS = 1, XR_FUSED = 2 };

struct HopParams {
    Geom g;
    int parity;             // parity of the output sites
    int nrhs;               // right-hand sides in the batch (>= 1)
    long long vs;           // units between right-hand sides of every spinor argument
    const uint4* links;     // gathered links of the output parity (shared by all rhs)
    const uint4* in;        // input spinor on parity 1 - parity
    uint4* out;             // output spinor on `parity`
    const uint4* y;         // epilogue operands on `parity`
    const uint4* z;
    const uint4* rstar;     // RED_RSV: sum conj(rstar) out
    double a, b, c;         // out = a * H in + b * y + c * z
    RedCtx rc;              // reduction target (partials, ticket, state, stage)
    const SolverState* guard;  // per-rhs state consulted by the guard
    int guard_kind;            // GuardKind
    int* err;                  // set to 1 by a kernel whose bounded wait gave up (may be null)
    const uint4* mat;          // site-local 12 x 12 complex block of the output parity (chiral packing,
                               // storage T) applied to the hop: out = M (a H in) + b y + c z; null = none
    int variant[2];            // kernel variant (hop_variant() numbering) without / with a fused
                               // reduction; 0 = the process default
    int block[2];              // threads per block, likewise; 0 = the process default
    int arith16;               // FP16 storage only: 1 = the hopping sum in FP16 arithmetic (hop16_kernel)
    int acc_exp;               // hop16_kernel: exponent of its accumulator scale (set by the launcher)
    unsigned wait_rounds;      // limit of a bounded device wait + 1 (wd_set_wait_limit); 0 = the default limit
    int rhs_group[2];          // FP16 arithmetic: right-hand sides per thread (hop16m_kernel) without / with a
                               // fused reduction; 0 or 1 = one (hop16_kernel); must divide nrhs to be used
    int rhs_smem[2];           // ... and 1 = the site's links in shared memory instead of registers
    int spt;                   // FP16 arithmetic, plain hop: sites per thread (grid-stride; 0 or 1 = one site)
};

// Largest number of blocks a reducing kernel uses per right-hand side.
constexpr int MAX_RED_BLOCKS = 8192;
constexpr int MAX_RED_SUMS = 4;
static_assert(MAX_RED_BLOCKS * MAX_RED_SUMS == RED_STRIDE, "partials layout");

// Units of 16 bytes per site of the gathered links of one parity.
int link_units(int prec, int recon);
// Units of 16 bytes per site of a spinor.
int spinor_units(int prec);

// Vector kernels: n = sites per parity, vs = units between right-hand sides
// (vs64 for FP64 vectors), st = state array, g = guard kind.
template <typename T> struct Ops {
    static cudaError_t hop(int recon, int epi, int red, const HopParams& P, cudaStream_t s);
    static cudaError_t pupdate(int n, int nrhs, long long vs, uint4* p, const uint4* v, const uint4* r,
                               const SolverState* st, cudaStream_t s);
    static cudaError_t supdate(int n, int nrhs, long long vs, uint4* r, const uint4* v, const SolverState* st,
                               cudaStream_t s);
    // mode: XrMode
    static cudaError_t xr(int mode, int n, int nrhs, long long vs, uint4* x, uint4* r, const uint4* p,
                          const uint4* t, const uint4* rstar, const uint4* xr_src, const uint4* xp_src,
                          SolverState* st, RedCtx rc, cudaStream_t s);
    static cudaError_t scale(int n, int nrhs, long long vs, uint4* r, uint4* x, const uint4* rstar, SolverState* st,
                             RedCtx rc, cudaStream_t s);
    static cudaError_t rescale_in(int n, int nrhs, long long vs, long long vs64, const uint4* r64, uint4* r,
                                  uint4* rstar, int ftz, SolverState* st, RedCtx rc, cudaStream_t s);
    static cudaError_t correct(int n, int nrhs, long long vs, long long vs64, uint4* x64, const uint4* xt,
                               const SolverState* st, cudaStream_t s);
    static cudaError_t norm2(int n, int nrhs, long long vs, const uint4* v, RedCtx rc, int guard_kind,
                             cudaStream_t s);
    // xo = eta + kappa t and the sum of |eta - xo + kappa t|^2 (Eq. 5 with t = H_oe xi_e)
    static cudaError_t odd_reconstruct(int n, int nrhs, long long vs, double kappa, const uint4* eta, const uint4* t,
                                       uint4* xo, RedCtx rc, cudaStream_t s);
    // out = M in, site by site, for every right-hand side (M: 12 x 12 complex blocks, storage T)
    static cudaError_t apply_mat(int n, int nrhs, long long vs, const uint4* mat, const uint4* in, uint4* out,
                                 cudaStream_t s);
    // blocks of storage T from FP64 blocks (288 reals per site, n sites)
    static cudaError_t mat_from64(int n, const uint4* src64, uint4* dst, cudaStream_t s);
    // out = M in with M in the chiral packing (80 reals per site, see mat_mul_chiral)
    static cudaError_t apply_chiral(int n, int nrhs, long long vs, const uint4* mat, const uint4* in, uint4* out,
                                    cudaStream_t s);
    // chiral packing in storage T from full FP64 blocks that commute with gamma_5
    static cudaError_t chiral_from64(int n, const uint4* src64, uint4* dst, cudaStream_t s);
    static cudaError_t pack(const Geom& g, int parity, const double* lex, uint4* out, cudaStream_t s);
    static cudaError_t unpack(const Geom& g, int parity, const uint4* in, double* lex, cudaStream_t s);
    static cudaError_t build_links(int recon, const Geom& g, int parity, const double* U, uint4* out, cudaStream_t s);
};

cudaError_t launch_unitarity(int nlinks, const double* U, unsigned long long* out, cudaStream_t s);

// Block size of every vector kernel; the hop kernels take theirs from
// HopParams::block (set by wd_tune) or else hop_block() (environment
// WD_HOP_BLOCK = 64 or 128, default 128).
constexpr int VEC_BLOCK = 256;
int hop_block();
void set_hop_block(int b);
// Hop kernel variant, read once from the environment variable WD_HOP_KERNEL:
// 4 = one site per thread, neighbour and link loads issued one direction
// ahead (default); 1 = one site per thread without the look-ahead; for
// FP32-arithmetic storage 2 = two sites per thread with packed FP32x2 math;
// for 16-bit storage 3 = tiles staged in shared memory by bulk copies and,
// with 12-real links, 5 = persistent threads streaming their operands through
// a per-thread two-slot ring of asynchronous copies in shared memory.
int hop_variant();
// Directions ahead that the FP16-arithmetic hop loads its neighbour spinors
// (environment WD_HOP16_AHEAD = 1 or 2, default 2: 3% faster at 32^3 x 64).
int hop16_ahead();
int num_sms();

}  // namespace wd
