// First pass of the collapsed learned preconditioner on the 5th-generation
// tensor cores (tcgen05, kind::f16 with BF16 operands, FP32 accumulation in
// tensor memory).
//
// For every odd site y and colour a, the eight transports of the input,
// x[d1][t] = (T_{1+d1} psi)(y)_{t,a} (d1 = 0..7, spin t), are mixed into the
// eight intermediate fields phi_{1+d2}(y)_{s,a} = sum_{d1,t} V[1+d2][1+d1]_{st} x[d1][t].
// Written over the reals this is, per (site, colour) row, a 64-vector
// (d1, t, re/im) times a fixed 64 x 64 matrix -- a dense contraction of
// 3 * V/2 rows, K = 64, N = 64:
//   D[m][n] = sum_k A[m][k] B[n][k],  k = 8 d1 + 2 t + c,  n = 8 d2 + 2 s + c',
//   B = [[Re V, -Im V], [Im V, Re V]] in that index order.
// One CTA takes 128 odd sites: its 128 threads compute the transports (one site
// each, FP32 arithmetic) and write them, rounded to BF16, as three M = 128 x
// K = 64 operand tiles (one per colour); one thread issues the MMAs
// (M = 128, N = 64, 4 x K = 16 per colour) into 64 TMEM columns; each warp reads
// its 32 rows back (tcgen05.ld) and stores phi colour-major: unit a of field d2
// holds (s = 0..3, re/im) of colour a.
//
// Operand layout in shared memory: the no-swizzle K-major canonical form of
// 8-row x 16-byte core matrices. Element (m, k) of a tile with K = 64 sits at
// byte ((m / 8) * 8 + k / 8) * 128 + (m % 8) * 16 + (k % 8) * 2: the K-adjacent
// core-matrix stride (leading byte offset) is 128 and the M-adjacent one
// (stride byte offset) 1024; the K = 16 slice j starts 256 j bytes in.
//
// Every wait is bounded: on expiry the kernel raises *err, still waits (bounded)
// for its own MMAs, frees its tensor memory and returns.
#pragma once

#include <cstdint>

namespace wd {

namespace tc {

constexpr int TILE_M = 128;                  // sites per CTA tile
constexpr int K = 64, N = 64;                // real K and N of the contraction
constexpr int A_TILE_BYTES = TILE_M * K * 2; // one colour's operand tile (16 KB)
constexpr int B_BYTES = N * K * 2;           // 8 KB
constexpr int SMEM_BYTES = 3 * A_TILE_BYTES + B_BYTES + 64;
constexpr int TMEM_COLS = 64;
constexpr unsigned WAIT_LIMIT = 1u << 22;    // try_wait rounds before giving up (the default)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a no-swizzle K-major tile with K = 64.
__host__ __device__ constexpr uint32_t kmajor_offset(int row, int k) {
    return (uint32_t)(((row >> 3) * 8 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading (K-adjacent) and
// stride (M/N-adjacent) core-matrix offsets, version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                           ((uint32_t)(TILE_M >> 4) << 24);

// The same descriptor for another N (a multiple of 16 up to 256) at M = 128.
constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TILE_M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                         uint32_t idesc = IDESC) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Wait for the phase with the given parity to complete; false when `limit`
// try_wait rounds ran out (limit 0: give up at once, without a round).
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, unsigned limit = WAIT_LIMIT) {
    const uint32_t a = smem_addr(bar);
    for (unsigned i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

}  // namespace tc

// First pass (odd sites) of the collapsed M with the mixing on tensor cores.
// in_e: FP16 even-site input; phi: 8 BF16 odd-site fields (colour-major
// units), pvs units apart; links_o: FP16 12-real gathered links of the odd
// parity; V: collapsed spin weights [k2][k1][s][t]. Block size 128.
template <typename TIN, typename LT, int R>
__global__ void __launch_bounds__(128, 3) k_ptc_s1_tc(Geom g, const uint4* in_e, uint4* phi, long long pvs,
                                                      const uint4* links_o, const float2* V, const SolverState* guard,
                                                      int* err, unsigned wait_rounds) {
    // wait_rounds = the limit of the MMA waits + 1; 0 = the default limit
    const unsigned limit = wait_rounds ? wait_rounds - 1 : tc::WAIT_LIMIT;
    using namespace tc;
    if (guarded(guard, GUARD_INNER)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* A = smem;                              // 3 colour tiles
    unsigned char* B = smem + 3 * A_TILE_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(B + B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(B + B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;

    // B[n][k] from V: n = 8 d2 + 2 s + c', k = 8 d1 + 2 t + c.
    for (int i = tid; i < N * K; i += blockDim.x) {
        const int n = i / K, k = i % K;
        const int d2 = n >> 3, s = (n >> 1) & 3, co = n & 1;
        const int d1 = k >> 3, t = (k >> 1) & 3, ci = k & 1;
        const float2 v = V[((1 + d2) * 9 + 1 + d1) * 16 + 4 * s + t];
        const float val = co == 0 ? (ci == 0 ? v.x : -v.y) : (ci == 0 ? v.y : v.x);
        *reinterpret_cast<__nv_bfloat16*>(B + kmajor_offset(n, k)) = __float2bfloat16_rn(val);
    }
    if (tid == 0) {
        bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t a_base = smem_addr(A), b_base = smem_addr(B);
    uint32_t phase = 0;
    bool failed = false;

    const int ntiles = (g.Vh + TILE_M - 1) / TILE_M;
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int h = tile * TILE_M + tid;
        const bool ok = h < g.Vh;
        static_assert(R == 12 && sizeof(TIN) == 2 && sizeof(LT) == 2, "FP16 input, FP16 12-real links");
        // transports -> BF16 operand rows (zero rows past the end); each
        // direction's neighbour and link units are loaded one direction ahead
        int nbr[8];
        unsigned wm = 0;
        uint4 fu[2][3], lu[2][2];
        if (ok) {
            wm = site_neighbours(g, 1, h, nbr);
#pragma unroll
            for (int u = 0; u < 3; ++u) fu[0][u] = __ldg(in_e + (size_t)u * g.Vh + nbr[0]);
            load_link_units<LT>(links_o, g.Vh, h, 0, lu[0]);
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            float t[24];
            if (ok) {
                if (d + 1 < 8) {
#pragma unroll
                    for (int u = 0; u < 3; ++u) fu[(d + 1) & 1][u] = __ldg(in_e + (size_t)u * g.Vh + nbr[d + 1]);
                    load_link_units<LT>(links_o, g.Vh, h, d + 1, lu[(d + 1) & 1]);
                }
                float f[24], m[18];
#pragma unroll
                for (int u = 0; u < 3; ++u)
#pragma unroll
                    for (int i = 0; i < 8; ++i) f[8 * u + i] = Unit<TIN>::get(fu[d & 1][u], i);
                link_from_units<LT>(lu[d & 1], d, m);
                colour_mul(m, f, t);
                if (((wm >> d) & 1u) && g.bc[d >> 1] < 0) {
#pragma unroll
                    for (int i = 0; i < 24; ++i) t[i] = -t[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) t[i] = 0.f;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {   // k = 8 d + 2 s + c: spins 0..3 of colour a, (re, im)
                uint4 w;
                w.x = pack_bf16(t[2 * (0 + a)], t[2 * (0 + a) + 1]);
                w.y = pack_bf16(t[2 * (3 + a)], t[2 * (3 + a) + 1]);
                w.z = pack_bf16(t[2 * (6 + a)], t[2 * (6 + a) + 1]);
                w.w = pack_bf16(t[2 * (9 + a)], t[2 * (9 + a) + 1]);
                *reinterpret_cast<uint4*>(A + a * A_TILE_BYTES + kmajor_offset(tid, 8 * d)) = w;
            }
        }
        fence_proxy_async();
        fence_before();
        __syncthreads();
        fence_after();

#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            if (tid == 0) {
#pragma unroll
                for (int j = 0; j < K / 16; ++j) {
                    const uint64_t ad = smem_desc(a_base + a * A_TILE_BYTES + 256 * j, 128, 1024);
                    const uint64_t bd = smem_desc(b_base + 256 * j, 128, 1024);
                    tc::mma_bf16(tmem, ad, bd, j > 0 ? 1u : 0u);
                }
                mma_commit(bar);
            }
            const bool landed = bar_wait(bar, phase, limit);
            failed = __syncthreads_or(!landed);     // uniform across the CTA
            if (failed) {                           // `phase` stays the one still pending
                if (tid == 0 && err) atomicExch(err, 1);
                break;
            }
            phase ^= 1;
            fence_after();
            // every lane takes part in the aligned TMEM loads; rows past the end are not stored
#pragma unroll
            for (int d2 = 0; d2 < 8; ++d2) {
                float v[8];
                tmem_ld8(tmem + lane_base + 8 * d2, v);
                tmem_ld_wait();
                if (ok) {
                    uint4 w;
                    w.x = pack_bf16(v[0], v[1]);
                    w.y = pack_bf16(v[2], v[3]);
                    w.z = pack_bf16(v[4], v[5]);
                    w.w = pack_bf16(v[6], v[7]);
                    phi[(size_t)d2 * pvs + (size_t)a * g.Vh + h] = w;
                }
            }
            fence_before();
            __syncthreads();
            fence_after();
        }
    }
    if (failed && tid == 0) bar_wait(bar, phase);   // default bound: let an MMA still in flight finish
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Training: the odd-site half of a fan-out layer, H_c(y) = sum_{d,t} W[1+d][c]_{st}
// (T_{1+d} in)(y)_{t,a} for the 12 channels c, with the input on the even
// sites only (the forward layer 1 on v, and the adjoint of layer 2 on the loss
// gradient): the same contraction as the first pass of M with the channel
// mixing as B, per (site, colour) row K = 64 (d, t, re/im) against N = 96
// (c, s, re/im):
//   B = [[Re W, -Im W], [Im W, Re W]],  n = 8 c + 2 s + c',  k = 8 d + 2 t + c.
// FP32 input and 18-real FP32 links (the training precision), transports in
// FP32 rounded to BF16 operands, FP32 accumulation in 128 TMEM columns,
// written to H in FP32 (layout [c][parity][units][Vh], parity 1 here). The
// waits are bounded as in k_ptc_s1_tc.
namespace tcf {
constexpr int N = 96;
constexpr int B_BYTES = N * tc::K * 2;                                 // 12 KB
constexpr int SMEM_BYTES = 3 * tc::A_TILE_BYTES + B_BYTES + 64;
constexpr int TMEM_COLS = 128;
constexpr uint32_t IDESC = tc::idesc_bf16(N);
}  // namespace tcf

__global__ void __launch_bounds__(128) k_ptc_fanout_odd_tc(Geom g, const uint4* in_e, uint4* H, long long hvs,
                                                           const uint4* links_o, const float* w, int* err,
                                                           unsigned wait_rounds) {
    using namespace tc;
    const unsigned limit = wait_rounds ? wait_rounds - 1 : WAIT_LIMIT;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* A = smem;                              // 3 colour tiles
    unsigned char* Bt = smem + 3 * A_TILE_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bt + tcf::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(Bt + tcf::B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int i = tid; i < tcf::N * K; i += blockDim.x) {
        const int n = i / K, k = i % K;
        const int c = n >> 3, s = (n >> 1) & 3, co = n & 1;
        const int d = k >> 3, t = (k >> 1) & 3, ci = k & 1;
        const float* wp = w + 2 * (((1 + d) * PTC_C + c) * 16 + 4 * s + t);
        const float val = co == 0 ? (ci == 0 ? wp[0] : -wp[1]) : (ci == 0 ? wp[1] : wp[0]);
        *reinterpret_cast<__nv_bfloat16*>(Bt + kmajor_offset(n, k)) = __float2bfloat16_rn(val);
    }
    if (tid == 0) {
        bar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                     "r"(tcf::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const uint32_t a_base = smem_addr(A), b_base = smem_addr(Bt);
    uint32_t phase = 0;
    bool failed = false;

    const int ntiles = (g.Vh + TILE_M - 1) / TILE_M;
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int h = tile * TILE_M + tid;
        const bool ok = h < g.Vh;
        const Coord co = ok ? coord_of(g, 1, h) : Coord{};
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            float t[24];
            if (ok) {
                bool wrap;
                const int hn = neighbour(g, h, co, d, &wrap);
                float f[24], m[18];
                load_spinor<float>(in_e, g.Vh, hn, f);
                load_link<float, 18>(links_o, g.Vh, h, d, m);
                colour_mul(m, f, t);
                if (wrap && g.bc[d >> 1] < 0) {
#pragma unroll
                    for (int i = 0; i < 24; ++i) t[i] = -t[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) t[i] = 0.f;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {   // k = 8 d + 2 t + c: spins 0..3 of colour a, (re, im)
                uint4 u;
                u.x = pack_bf16(t[2 * (0 + a)], t[2 * (0 + a) + 1]);
                u.y = pack_bf16(t[2 * (3 + a)], t[2 * (3 + a) + 1]);
                u.z = pack_bf16(t[2 * (6 + a)], t[2 * (6 + a) + 1]);
                u.w = pack_bf16(t[2 * (9 + a)], t[2 * (9 + a) + 1]);
                *reinterpret_cast<uint4*>(A + a * A_TILE_BYTES + kmajor_offset(tid, 8 * d)) = u;
            }
        }
        fence_proxy_async();
        fence_before();
        __syncthreads();
        fence_after();

#pragma unroll 1
        for (int a = 0; a < 3; ++a) {
            if (tid == 0) {
#pragma unroll
                for (int j = 0; j < K / 16; ++j) {
                    const uint64_t ad = smem_desc(a_base + a * A_TILE_BYTES + 256 * j, 128, 1024);
                    const uint64_t bd = smem_desc(b_base + 256 * j, 128, 1024);
                    tc::mma_bf16(tmem, ad, bd, j > 0 ? 1u : 0u, tcf::IDESC);
                }
                mma_commit(bar);
            }
            const bool landed = bar_wait(bar, phase, limit);
            failed = __syncthreads_or(!landed);
            if (failed) {
                if (tid == 0 && err) atomicExch(err, 1);
                break;
            }
            phase ^= 1;
            fence_after();
            // every lane takes part in the aligned TMEM loads; rows past the end are not stored
#pragma unroll 1
            for (int c = 0; c < PTC_C; ++c) {
                float v[8];
                tmem_ld8(tmem + lane_base + 8 * c, v);
                tmem_ld_wait();
                if (ok) {
                    float* out = reinterpret_cast<float*>(H + (size_t)(2 * c + 1) * hvs);
#pragma unroll
                    for (int s = 0; s < 4; ++s) {   // (re, im) of spin s, colour a: reals 2 (3 s + a), + 1
                        const int i = 2 * (3 * s + a);
                        *reinterpret_cast<float2*>(out + ((size_t)(i >> 2) * g.Vh + h) * 4 + (i & 3)) =
                            make_float2(v[2 * s], v[2 * s + 1]);
                    }
                }
            }
            fence_before();
            __syncthreads();
            fence_after();
        }
    }
    if (failed && tid == 0) bar_wait(bar, phase);   // default bound: let an MMA still in flight finish
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tcf::TMEM_COLS)
                     : "memory");
}

}  // namespace wd
