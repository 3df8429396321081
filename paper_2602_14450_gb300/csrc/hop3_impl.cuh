// Hopping term (Eq. 1) for 16-bit storage with FP32 arithmetic, staged in
// shared memory by bulk asynchronous copies (1-D TMA).
//
// The output sites are cut into tiles of TR consecutive EO rows (x-lines) at
// fixed (z, t), with TR dividing Ly, so that every neighbour of a tile lies in
// one of five row blocks of the input vector:
//   block 0: rows y0-1 .. y0+TR (the tile's own rows plus one halo row on each
//            side, wrapped in y) at (z, t)       -> x and y neighbours
//   block 1: rows y0 .. y0+TR-1 at (z+1, t)      -> +z neighbours
//   block 2: the same rows at (z-1, t)           -> -z neighbours
//   block 3: the same rows at (z, t+1)           -> +t neighbours
//   block 4: the same rows at (z, t-1)           -> -t neighbours
// Each block is one or three contiguous runs of the packed input, copied unit
// plane by unit plane with cp.async.bulk; the tile's gathered links (one
// contiguous run per unit plane) are copied the same way. One thread issues
// the copies, an mbarrier counts their bytes, every thread waits (bounded)
// and then computes two output sites, i and i + TS/2 of the tile, with packed
// FP32x2 arithmetic (the math of hop2_impl.cuh) from shared memory.
#pragma once

#include "hop2_impl.cuh"

namespace wd {

// Tiling of one launch (host computed).
struct StageGeom {
    int TR;          // rows per tile (divides Ly)
    int TS;          // sites per tile = TR * Lxh (even)
    int ntiles;      // Vh / TS
    int nrows;       // 5 * TR + 2 rows of input staged per tile
    int spin_units;  // spinor unit planes per row block (24 reals / unit size)
    int link_units;  // link unit planes per site
    unsigned bytes;  // bytes copied per tile
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into shared memory.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Wait for the phase of the tile; false after `limit` rounds (the default is
// about a second; 0 gives up at once).
constexpr unsigned MBAR_WAIT_LIMIT = 1u << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned phase, unsigned limit = MBAR_WAIT_LIMIT) {
    for (unsigned i = 0; i < limit; ++i) {
        if (mbar_test(bar, phase)) return true;
        __nanosleep(64);
    }
    return false;
}

template <typename T, int R, int EPI, int RED>
__global__ void __launch_bounds__(128) hop3_kernel(const HopParams P, const StageGeom sg, int* err) {
    pdl_begin();
    typedef LinkFmt<T, R> LF;
    constexpr int NS = RedSums<RED>::N;
    constexpr float SC = Wide<T>::SCALE;
    extern __shared__ __align__(128) uint4 smem[];
    __shared__ __align__(8) uint64_t bar;

    const Slice sl = slice_of(P.nrhs);
    if (guarded(P.guard ? P.guard + sl.rhs : nullptr, P.guard_kind)) return;
    const long long ro = (long long)sl.rhs * P.vs;
    const uint4* vin = P.in + ro;
    uint4* vout = P.out + ro;
    const uint4* vy = P.y ? P.y + ro : nullptr;
    const uint4* vz = P.z ? P.z + ro : nullptr;
    const uint4* vrs = P.rstar ? P.rstar + ro : nullptr;

    const Geom& g = P.g;
    const int p = P.parity;
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3], Lxh = g.Lxh, Vh = g.Vh;
    const int TR = sg.TR, TS = sg.TS, half = TS >> 1;
    const int plane_in = sg.nrows * Lxh;      // units of one staged spinor plane
    uint4* s_in = smem;                       // [spin_units][nrows * Lxh]
    uint4* s_lk = smem + (size_t)sg.spin_units * plane_in;   // [link_units][TS]

    const float2 A2 = f2((float)P.a, (float)P.a);
    const float2 B2 = f2((float)P.b * SC, (float)P.b * SC);
    const float2 C2 = f2((float)P.c * SC, (float)P.c * SC);
    const float2 SC2 = f2(SC, SC);
    float part[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) part[k] = 0.f;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    unsigned phase = 0;
    for (int tile = sl.b; tile < sg.ntiles; tile += sl.nb, phase ^= 1u) {
        const int row0 = tile * TR;                   // first EO row of the tile
        const int y0 = row0 % Ly;
        const int zt = row0 / Ly;
        const int z = zt % Lz, t = zt / Lz;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar, sg.bytes);
            const int zp = (z + 1) % Lz, zm = (z + Lz - 1) % Lz, tp = (t + 1) % Lt, tm = (t + Lt - 1) % Lt;
            const int rbase[4] = {(t * Lz + zp) * Ly + y0, (t * Lz + zm) * Ly + y0, (tp * Lz + z) * Ly + y0,
                                  (tm * Lz + z) * Ly + y0};
            const int ylo = (y0 + Ly - 1) % Ly, yhi = (y0 + TR) % Ly;
            const int rself = (t * Lz + z) * Ly;
            const unsigned rowb = (unsigned)Lxh * 16u;
            for (int u = 0; u < sg.spin_units; ++u) {
                const uint4* src = vin + (size_t)u * Vh;
                uint4* dst = s_in + (size_t)u * plane_in;
                bulk_copy(dst, src + (size_t)(rself + ylo) * Lxh, rowb, &bar);
                bulk_copy(dst + Lxh, src + (size_t)(rself + y0) * Lxh, rowb * TR, &bar);
                bulk_copy(dst + (size_t)(TR + 1) * Lxh, src + (size_t)(rself + yhi) * Lxh, rowb, &bar);
                for (int b = 0; b < 4; ++b)
                    bulk_copy(dst + (size_t)(TR + 2 + b * TR) * Lxh, src + (size_t)rbase[b] * Lxh, rowb * TR, &bar);
            }
            for (int k = 0; k < sg.link_units; ++k)
                bulk_copy(s_lk + (size_t)k * TS, P.links + (size_t)k * Vh + (size_t)row0 * Lxh, (unsigned)TS * 16u,
                          &bar);
        }
        const bool landed = mbar_wait(&bar, phase, P.wait_rounds ? P.wait_rounds - 1 : MBAR_WAIT_LIMIT);
        if (__syncthreads_or(!landed)) {              // uniform across the block
            if (threadIdx.x == 0 && err) atomicExch(err, 1);
            mbar_wait(&bar, phase);                   // default bound: let the copies land before the block goes on
            break;                                    // still takes its part in the grid reduction below
        }

        for (int i = threadIdx.x; i < half; i += blockDim.x) {
            const int la = i, lb = i + half;          // tile-local sites
            const int ra = la / Lxh, rb = lb / Lxh;   // tile-local rows
            const int xha = la - ra * Lxh, xhb = lb - rb * Lxh;
            const int ya = y0 + ra, yb = y0 + rb;
            const int xa = 2 * xha + ((p + ya + z + t) & 1);
            const int xb = 2 * xhb + ((p + yb + z + t) & 1);
            float2 acc[24];
#pragma unroll
            for (int q = 0; q < 24; ++q) acc[q] = f2(0.f, 0.f);
#pragma unroll
            for (int grp = 0; grp < 8 / LF::G; ++grp) {
                uint4 lka[LF::GROUP_UNITS], lkb[LF::GROUP_UNITS];
#pragma unroll
                for (int k = 0; k < LF::GROUP_UNITS; ++k) {
                    lka[k] = s_lk[(size_t)(grp * LF::GROUP_UNITS + k) * TS + la];
                    lkb[k] = s_lk[(size_t)(grp * LF::GROUP_UNITS + k) * TS + lb];
                }
#pragma unroll
                for (int j = 0; j < LF::G; ++j) {
                    const int d = grp * LF::G + j;
                    const int mu = d >> 1;
                    const bool fwd = (d & 1) == 0;
                    int na, nb;                       // staged-row site indices
                    bool wa, wb;
                    if (mu == 0) {
                        wa = fwd ? (xa == Lx - 1) : (xa == 0);
                        wb = fwd ? (xb == Lx - 1) : (xb == 0);
                        const int xna = fwd ? (wa ? 0 : xa + 1) : (wa ? Lx - 1 : xa - 1);
                        const int xnb = fwd ? (wb ? 0 : xb + 1) : (wb ? Lx - 1 : xb - 1);
                        na = (ra + 1) * Lxh + (xna >> 1);
                        nb = (rb + 1) * Lxh + (xnb >> 1);
                    } else if (mu == 1) {
                        wa = fwd ? (ya == Ly - 1) : (ya == 0);
                        wb = fwd ? (yb == Ly - 1) : (yb == 0);
                        na = (ra + (fwd ? 2 : 0)) * Lxh + xha;
                        nb = (rb + (fwd ? 2 : 0)) * Lxh + xhb;
                    } else {
                        const int blk = mu == 2 ? (fwd ? 0 : 1) : (fwd ? 2 : 3);
                        const int c = mu == 2 ? z : t;
                        const int L = mu == 2 ? Lz : Lt;
                        wa = wb = fwd ? (c == L - 1) : (c == 0);
                        na = (TR + 2 + blk * TR + ra) * Lxh + xha;
                        nb = (TR + 2 + blk * TR + rb) * Lxh + xhb;
                    }
                    const float pha = (wa && g.bc[mu] < 0) ? -SC : SC;
                    const float phb = (wb && g.bc[mu] < 0) ? -SC : SC;
                    float2 nbp[24];
                    constexpr int N = Wide<T>::N;
#pragma unroll
                    for (int u = 0; u < 24 / N; ++u) {
                        const uint4 wau = s_in[(size_t)u * plane_in + na];
                        const uint4 wbu = s_in[(size_t)u * plane_in + nb];
#pragma unroll
                        for (int q = 0; q < N; ++q) nbp[u * N + q] = f2(Wide<T>::get(wau, q), Wide<T>::get(wbu, q));
                    }
                    float2 hs[12], chi[12];
                    project2(mu, fwd, nbp, f2(pha, phb), hs);
                    link_mul2<T, R>(lka, lkb, j * R, hs, chi);
                    reconstruct2(mu, fwd, chi, acc);
                }
            }
            const int ha = row0 * Lxh + la, hb = row0 * Lxh + lb;   // output sites
            float2 o[24];
#pragma unroll
            for (int q = 0; q < 24; ++q) o[q] = mul2(A2, acc[q]);
            float2 yv[24];
            if constexpr (EPI >= EPI_Y) {
                load_pair<T>(vy, Vh, ha, hb, yv);
#pragma unroll
                for (int q = 0; q < 24; ++q) o[q] = fma2(B2, yv[q], o[q]);
            }
            if constexpr (EPI >= EPI_YZ) {
                float2 zv[24];
                load_pair<T>(vz, Vh, ha, hb, zv);
#pragma unroll
                for (int q = 0; q < 24; ++q) o[q] = fma2(C2, zv[q], o[q]);
            }
            store_pair<T>(vout, Vh, ha, hb, o, P.guard != nullptr && P.guard[sl.rhs].ftz);
            if constexpr (RED == RED_RSV) {
                float2 rs[24];
                load_pair<T>(vrs, Vh, ha, hb, rs);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float2 rr = mul2(rs[2 * q], SC2), ri = mul2(rs[2 * q + 1], SC2);
                    const float2 re = fma2(ri, o[2 * q + 1], mul2(rr, o[2 * q]));
                    const float2 im = fma2(neg2(ri), o[2 * q], mul2(rr, o[2 * q + 1]));
                    part[0] += re.x + re.y;
                    part[1] += im.x + im.y;
                }
            } else if constexpr (RED == RED_TS) {
                if (vrs) load_pair<T>(vrs, Vh, ha, hb, yv);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const float2 yr = mul2(yv[2 * q], SC2), yi = mul2(yv[2 * q + 1], SC2);
                    const float2 re = fma2(o[2 * q + 1], yi, mul2(o[2 * q], yr));
                    const float2 im = fma2(neg2(o[2 * q + 1]), yr, mul2(o[2 * q], yi));
                    const float2 oo = fma2(o[2 * q + 1], o[2 * q + 1], mul2(o[2 * q], o[2 * q]));
                    const float2 yy = fma2(yi, yi, mul2(yr, yr));
                    part[0] += re.x + re.y;
                    part[1] += im.x + im.y;
                    part[2] += oo.x + oo.y;
                    part[NS - 1] += yy.x + yy.y;
                }
            } else if constexpr (RED == RED_NORM) {
#pragma unroll
                for (int q = 0; q < 24; ++q) {
                    const float2 oo = mul2(o[q], o[q]);
                    part[0] += oo.x + oo.y;
                }
            }
        }
        __syncthreads();   // the staged tile is read; its buffers may be refilled
    }

    if constexpr (RED != RED_NONE) {
        grid_reduce<NS, RedStage<RED>::HINT>(part, P.rc, sl);   // FP32 or FP64 partials, as the arithmetic
    }
}

}  // namespace wd
