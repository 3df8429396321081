// Arithmetic throughput probe: long chains of independent fused multiply-adds
// on the FP64, FP32 or packed FP16 pipe, for stating which roof bounds a
// kernel (GB300's FP64 rate is a small fraction of its FP32 rate). Not a
// feature of the paper.
#include <cuda_fp16.h>

#include "handle.h"

namespace wd {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_BLOCK = 256;

template <typename T>
__device__ __forceinline__ T fma_step(T a, T b, T c);
template <> __device__ __forceinline__ double fma_step<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ float fma_step<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ __half2 fma_step<__half2>(__half2 a, __half2 b, __half2 c) { return __hfma2(a, b, c); }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ double from_f<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half2 from_f<__half2>(float v) { return __float2half2_rn(v); }

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half2>(__half2 v) { return __low2float(v) + __high2float(v); }

// x_i := x_i * m + c for PROBE_CHAINS independent chains; m close to 1 and c
// small keep the values finite over any number of steps.
template <typename T>
__global__ void __launch_bounds__(PROBE_BLOCK) k_fma_probe(long long iters, float seed, float* sink) {
    T x[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = from_f<T>(seed + 0.001f * (i + threadIdx.x));
    const T m = from_f<T>(0.9999f), c = from_f<T>(1e-4f);
    for (long long k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) x[i] = fma_step<T>(x[i], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += to_f<T>(x[i]);
    if (s == 1234.5f) sink[blockIdx.x] = s;   // keeps the chains alive; never true for these values
}

}  // namespace wd

using namespace wd;

extern "C" int wd_fma_probe(int bits, long long iters, void* sink, void* stream, double* flops) {
    if ((bits != 64 && bits != 32 && bits != 16) || iters < 1 || !sink || !flops) return WD_ERR_INVALID_ARG;
    const int blocks = num_sms() * 8;
    const long long threads = (long long)blocks * PROBE_BLOCK;
    cudaStream_t s = (cudaStream_t)stream;
    if (bits == 64) k_fma_probe<double><<<blocks, PROBE_BLOCK, 0, s>>>(iters, 0.5f, (float*)sink);
    else if (bits == 32) k_fma_probe<float><<<blocks, PROBE_BLOCK, 0, s>>>(iters, 0.5f, (float*)sink);
    else k_fma_probe<__half2><<<blocks, PROBE_BLOCK, 0, s>>>(iters, 0.5f, (float*)sink);
    if (cudaGetLastError() != cudaSuccess) return WD_ERR_CUDA;
    // 2 flops per fused multiply-add and lane; a packed FP16 FMA is 2 lanes
    *flops = 2.0 * (bits == 16 ? 2.0 : 1.0) * PROBE_CHAINS * (double)iters * (double)threads;
    return WD_OK;
}
