// common.cuh -- shared device helpers of the pcgipm CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pcgipm {

constexpr int kWarp = 32;

// Number of kernel launches of this library that reached the device (counted by
// the first thread of each launch; read by qp_kernel_launches()).
__device__ unsigned long long g_kernel_launches = 0;

#define PCG_COUNT_KERNEL()                                                                   \
    do {                                                                                     \
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&    \
            threadIdx.y == 0)                                                                \
            atomicAdd(&::pcgipm::g_kernel_launches, 1ULL);                                   \
    } while (0)

// 16-byte vector type of T (float4 for float, double2 for double).
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ __forceinline__ static float dot(const float4 a, const float4 b, float acc) {
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        return fmaf(a.w, b.w, acc);
    }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ __forceinline__ static double dot(const double2 a, const double2 b, double acc) {
        acc = fma(a.x, b.x, acc);
        return fma(a.y, b.y, acc);
    }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of one double per thread, result valid in thread 0.
// Fixed reduction tree: deterministic for a fixed block size.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh /* >= NT/32 */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? sh[l] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = -1.0e308;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? sh[l] : -1.0e308;
        r = warp_max(r);
    }
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double* sh) {
    v = warp_min(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 1.0e308;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? sh[l] : 1.0e308;
        r = warp_min(r);
    }
    __syncthreads();
    return r;
}

// Sum of `count` partials in a fixed order by one block (all threads get it).
template <int NT>
__device__ __forceinline__ double reduce_partials(const double* __restrict__ part, int count,
                                                  double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += NT) v += part[i];
    v = block_sum<NT>(v, sh);
    if (threadIdx.x == 0) sh[32] = v;
    __syncthreads();
    v = sh[32];
    __syncthreads();
    return v;
}

// Leading dimension padded to a multiple of 32 elements (>= 128-byte rows for
// float, 256-byte for double) so every row starts 16-byte aligned.
inline int pad_ld(int cols) { return ((cols + 31) / 32) * 32; }

}  // namespace pcgipm
