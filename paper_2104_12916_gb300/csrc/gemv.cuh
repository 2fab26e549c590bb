// gemv.cuh -- row-parallel matrix-vector products of the PCG hot path.
//
// One K_F product (Sec. 5.2: a product with C', a forward/backward solve with
// the LDL' factor of F, a product with C) is a chain of row-GEMVs here:
//   u  = C' p             (C' stored row-major as its own copy)
//   z1 = R^{-T} u         (lower triangle: the stored inverse of R')
//   z2 = -(L_S^{-1} G) z1
//   w  = z1 + (L_S^{-1} G)' z2
//   y  = R^{-1} w         (upper triangle)
//   q  = D o p + C y      (+ per-CTA partial of p'q)
// Each output element is produced by one warp (or WPR warps) that streams its
// matrix row with 16-byte loads, so no output needs a cross-CTA reduction and
// every result is deterministic.  Matrices use a padded leading dimension with
// zero padding; triangles store explicit zeros, so row ranges may be rounded
// outward to the vector width.
#pragma once

#include "common.cuh"
#include "dense.cuh"

namespace pcgipm {

constexpr int kGemvThreads = 256;
constexpr int kGemvWarps = kGemvThreads / 32;

// Sum over vector indices v = v0, v0+step, ... < v1 of m[v] . x[v] (4 loads in flight).
template <typename T>
__device__ __forceinline__ T row_dot(const typename Vec16<T>::type* __restrict__ m,
                                     const typename Vec16<T>::type* __restrict__ x, int v, int v1,
                                     int step) {
    using VT = Vec16<T>;
    using V = typename VT::type;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    for (; v + 3 * step < v1; v += 4 * step) {
        const V m0 = __ldg(m + v), m1 = __ldg(m + v + step), m2 = __ldg(m + v + 2 * step),
                m3 = __ldg(m + v + 3 * step);
        const V x0 = __ldg(x + v), x1 = __ldg(x + v + step), x2 = __ldg(x + v + 2 * step),
                x3 = __ldg(x + v + 3 * step);
        a0 = VT::dot(m0, x0, a0);
        a1 = VT::dot(m1, x1, a1);
        a2 = VT::dot(m2, x2, a2);
        a3 = VT::dot(m3, x3, a3);
    }
    for (; v < v1; v += step) a0 = VT::dot(__ldg(m + v), __ldg(x + v), a0);
    return (a0 + a1) + (a2 + a3);
}

// y_i = epi(i, sum_k M[i,k] x[k]); the value epi returns is summed per CTA
// into partials[blockIdx.x] (when partials != nullptr).
// TRI_NONE: WPR warps per row.  TRI_LOWER / TRI_UPPER (square, WPR = 1): each
// warp takes rows i and rows-1-i so that the triangle's work is balanced.
// skip: optional device flag; when *skip != 0 the kernel does nothing (used to
// end a graph-captured PCG loop early once it has converged).
template <typename T, int TRI, int WPR, class Epi>
__global__ void __launch_bounds__(kGemvThreads) gemv_kernel(const T* __restrict__ M, int rows, int cols,
                                                            long long ld, const T* __restrict__ x,
                                                            Epi epi, double* __restrict__ partials,
                                                            const int* __restrict__ skip) {
    PCG_COUNT_KERNEL();
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    __shared__ double sh[40];
    __shared__ T wsum[kGemvWarps];
    if (skip && *skip) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const V* xv = reinterpret_cast<const V*>(x);
    double contrib = 0.0;
    if (TRI == TRI_NONE) {
        constexpr int RPC = kGemvWarps / WPR;
        const int row = blockIdx.x * RPC + warp / WPR;
        const int sub = warp % WPR;
        T acc = T(0);
        if (row < rows) {
            const V* mrow = reinterpret_cast<const V*>(M + (long long)row * ld);
            const int nvec = (cols + VN - 1) / VN;
            acc = row_dot<T>(mrow, xv, sub * 32 + lane, nvec, WPR * 32);
        }
        acc = warp_sum(acc);
        if (WPR > 1) {
            if (lane == 0) wsum[warp] = acc;
            __syncthreads();
            if (sub == 0 && lane == 0) {
                acc = T(0);
#pragma unroll
                for (int t = 0; t < WPR; ++t) acc += wsum[warp + t];
            }
        }
        if (row < rows && sub == 0 && lane == 0) contrib = epi(row, acc);
    } else {
        const int i = blockIdx.x * kGemvWarps + warp;
        const int half = (rows + 1) / 2;
        if (i < half) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int row = (t == 0) ? i : rows - 1 - i;
                if (t == 1 && row == i) break;
                int lo, hi;
                if (TRI == TRI_LOWER) { lo = 0; hi = row + 1; } else { lo = row; hi = cols; }
                const V* mrow = reinterpret_cast<const V*>(M + (long long)row * ld);
                T acc = row_dot<T>(mrow, xv, lo / VN + lane, (hi + VN - 1) / VN, 32);
                acc = warp_sum(acc);
                if (lane == 0) contrib += epi(row, acc);
            }
        }
    }
    if (partials) {
        const double s = block_sum<kGemvThreads>(contrib, sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = s;
    }
}

template <int TRI, int WPR>
inline int gemv_grid(int rows) {
    if (TRI == TRI_NONE) {
        constexpr int RPC = kGemvWarps / WPR;
        return (rows + RPC - 1) / RPC;
    }
    const int half = (rows + 1) / 2;
    return (half + kGemvWarps - 1) / kGemvWarps;
}

// Warps per row for a plain GEMV: enough warps in flight to cover HBM latency
// when there are few long rows.
inline int choose_wpr(int rows, int cols) {
    if (rows >= 4 * 152 * kGemvWarps || cols < 512) return 1;
    if (rows >= 152 * kGemvWarps) return 2;
    if (rows >= 152 * 2) return 4;
    return 8;
}

template <typename T, int TRI, class Epi>
inline int launch_gemv(const T* M, int rows, int cols, long long ld, const T* x, Epi epi,
                       double* partials, const int* skip, cudaStream_t s, int wpr = 0) {
    if (rows <= 0) return 0;
    if (TRI != TRI_NONE) {
        const int g = gemv_grid<TRI, 1>(rows);
        gemv_kernel<T, TRI, 1, Epi><<<g, kGemvThreads, 0, s>>>(M, rows, cols, ld, x, epi, partials, skip);
        return g;
    }
    if (wpr == 0) wpr = choose_wpr(rows, cols);
    int g = 0;
    switch (wpr) {
        case 1: g = gemv_grid<TRI_NONE, 1>(rows);
            gemv_kernel<T, TRI_NONE, 1, Epi><<<g, kGemvThreads, 0, s>>>(M, rows, cols, ld, x, epi, partials, skip);
            break;
        case 2: g = gemv_grid<TRI_NONE, 2>(rows);
            gemv_kernel<T, TRI_NONE, 2, Epi><<<g, kGemvThreads, 0, s>>>(M, rows, cols, ld, x, epi, partials, skip);
            break;
        case 4: g = gemv_grid<TRI_NONE, 4>(rows);
            gemv_kernel<T, TRI_NONE, 4, Epi><<<g, kGemvThreads, 0, s>>>(M, rows, cols, ld, x, epi, partials, skip);
            break;
        default: g = gemv_grid<TRI_NONE, 8>(rows);
            gemv_kernel<T, TRI_NONE, 8, Epi><<<g, kGemvThreads, 0, s>>>(M, rows, cols, ld, x, epi, partials, skip);
            break;
    }
    return g;
}

// ------------------------------------------------------------------ epilogues
// K_F product (Sec. 4.1, eq. [ineq-const-reduced] in the K0 convention):
// q_i = D_i p_i + acc; returns p_i q_i for the PCG step length.
template <typename T>
struct EpiKF {
    T* q; const T* D; const T* p;
    __device__ __forceinline__ double operator()(int i, T acc) const {
        const T v = D[i] * p[i] + acc;
        q[i] = v;
        return (double)p[i] * (double)v;
    }
};

// Second triangular product of the Jacobi-scaled P_H solve:
// z_i = sg_i * acc (acc in the preconditioner precision TP, z and r in the
// operator precision TO); returns r_i z_i.
template <typename TP, typename TO>
struct EpiScaleDot {
    TO* z; const TP* sg; const TO* r;
    __device__ __forceinline__ double operator()(int i, TP acc) const {
        const TO v = (TO)((double)sg[i] * (double)acc);
        z[i] = v;
        return (double)r[i] * (double)v;
    }
};

// r_nu_i = f_i - acc  (right-hand side of the reduced system, Sec. 4.1)
template <typename T>
struct EpiRnu {
    T* y; const T* f;
    __device__ __forceinline__ double operator()(int i, T acc) const {
        y[i] = f[i] - acc;
        return 0.0;
    }
};

}  // namespace pcgipm
