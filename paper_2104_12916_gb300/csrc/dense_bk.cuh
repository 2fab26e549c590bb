// dense_bk.cuh -- Bunch-Kaufman LDL' factorization of the equality-only KKT matrix
// K0 = [H A'; A 0] (symmetric indefinite, N = n + m1), and M0 = [K0^{-1}]_11 from it.
//
// P K0 P' = L D L' with L unit lower triangular, D block diagonal with 1x1 and 2x2
// blocks, P the product of the symmetric interchanges -- the factorization the
// paper's setup phase takes (Sec. 6: the symmetric indefinite LDL' of SciPy, i.e.
// LAPACK's sytrf, with Bunch-Kaufman partial pivoting).  Step k looks at column k of
// the trailing matrix: lambda = max_{i>k} |a_ik| (row r); a 1x1 pivot at k if
// |a_kk| >= alpha lambda, else sigma = max_{i>=k, i!=r} |a_ir| and a 1x1 pivot at k
// if |a_kk| sigma >= alpha lambda^2, a 1x1 pivot at r (rows and columns k and r
// interchanged) if |a_rr| >= alpha sigma, else a 2x2 pivot on (k, r) after the
// interchange of k+1 and r; alpha = (1 + sqrt(17)) / 8.  The inertia of D is K0's
// (Sylvester): (n positive, m1 negative) for a convex QP with full-rank A (Sec. 4.1).
//
// One cooperative kernel runs every step: CTA b owns rows [b N / G, (b + 1) N / G)
// (and the same range of columns for the row interchange), the matrix is held in
// full (both triangles, so that interchanges are plain row and column swaps) and
// every step updates the whole trailing matrix.  A step has two to four grid
// barriers: after the column-k maximum, after the column-r maximum (if needed),
// after the row swap (if any), and after the pivot columns are copied (the update
// of row i then reads only row i and the copied columns).  Every load of data
// another CTA may have written goes to L2 (ld.global.cg): an L1 copy from an
// earlier step could be stale, and CTAs that read different pivots would take
// different branches.  For the same reason every value a pivot decision uses is
// read before the barrier that precedes the next write to it.  Every wait is bounded (2 s of %globaltimer); a wait that runs
// out sets *err and ends the kernel.
//
// M0 = Z' D^{-1} Z with Z = L^{-1} P E, E = [I_n; 0] (so [K0^{-1}]_11 = E' P' L^{-T}
// D^{-1} L^{-1} P E): a blocked forward substitution (64-row blocks: a GEMM with the
// rows above, then the 64 x 64 unit-lower block by rows), D^{-1} applied block by
// block, and one GEMM.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace pcgipm {

constexpr int kBkThreads = 256;
constexpr int kBkRows = 64;   // rows of one forward-substitution block

struct BkArgs {
    double* A;          // N x N, full symmetric on entry; on exit L below the diagonal (unit diagonal implied)
    long long lda;
    int N;
    double* w;          // 2 N: the pivot column(s) of the current step
    double* cval;       // G candidate maxima (and 1024 more for the second search)
    int* cidx;
    int* perm;          // N: on entry the identity; on exit perm[i] = original index of position i
    double* d;          // N: D's diagonal
    double* e;          // N: e[k] = D[k+1][k] for a 2x2 block starting at k, else 0
    int* ptype;         // N: 1 (1x1 pivot), 2 (first row of a 2x2), 0 (second row of a 2x2)
    unsigned* bar;      // zeroed before the launch
    int* err;           // 1: a wait ran out
    int* status;        // 0, or k + 1 if column k of the trailing matrix is zero (singular K0)
};

__device__ __forceinline__ unsigned long long bk_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kBkThreads) bk_factor_kernel(const BkArgs a) {
    PCG_COUNT_KERNEL();
    __shared__ double s_val[kBkThreads / 32];
    __shared__ int s_idx[kBkThreads / 32];
    __shared__ int s_stop;
    __shared__ double s_sc[8];
    __shared__ int s_ic[8];
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int N = a.N;
    const long long lda = a.lda;
    double* A = a.A;
    const int r0 = (int)((long long)N * b / G), r1 = (int)((long long)N * (b + 1) / G);
    unsigned target = 0;
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;

    auto grid_barrier = [&]() {
        __syncthreads();
        target += G;
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.bar, 1u);
            const unsigned long long t0 = bk_timer();
            unsigned polls = 0;
            s_stop = 0;
            while ((int)(*(volatile unsigned*)a.bar - target) < 0) {
                if (*(volatile int*)a.err) { s_stop = 1; break; }
                if ((++polls & 1023) == 0 && bk_timer() - t0 > 2000000000ull) {
                    atomicExch(a.err, 1);
                    s_stop = 1;
                    break;
                }
            }
            __threadfence();
        }
        __syncthreads();
        return s_stop == 0;
    };
    // block maximum of |A[i][col]| over this block's rows i in [lo, N), i != skip
    // (ties to the smaller row), published as candidate `slot` * G + b
    auto column_max = [&](int col, int lo, int skip, int slot) {
        double best = -1.0;
        int bi = -1;
        for (int i = max(r0, lo) + tid; i < r1; i += kBkThreads) {
            if (i == skip) continue;
            const double v = fabs(__ldcg(A + (long long)i * lda + col));
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bv = -1.0;
            int bb = -1;
            for (int w = 0; w < kBkThreads / 32; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] >= 0 && (bb < 0 || s_idx[w] < bb))) {
                    bv = s_val[w];
                    bb = s_idx[w];
                }
            a.cval[slot * G + b] = bv;
            a.cidx[slot * G + b] = bb;
        }
    };
    // the G candidates of `slot`, reduced in block order (the same in every CTA)
    auto reduce_candidates = [&](int slot, double& v, int& idx) {
        if (tid == 0) {
            double bv = -1.0;
            int bb = -1;
            for (int c = 0; c < G; ++c) {
                const double cv = *(volatile double*)&a.cval[slot * G + c];
                const int ci = *(volatile int*)&a.cidx[slot * G + c];
                if (cv > bv || (cv == bv && ci >= 0 && (bb < 0 || ci < bb))) { bv = cv; bb = ci; }
            }
            s_sc[slot] = bv;
            s_ic[slot] = bb;
        }
        __syncthreads();
        v = s_sc[slot];
        idx = s_ic[slot];
    };

    int k = 0;
    while (k < N) {
        // ---- lambda = max_{i>k} |a_ik|, row r
        column_max(k, k + 1, -1, 0);
        if (!grid_barrier()) return;
        double lambda;
        int r;
        reduce_candidates(0, lambda, r);
        const double akk = __ldcg(A + (long long)k * lda + k);
        if (fabs(akk) == 0.0 && lambda <= 0.0) {       // a zero column: K0 is singular
            if (b == 0 && tid == 0) *a.status = k + 1;
            return;
        }
        int size = 1, p = k, swap_row = -1;
        if (lambda > 0.0 && fabs(akk) < alpha * lambda) {
            // ---- sigma = max_{i>=k, i!=r} |a_ir|.  a_rr is read before the barrier: after
            // it, the row swap of a faster CTA may already have moved it
            const double arr = __ldcg(A + (long long)r * lda + r);
            column_max(r, k, r, 1);
            if (!grid_barrier()) return;
            double sigma;
            int rs;
            reduce_candidates(1, sigma, rs);
            if (fabs(akk) * sigma >= alpha * lambda * lambda) {
                size = 1;
            } else if (fabs(arr) >= alpha * sigma) {
                size = 1; p = k; swap_row = r;
            } else {
                size = 2; p = k + 1; swap_row = (r == k + 1) ? -1 : r;
            }
        }
        if (swap_row >= 0) {
            // ---- rows p and r over this block's columns, then (after a barrier) columns p and r
            const int rr = swap_row;
            for (int c = r0 + tid; c < r1; c += kBkThreads) {
                const double t = __ldcg(A + (long long)p * lda + c);
                A[(long long)p * lda + c] = __ldcg(A + (long long)rr * lda + c);
                A[(long long)rr * lda + c] = t;
            }
            if (b == 0 && tid == 0) {
                const int t = a.perm[p];
                a.perm[p] = a.perm[rr];
                a.perm[rr] = t;
            }
            if (!grid_barrier()) return;
            for (int i = max(r0, k) + tid; i < r1; i += kBkThreads) {
                const double t = __ldcg(A + (long long)i * lda + p);
                A[(long long)i * lda + p] = __ldcg(A + (long long)i * lda + rr);
                A[(long long)i * lda + rr] = t;
            }
        }
        // ---- the pivot column(s) of this block's rows, for every block's update
        for (int i = max(r0, k) + tid; i < r1; i += kBkThreads) {
            a.w[i] = __ldcg(A + (long long)i * lda + k);
            if (size == 2) a.w[N + i] = __ldcg(A + (long long)i * lda + k + 1);
        }
        if (!grid_barrier()) return;
        const int k1 = k + size;
        if (size == 1) {
            const double dk = __ldcg(a.w + k);
            if (b == 0 && tid == 0) { a.d[k] = dk; a.e[k] = 0.0; a.ptype[k] = 1; }
            const double inv = 1.0 / dk;
            for (int i = max(r0, k1); i < r1; ++i) {
                const double li = __ldcg(a.w + i) * inv;
                double* Ai = A + (long long)i * lda;
                for (int j = k1 + tid; j < N; j += kBkThreads) Ai[j] = fma(-li, __ldcg(a.w + j), __ldcg(Ai + j));
                if (tid == 0) Ai[k] = li;   // (column k is not among the updated j >= k1)
            }
        } else {
            const double d11 = __ldcg(a.w + k), d21 = __ldcg(a.w + k + 1), d22 = __ldcg(a.w + N + k + 1);
            const double det = d11 * d22 - d21 * d21;
            if (b == 0 && tid == 0) {
                a.d[k] = d11; a.d[k + 1] = d22; a.e[k] = d21; a.e[k + 1] = 0.0;
                a.ptype[k] = 2; a.ptype[k + 1] = 0;
            }
            for (int i = max(r0, k1); i < r1; ++i) {
                // [l_i0 l_i1] = [w0_i w1_i] D^{-1};  A_ij -= l_i0 w0_j + l_i1 w1_j
                const double w0 = __ldcg(a.w + i), w1 = __ldcg(a.w + N + i);
                const double l0 = (w0 * d22 - w1 * d21) / det, l1 = (w1 * d11 - w0 * d21) / det;
                double* Ai = A + (long long)i * lda;
                for (int j = k1 + tid; j < N; j += kBkThreads)
                    Ai[j] = fma(-l1, __ldcg(a.w + N + j), fma(-l0, __ldcg(a.w + j), __ldcg(Ai + j)));
                if (tid == 0) { Ai[k] = l0; Ai[k + 1] = l1; }
            }
            // L's block for the pivot rows is the identity: its entry below the diagonal
            // (which held D's off-diagonal, now in e[k]) is zero
            if (k + 1 >= r0 && k + 1 < r1 && tid == 0) A[(long long)(k + 1) * lda + k] = 0.0;
        }
        k = k1;
    }
}

// K = [H A'; A 0] in full (N = n + m1, leading dimension ldk; padding zero) and
// perm = the identity.
__global__ void bk_build_k0_kernel(const double* __restrict__ H, long long ldh, const double* __restrict__ A,
                                   long long lda, int n, int m1, double* __restrict__ K, long long ldk,
                                   int* __restrict__ perm) {
    PCG_COUNT_KERNEL();
    const int N = n + m1;
    const long long total = (long long)N * ldk;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ldk), j = (int)(t % ldk);
        double v = 0.0;
        if (j < N) {
            if (i < n && j < n) v = H[(long long)i * ldh + j];
            else if (i < n) v = A[(long long)(j - n) * lda + i];
            else if (j < n) v = A[(long long)(i - n) * lda + j];
        }
        K[t] = v;
        if (j == 0) perm[i] = i;
    }
}

// Z[i, c] = 1 if perm[i] == c (c < n), else 0: the columns of P E.  Z is N x n (ldz).
__global__ void bk_pe_kernel(const int* __restrict__ perm, int N, int n, double* __restrict__ Z, long long ldz) {
    PCG_COUNT_KERNEL();
    const long long total = (long long)N * ldz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ldz), c = (int)(t % ldz);
        Z[t] = (c < n && perm[i] == c) ? 1.0 : 0.0;
    }
}

// Rows [k0, k0 + kb) of Z: forward substitution with the unit-lower diagonal block of
// L (the rows above are already subtracted): thread t owns columns t, t + T, ...
__global__ void bk_trsm_block_kernel(const double* __restrict__ L, long long lda, int k0, int kb, double* __restrict__ Z,
                                     long long ldz, int n) {
    PCG_COUNT_KERNEL();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        for (int i = 1; i < kb; ++i) {
            double s = Z[(long long)(k0 + i) * ldz + c];
            for (int j = 0; j < i; ++j) s = fma(-L[(long long)(k0 + i) * lda + k0 + j], Z[(long long)(k0 + j) * ldz + c], s);
            Z[(long long)(k0 + i) * ldz + c] = s;
        }
    }
}

// Y = D^{-1} Z, block by block (1x1 and 2x2 blocks of D).
__global__ void bk_dinv_kernel(const double* __restrict__ d, const double* __restrict__ e, const int* __restrict__ ptype,
                               int N, int n, const double* __restrict__ Z, double* __restrict__ Y, long long ldz) {
    PCG_COUNT_KERNEL();
    const long long total = (long long)N * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), c = (int)(t % n);
        const long long o = (long long)i * ldz + c;
        if (ptype[i] == 1) {
            Y[o] = Z[o] / d[i];
        } else if (ptype[i] == 2) {
            const double a = d[i], bb = e[i], cc = d[i + 1], det = a * cc - bb * bb;
            Y[o] = (cc * Z[o] - bb * Z[o + ldz]) / det;
        } else {   // second row of a 2x2 block
            const double a = d[i - 1], bb = e[i - 1], cc = d[i], det = a * cc - bb * bb;
            Y[o] = (a * Z[o] - bb * Z[o - ldz]) / det;
        }
    }
}

}  // namespace pcgipm
