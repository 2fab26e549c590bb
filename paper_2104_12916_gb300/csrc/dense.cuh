// dense.cuh -- dense factorization kernels: tiled GEMM, blocked Cholesky with
// in-place triangular inverse, transposes and conversions.
//
// These implement the setup phase of Sec. 4.1 (the factorization of the fixed
// equality-only KKT matrix) and the per-iteration Cholesky of P_H (Sec. 5.2,
// PH-KF: "perform a Cholesky factorization P_H = L L^T at every IPM iteration").
// Every triangular factor is also inverted (W = L^{-1}) so that the triangular
// solves inside PCG become parallel triangular matrix-vector products.
#pragma once

#include "common.cuh"
#include "tc_gemm.cuh"

namespace pcgipm {

enum Tri { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

// ---------------------------------------------------------------- tiled GEMM
// C[i,j] = alpha * sum_k opA(i,k) opB(k,j) + beta * C[i,j]
//   opA(i,k) = A[i*sai + k*sak],  opB(k,j) = B[k*sbk + j*sbj]
// a_tri / b_tri declare the zero pattern of the logical operand (the zeros are
// present in memory; declaring them only skips work): lower = zero above the
// diagonal, upper = zero below.  lower_out: only tiles/elements with j <= i.
template <typename T>
struct GemmArgs {
    int M, N, K;
    const T* A; long long sai, sak;
    const T* B; long long sbk, sbj;
    T* C; long long ldc;
    T alpha, beta;
    int a_tri, b_tri, lower_out;
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs<T> g) {
    PCG_COUNT_KERNEL();
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    __shared__ T As[2][BK][BM + 4];
    __shared__ T Bs[2][BK][BN + 4];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (g.lower_out && n0 > m0 + BM - 1) return;
    int kLo = 0, kHi = g.K;
    if (g.a_tri == TRI_LOWER) kHi = min(kHi, m0 + BM);
    if (g.a_tri == TRI_UPPER) kLo = max(kLo, m0);
    if (g.b_tri == TRI_LOWER) kLo = max(kLo, n0);
    if (g.b_tri == TRI_UPPER) kHi = min(kHi, n0 + BN);
    const int tid = threadIdx.x;
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = T(0);

    const bool a_m_contig = (g.sai == 1);
    const bool b_n_contig = (g.sbj == 1);
    constexpr int A_PER = BM * BK / 256, B_PER = BK * BN / 256;
    T ra[A_PER], rb[B_PER];

    auto load_regs = [&](int k0) {
#pragma unroll
        for (int t = 0; t < A_PER; ++t) {
            const int e = tid + 256 * t;
            int mm, kk;
            if (a_m_contig) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
            const int gi = m0 + mm, gk = k0 + kk;
            ra[t] = (gi < g.M && gk < kHi && gk >= kLo) ? g.A[gi * g.sai + gk * g.sak] : T(0);
        }
#pragma unroll
        for (int t = 0; t < B_PER; ++t) {
            const int e = tid + 256 * t;
            int kk, nn;
            if (b_n_contig) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
            const int gj = n0 + nn, gk = k0 + kk;
            rb[t] = (gj < g.N && gk < kHi && gk >= kLo) ? g.B[gk * g.sbk + gj * g.sbj] : T(0);
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int t = 0; t < A_PER; ++t) {
            const int e = tid + 256 * t;
            int mm, kk;
            if (a_m_contig) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
            As[buf][kk][mm] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < B_PER; ++t) {
            const int e = tid + 256 * t;
            int kk, nn;
            if (b_n_contig) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
            Bs[buf][kk][nn] = rb[t];
        }
    };

    int k0 = (kLo / BK) * BK;
    if (k0 < kHi) {
        load_regs(k0);
        store_smem(0);
        __syncthreads();
        int buf = 0;
        for (; k0 < kHi; k0 += BK) {
            const bool more = (k0 + BK < kHi);
            if (more) load_regs(k0 + BK);
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T a[TM], b[TN];
#pragma unroll
                for (int r = 0; r < TM; ++r) a[r] = As[buf][kk][ty + r * (BM / TM)];
#pragma unroll
                for (int c = 0; c < TN; ++c) b[c] = Bs[buf][kk][tx + c * (BN / TN)];
#pragma unroll
                for (int r = 0; r < TM; ++r)
#pragma unroll
                    for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
            }
            if (more) {
                store_smem(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < TM; ++r) {
        const int i = m0 + ty + r * (BM / TM);
        if (i >= g.M) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int j = n0 + tx + c * (BN / TN);
            if (j >= g.N) continue;
            if (g.lower_out && j > i) continue;
            T* p = g.C + i * g.ldc + j;
            T v = g.alpha * acc[r][c];
            if (g.beta != T(0)) v = fma(g.beta, *p, v);
            *p = v;
        }
    }
}

template <typename T>
inline void gemm(const GemmArgs<T>& g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return;
    if constexpr (sizeof(T) == 4) {
        constexpr int BM = 128, BN = 128;
        dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
        gemm_kernel<T, BM, BN, 8, 8, 8><<<grid, 256, 0, s>>>(g);
    } else {
        constexpr int BM = 64, BN = 64;
        dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
        gemm_kernel<T, BM, BN, 16, 4, 4><<<grid, 256, 0, s>>>(g);
    }
}

// ------------------------------------------------- blocked Cholesky + inverse
constexpr int kNB = 64;   // block size of the blocked factorization

// Factor the kb x kb diagonal block A[k0.., k0..] (lower) in compute type CT,
// write L_kk back (upper part of the block zeroed) and W_kk = L_kk^{-1} into W.
// floor_mode = 0: a pivot d <= piv_floor * diag0[k0+j] (diag0: the matrix's
//   original diagonal; a non-positive or numerically zero pivot) records
//   info = k0 + j + 1 (first failure wins) and continues with d = 1 so that the
//   kernel stays finite.  With `warn`, the first pivot d <= warn_floor * diag0
//   is also recorded there.
// floor_mode = 1: a pivot d < piv_floor is replaced by piv_floor (a diagonal
//   shift of a preconditioner; counted in info as a positive number of shifts).
// Right-looking with one block barrier per column: every thread derives the
// pivot of column j itself from the updated diagonal entry, the update
// a[i][l] -= a[i][j] a[l][j] / d uses the unscaled column, and the scaled column
// goes to a separate tile (lf), so no thread writes what another reads in the
// same step.
template <typename T, typename CT>
__global__ void __launch_bounds__(256) potrf_diag_kernel(T* A, long long lda, T* W, long long ldw,
                                                         int k0, int kb, int floor_mode,
                                                         double piv_floor, int* info,
                                                         const double* __restrict__ diag0,
                                                         double warn_floor, int* warn) {
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto a = reinterpret_cast<CT(*)[kNB + 1]>(smem_raw);
    auto w = reinterpret_cast<CT(*)[kNB + 1]>(smem_raw + sizeof(CT) * kNB * (kNB + 1));
    auto lf = reinterpret_cast<CT(*)[kNB + 1]>(smem_raw + 2 * sizeof(CT) * kNB * (kNB + 1));
    const int tid = threadIdx.x;
    for (int e = tid; e < kb * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        a[i][j] = (j <= i) ? CT(A[(k0 + i) * lda + k0 + j]) : CT(0);
        lf[i][j] = CT(0);
    }
    __syncthreads();
    // thread (ty, tx) of a 16 x 16 layout takes rows ty + 16 r and columns tx + 16 c
    const int tx = tid & 15, ty = tid >> 4;
    for (int j = 0; j < kb; ++j) {
        CT d = a[j][j];
        bool bad = false;
        if (floor_mode == 0) {
            if (tid == 0 && warn && !(d > CT(warn_floor * diag0[k0 + j]))) atomicCAS(warn, 0, k0 + j + 1);
            if (!(d > CT(piv_floor * diag0[k0 + j]))) {
                bad = true;
                d = CT(1);
            }
        } else if (!(d >= CT(piv_floor))) {
            bad = true;
            d = CT(piv_floor);
        }
        if (bad && tid == 0) {
            if (floor_mode == 0) atomicCAS(info, 0, k0 + j + 1);
            else atomicAdd(info, 1);
        }
        const CT piv = sqrt(d);
        const CT inv = CT(1) / piv, dinv = CT(1) / d;
        if (tid == 0) lf[j][j] = piv;
        for (int i = j + 1 + tid; i < kb; i += 256) lf[i][j] = a[i][j] * inv;
        for (int i = j + 1 + ty; i < kb; i += 16) {
            const CT aij = a[i][j] * dinv;
            for (int l = j + 1 + tx; l <= i; l += 16) a[i][l] -= aij * a[l][j];
        }
        __syncthreads();
    }
    // W = L^{-1}, row by row: w[i][i] = 1 / l_ii and, for t < i,
    // w[i][t] = -(sum_{k=t}^{i-1} l_ik w[k][t]) / l_ii.  Four threads share a
    // column t (k split four ways, shuffle-reduced), so all 256 threads work.
    const int t = tid >> 2, q = tid & 3;
    for (int i = 0; i < kb; ++i) {
        CT sum = CT(0);
        if (t < i)
            for (int k = t + q; k < i; k += 4) sum += lf[i][k] * w[k][t];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if (q == 0) {
            if (t < i) w[i][t] = -sum / lf[i][i];
            else if (t == i) w[i][i] = CT(1) / lf[i][i];
        }
        __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        A[(k0 + i) * lda + k0 + j] = (j <= i) ? T(lf[i][j]) : T(0);
        W[(k0 + i) * ldw + k0 + j] = (j <= i) ? T(w[i][j]) : T(0);
    }
}

// Panel of the right-looking Cholesky: A[r, k0:k0+kb] <- A[r, k0:k0+kb] W_kk^T
// for rows r in [k0+kb, n), in place (one CTA per 64-row slab).
template <typename T>
__global__ void __launch_bounds__(256) trsm_panel_kernel(T* A, long long lda, const T* W, long long ldw,
                                                         int k0, int kb, int n) {
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto wk = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);
    auto ap = reinterpret_cast<T(*)[kNB + 1]>(smem_raw + sizeof(T) * kNB * (kNB + 1));
    const int r0 = k0 + kb + blockIdx.x * kNB;
    const int tid = threadIdx.x;
    for (int e = tid; e < kb * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        wk[i][j] = W[(k0 + i) * ldw + k0 + j];
    }
    for (int e = tid; e < kNB * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        ap[i][j] = (r0 + i < n) ? A[(r0 + i) * lda + k0 + j] : T(0);
    }
    __syncthreads();
    // out[i][j] = sum_{l <= j} ap[i][l] * wk[j][l]   (W lower => W^T upper)
    for (int e = tid; e < kNB * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        if (r0 + i >= n) continue;
        T s = T(0);
        for (int l = 0; l <= j; ++l) s = fma(ap[i][l], wk[j][l], s);
        A[(r0 + i) * lda + k0 + j] = s;
    }
}

// Right-looking triangular inverse, scaling step: W[k0:k0+kb, 0:k0] <- W_kk W[k0:k0+kb, 0:k0]
// (in place, one CTA per 64-column slab; W_kk lower).
template <typename T>
__global__ void __launch_bounds__(256) trmm_rowblock_kernel(T* W, long long ldw, int k0, int kb) {
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto wk = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);
    auto rs = reinterpret_cast<T(*)[kNB + 1]>(smem_raw + sizeof(T) * kNB * (kNB + 1));
    const int c0 = blockIdx.x * kNB;
    const int cw = min(kNB, k0 - c0);
    const int tid = threadIdx.x;
    for (int e = tid; e < kb * kb; e += 256) {
        const int i = e / kb, j = e % kb;
        wk[i][j] = W[(k0 + i) * ldw + k0 + j];
    }
    for (int e = tid; e < kb * cw; e += 256) {
        const int i = e / cw, j = e % cw;
        rs[i][j] = W[(k0 + i) * ldw + c0 + j];
    }
    __syncthreads();
    for (int e = tid; e < kb * cw; e += 256) {
        const int i = e / cw, j = e % cw;
        T s = T(0);
        for (int l = 0; l <= i; ++l) s = fma(wk[i][l], rs[l][j], s);
        W[(k0 + i) * ldw + c0 + j] = s;
    }
}

// In-place blocked Cholesky of the lower triangle of A (n x n, leading dim lda)
// and its inverse W = L^{-1} (lower, zeros above the diagonal; W must be
// zero-initialised by the caller).  CT is the compute type of the diagonal
// blocks (double: FP64 pivots).  Right-looking: per block column k
//   1. factor the diagonal block and invert it,
//   2. panel  L21 = A21 W_kk^T,
//   3. trailing update A22 -= L21 L21^T (lower tiles),
//   4. inverse: W[k, 0:k] <- W_kk R[k, 0:k];  R[k+1:, 0:k+1] -= L21 W[k, 0:k+1].
// Dynamic shared memory of the three block kernels: two (kNB x kNB+1) tiles.
template <typename X>
constexpr size_t two_tiles_bytes() { return 2 * sizeof(X) * kNB * (kNB + 1); }
template <typename X>
constexpr size_t three_tiles_bytes() { return 3 * sizeof(X) * kNB * (kNB + 1); }

// Sets the (process-wide) shared-memory attributes once per instantiation; the
// values are fixed, so concurrent callers agree.
template <typename T, typename CT>
inline void chol_inv_prepare() {
    static const bool done = []() {
        cudaFuncSetAttribute(potrf_diag_kernel<T, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)three_tiles_bytes<CT>());
        cudaFuncSetAttribute(trsm_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)two_tiles_bytes<T>());
        cudaFuncSetAttribute(trmm_rowblock_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)two_tiles_bytes<T>());
        return true;
    }();
    (void)done;
}

template <typename T>
__global__ void save_diag_kernel(const T* __restrict__ A, long long lda, int n, double* __restrict__ out) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (double)A[i * lda + i];
}

// diag0: scratch of n doubles (used when floor_mode == 0).  With floor_mode 0 and
// `warn` non-null, the first pivot d <= warn_floor * diag0 is also recorded in *warn.
template <typename T, typename CT>
void chol_inv(T* A, long long lda, T* W, long long ldw, int n, int floor_mode, double piv_floor,
              int* d_info, cudaStream_t s, double* diag0 = nullptr, double warn_floor = 0.0,
              int* warn = nullptr) {
    if (floor_mode == 0) save_diag_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(A, lda, n, diag0);
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kb = min(kNB, n - k0);
        potrf_diag_kernel<T, CT><<<1, 256, three_tiles_bytes<CT>(), s>>>(A, lda, W, ldw, k0, kb,
                                                                      floor_mode, piv_floor, d_info, diag0,
                                                                      warn_floor, warn);
        const int rest = n - k0 - kb;
        if (k0 > 0) {
            trmm_rowblock_kernel<T><<<(k0 + kNB - 1) / kNB, 256, two_tiles_bytes<T>(), s>>>(W, ldw, k0, kb);
        }
        if (rest > 0) {
            trsm_panel_kernel<T><<<(rest + kNB - 1) / kNB, 256, two_tiles_bytes<T>(), s>>>(A, lda, W, ldw,
                                                                                          k0, kb, n);
            GemmArgs<T> g{};
            // trailing update A22 -= L21 L21^T
            g.M = rest; g.N = rest; g.K = kb;
            g.A = A + (k0 + kb) * lda + k0; g.sai = lda; g.sak = 1;
            g.B = A + (k0 + kb) * lda + k0; g.sbk = 1; g.sbj = lda;
            g.C = A + (k0 + kb) * lda + k0 + kb; g.ldc = lda;
            g.alpha = T(-1); g.beta = T(1); g.lower_out = 1;
            gemm<T>(g, s);
            // inverse update R[k+1:, 0:k0+kb] -= L21 W[k0:k0+kb, 0:k0+kb]
            GemmArgs<T> h{};
            h.M = rest; h.N = k0 + kb; h.K = kb;
            h.A = A + (k0 + kb) * lda + k0; h.sai = lda; h.sak = 1;
            h.B = W + k0 * ldw; h.sbk = ldw; h.sbj = 1;
            h.C = W + (k0 + kb) * ldw; h.ldc = ldw;
            h.alpha = T(-1); h.beta = T(1);
            gemm<T>(h, s);
        }
    }
}

// out[j * ldo + i] = hi/lo parts of in[i * ldi + j] (rows x cols in, cols x rows out):
// the transposed, TF32-split copy of a row block that the tensor-core GEMM takes
// as its K-major B operand.
__global__ void tc_transpose_split_kernel(const float* __restrict__ in, long long ldi, int rows, int cols,
                                          float* __restrict__ hi, float* __restrict__ lo, long long ldo) {
    PCG_COUNT_KERNEL();
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = by + r, j = bx + threadIdx.x;
        tile[r][threadIdx.x] = (i < rows && j < cols) ? in[i * ldi + j] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = bx + r, i = by + threadIdx.x;
        if (i < rows && j < cols) {
            const float v = tile[threadIdx.x][r];
            uint32_t h;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            hi[j * ldo + i] = __uint_as_float(h);
            lo[j * ldo + i] = v - __uint_as_float(h);
        }
    }
}

inline void tc_split(const float* x, long long ldx, int rows, int cols, float* hi, float* lo, long long ldo,
                     cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    const long long total = (long long)rows * cols;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    tc_split_kernel<<<blocks, 256, 0, s>>>(x, ldx, rows, cols, hi, lo, ldo);
}

// Floats of tensor-core scratch chol_inv_tc needs for an n x n factorization.
inline size_t chol_tc_scratch(int n) { return 4 * (size_t)(n + kTcBM) * kNB; }

// chol_inv for FP32 storage with the two rank-kNB updates of every block column
// on the tensor cores (FP32-accurate 3xTF32): the trailing update
// A22 -= L21 L21' (lower tiles) and the inverse update
// W[k+1:, 0:k+1] -= L21 W[k, 0:k+1].  The diagonal blocks, their inverses and
// the panel stay on the CUDA cores in compute type CT.  scratch: at least
// chol_tc_scratch(n) floats; d_err receives a tensor-core wait failure.  Falls
// back to the CUDA-core GEMM if a tensor map cannot be made.
template <typename CT>
void chol_inv_tc(float* A, long long lda, float* W, long long ldw, int n, int floor_mode, double piv_floor,
                 int* d_info, cudaStream_t s, float* scratch, int* d_err, double* diag0 = nullptr,
                 double warn_floor = 0.0, int* warn = nullptr) {
    if (floor_mode == 0) save_diag_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(A, lda, n, diag0);
    const long long ldk = kNB;
    float* lh = scratch;
    float* ll = lh + (size_t)n * ldk;
    float* bh = ll + (size_t)n * ldk;
    float* bl = bh + (size_t)n * ldk;
    for (int k0 = 0; k0 < n; k0 += kNB) {
        const int kb = min(kNB, n - k0);
        potrf_diag_kernel<float, CT><<<1, 256, three_tiles_bytes<CT>(), s>>>(A, lda, W, ldw, k0, kb, floor_mode,
                                                                            piv_floor, d_info, diag0, warn_floor,
                                                                            warn);
        const int rest = n - k0 - kb;
        if (k0 > 0)
            trmm_rowblock_kernel<float><<<(k0 + kNB - 1) / kNB, 256, two_tiles_bytes<float>(), s>>>(W, ldw, k0, kb);
        if (rest <= 0) continue;
        trsm_panel_kernel<float><<<(rest + kNB - 1) / kNB, 256, two_tiles_bytes<float>(), s>>>(A, lda, W, ldw,
                                                                                             k0, kb, n);
        float* L21 = A + (long long)(k0 + kb) * lda + k0;
        tc_split(L21, lda, rest, kb, lh, ll, ldk, s);   // (the GEMM's K is kb: columns beyond read as zeros)
        bool ok = tc_gemm(rest, rest, kb, -1.0f, lh, ll, ldk, lh, ll, ldk, 1.0f,
                          A + (long long)(k0 + kb) * lda + k0 + kb, lda, true, true, d_err, s);
        dim3 tg((k0 + kb + 31) / 32, (kb + 31) / 32), tb(32, 8);
        tc_transpose_split_kernel<<<tg, tb, 0, s>>>(W + (long long)k0 * ldw, ldw, kb, k0 + kb, bh, bl, ldk);
        ok = ok && tc_gemm(rest, k0 + kb, kb, -1.0f, lh, ll, ldk, bh, bl, ldk, 1.0f, W + (long long)(k0 + kb) * ldw,
                           ldw, true, false, d_err, s);
        if (!ok) {
            cudaGetLastError();
            GemmArgs<float> g{};
            g.M = rest; g.N = rest; g.K = kb;
            g.A = L21; g.sai = lda; g.sak = 1;
            g.B = L21; g.sbk = 1; g.sbj = lda;
            g.C = A + (long long)(k0 + kb) * lda + k0 + kb; g.ldc = lda;
            g.alpha = -1.0f; g.beta = 1.0f; g.lower_out = 1;
            gemm<float>(g, s);
            GemmArgs<float> h{};
            h.M = rest; h.N = k0 + kb; h.K = kb;
            h.A = L21; h.sai = lda; h.sak = 1;
            h.B = W + (long long)k0 * ldw; h.sbk = ldw; h.sbj = 1;
            h.C = W + (long long)(k0 + kb) * ldw; h.ldc = ldw;
            h.alpha = -1.0f; h.beta = 1.0f;
            gemm<float>(h, s);
        }
    }
}

// ------------------------------------------------ pivoted Cholesky, low rank
// M = Z Z' for a symmetric positive semidefinite M (n x n, FP64) of known rank
// r: r steps of the outer-product Cholesky, each on the largest remaining
// diagonal entry (complete diagonal pivoting); Zt = Z' (r x n, row k = column k
// of Z) so that every thread's reads of a column are coalesced.  *rank_out
// receives the number of steps taken (fewer than r if a pivot falls to
// rel_floor times the largest diagonal entry).  d: scratch of n doubles.
// Spread over a cooperative grid: CTA b owns rows
// [b n / G, (b + 1) n / G).  One grid barrier per step: before it, every CTA
// publishes the largest remaining diagonal entry of its rows (value, index) for
// the step; after it, every CTA reads the G candidates, takes the same pivot p
// (ties to the smaller index), and computes its rows of column k from Zt rows
// written in earlier steps.  bar: a zeroed counter; every wait is bounded
// (2 s of %globaltimer) and a wait that runs out sets *err and ends the kernel.
__global__ void __launch_bounds__(256) pivoted_chol_grid_kernel(const double* __restrict__ M, long long ldm, int n,
                                                                int r, double* __restrict__ Zt, long long ldz,
                                                                double* __restrict__ d, double* __restrict__ cval,
                                                                int* __restrict__ cidx, unsigned* bar,
                                                                double rel_floor, int* __restrict__ rank_out,
                                                                int* __restrict__ err) {
    PCG_COUNT_KERNEL();
    __shared__ double s_val[8];
    __shared__ int s_idx[8];
    __shared__ int s_piv;
    __shared__ double s_pv, s_dmax;
    __shared__ int s_stop;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int i0 = (int)((long long)n * b / G), i1 = (int)((long long)n * (b + 1) / G);
    for (int i = i0 + tid; i < i1; i += 256) d[i] = M[i * ldm + i];
    unsigned target = 0;
    auto local_best = [&]() {
        double best = -1.0;
        int bi = -1;
        for (int i = i0 + tid; i < i1; i += 256)
            if (d[i] > best) { best = d[i]; bi = i; }
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
            for (int w = 0; w < 8; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] >= 0 && (bb < 0 || s_idx[w] < bb))) { bv = s_val[w]; bb = s_idx[w]; }
            cval[b] = bv;
            cidx[b] = bb;
        }
    };
    auto grid_barrier = [&]() {
        __syncthreads();
        target += G;
        if (tid == 0) {
            __threadfence();
            atomicAdd(bar, 1u);
            const unsigned long long t0 = [] { unsigned long long t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t; }();
            unsigned polls = 0;
            s_stop = 0;
            while ((int)(*(volatile unsigned*)bar - target) < 0) {
                if (*(volatile int*)err) { s_stop = 1; break; }
                if ((++polls & 1023) == 0) {
                    unsigned long long t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (t - t0 > 2000000000ull) { atomicExch(err, 1); s_stop = 1; break; }
                }
            }
            __threadfence();
        }
        __syncthreads();
        return s_stop == 0;
    };
    local_best();
    int k = 0;
    for (; k < r; ++k) {
        if (!grid_barrier()) break;
        if (tid == 0) {
            double bv = -1.0;
            int bb = -1;
            for (int c = 0; c < G; ++c) {
                const double v = *(volatile double*)&cval[c];
                const int ix = *(volatile int*)&cidx[c];
                if (v > bv || (v == bv && ix >= 0 && (bb < 0 || ix < bb))) { bv = v; bb = ix; }
            }
            if (k == 0) s_dmax = bv;
            s_piv = (bb >= 0 && bv > rel_floor * s_dmax) ? bb : -1;
            s_pv = (s_piv >= 0) ? sqrt(bv) : 0.0;
        }
        __syncthreads();
        const int p = s_piv;
        if (p < 0) break;   // (every CTA reads the same candidates: all stop here together)
        const double inv = 1.0 / s_pv;
        for (int i = i0 + tid; i < i1; i += 256) {
            double v = M[(long long)p * ldm + i];
            for (int t = 0; t < k; ++t) v -= Zt[t * ldz + i] * __ldcg(Zt + t * ldz + p);
            const double z = (i == p) ? s_pv : v * inv;
            Zt[k * ldz + i] = z;
            d[i] = (i == p) ? -1.0 : d[i] - z * z;
        }
        __syncthreads();
        local_best();
    }
    if (b == 0 && tid == 0) *rank_out = k;
}

// ------------------------------------------------------------- small helpers
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, long long ldi, T* __restrict__ out,
                                 long long ldo, int rows, int cols) {
    PCG_COUNT_KERNEL();
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = by + r, j = bx + threadIdx.x;
        if (i < rows && j < cols) tile[r][threadIdx.x] = in[i * ldi + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = bx + r, i = by + threadIdx.x;
        if (i < rows && j < cols) out[j * ldo + i] = tile[threadIdx.x][r];
    }
}

template <typename T>
inline void transpose(const T* in, long long ldi, T* out, long long ldo, int rows, int cols,
                      cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_kernel<T><<<grid, block, 0, s>>>(in, ldi, out, ldo, rows, cols);
}

// out[i*ldo + j] = (TO) in[i*ldi + j] * (colscale ? colscale[j] : 1)
template <typename TI, typename TO>
__global__ void convert2d_kernel(const TI* __restrict__ in, long long ldi, TO* __restrict__ out,
                                 long long ldo, int rows, int cols, const double* __restrict__ colscale) {
    PCG_COUNT_KERNEL();
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        double v = (double)in[i * ldi + j];
        if (colscale) v *= colscale[j];
        out[i * ldo + j] = (TO)v;
    }
}

template <typename TI, typename TO>
inline void convert2d(const TI* in, long long ldi, TO* out, long long ldo, int rows, int cols,
                      cudaStream_t s, const double* colscale = nullptr) {
    if (rows <= 0 || cols <= 0) return;
    long long total = (long long)rows * cols;
    long long want = (total + 255) / 256;
    int blocks = (int)(want < 152LL * 16 ? want : 152LL * 16);
    convert2d_kernel<TI, TO><<<blocks, 256, 0, s>>>(in, ldi, out, ldo, rows, cols, colscale);
}

// Jacobi-scaled preconditioner matrix P~ = Sg (D + T) Sg + shift I, Sg = diag(D + T)^{-1/2}
// (lower triangle), and sg = diag(Sg).
template <typename T>
__global__ void build_scaled_ph_kernel(const T* __restrict__ Tm, long long ldt, const T* __restrict__ D,
                                       T* __restrict__ P, long long ldp, T* __restrict__ sg, int m,
                                       double shift) {
    PCG_COUNT_KERNEL();
    const long long total = (long long)m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        if (j > i) continue;
        const double di = (double)Tm[i * ldt + i] + (double)D[i];
        const double dj = (double)Tm[j * ldt + j] + (double)D[j];
        const double si = 1.0 / sqrt(di), sj = 1.0 / sqrt(dj);
        double v = (double)Tm[i * ldt + j];
        if (i == j) {
            v = 1.0 + shift;
            sg[i] = (T)si;
        } else {
            v *= si * sj;
        }
        P[i * ldp + j] = (T)v;
    }
}

}  // namespace pcgipm
