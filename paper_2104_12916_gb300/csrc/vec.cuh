// vec.cuh -- PCG vector updates (fused, with per-CTA partial dot products) and
// the FP64 elementwise / reduction kernels of the IPM iteration.
#pragma once

#include "common.cuh"

namespace pcgipm {

constexpr int kVecThreads = 256;

// Device-resident state of one PCG solve.  Each field is written by exactly one
// kernel of an iteration (thread 0 of block 0) and read only by the kernels that
// follow it, so no kernel reads a field it may be writing.
struct PcgState {
    double rz_cur;    // r'z of the current iterate (written by init2 / beta)
    double rz_prev;   // r'z used by the next beta (written by alpha)
    double bb;        // |rhs|^2
    double rr;        // |r|^2 after the last completed iteration
    double tol2;      // tol^2 |rhs|^2
    double alpha;     // last step length (diagnostic)
    int iter;         // completed iterations (written by beta)
    int iter_next;    // iter + 1 (written by alpha, read by beta)
    int done;         // 0 running, 1 converged, 2 iteration limit, 3 non-finite, 4 stagnated
    int maxit;
    double best_rr;   // smallest |r|^2 seen (read and written by thread 0 of block 0 only)
    int best_it;      // iteration of the last 4x improvement of best_rr
    int stall;        // iterations without a 4x improvement that count as stagnation (0: off)
};

enum PcKind { PC_NONE_K = 0, PC_L_K = 1, PC_H_K = 2 };

inline int vec_grid(int m) {
    int g = (m + kVecThreads - 1) / kVecThreads;
    return g < 1 ? 1 : (g > 2 * 152 ? 2 * 152 : g);
}

// x = 0, r = rhs; PL: z = r / D (dinv = 1/D), NONE: z = r, PH: rs = sg r (the
// Jacobi-scaled residual, in the preconditioner's precision TZ); partials of
// |r|^2 and r'z.
template <typename T, typename TZ, int PC>
__global__ void __launch_bounds__(kVecThreads) pcg_init1_kernel(int m, const T* __restrict__ rhs,
                                                                T* __restrict__ x, T* __restrict__ r,
                                                                T* __restrict__ z, const T* __restrict__ dinv,
                                                                TZ* __restrict__ rs, const TZ* __restrict__ sg,
                                                                double* bb_part, double* rz_part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    double bb = 0.0, rz = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads) {
        const T ri = rhs[i];
        x[i] = T(0);
        r[i] = ri;
        bb += (double)ri * (double)ri;
        if (PC == PC_L_K) { const T zi = ri * dinv[i]; z[i] = zi; rz += (double)ri * (double)zi; }
        if (PC == PC_NONE_K) { z[i] = ri; rz += (double)ri * (double)ri; }
        if (PC == PC_H_K) { rs[i] = (TZ)((double)ri * (double)sg[i]); }
    }
    bb = block_sum<kVecThreads>(bb, sh);
    rz = block_sum<kVecThreads>(rz, sh);
    if (threadIdx.x == 0) { bb_part[blockIdx.x] = bb; rz_part[blockIdx.x] = rz; }
}

// p = z; state <- (r'z, |rhs|^2, tol, maxit).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) pcg_init2_kernel(int m, PcgState* st, const T* __restrict__ z,
                                                                T* __restrict__ p, const double* bb_part, int nbb,
                                                                const double* rz_part, int nrz, double tol,
                                                                int maxit, int stall) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    const double bb = reduce_partials<kVecThreads>(bb_part, nbb, sh);
    const double rz = reduce_partials<kVecThreads>(rz_part, nrz, sh);
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads) p[i] = z[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rz_cur = rz;
        st->rz_prev = rz;
        st->bb = bb;
        st->rr = bb;
        st->tol2 = tol * tol * bb;
        st->alpha = 0.0;
        st->iter = 0;
        st->iter_next = 0;
        st->maxit = maxit;
        st->best_rr = bb;
        st->best_it = 0;
        st->stall = stall;
        st->done = (bb == 0.0) ? 1 : ((maxit <= 0) ? 2 : 0);
    }
}

// alpha = r'z / p'q;  x += alpha p;  r -= alpha q;  then the preconditioner's
// elementwise part: PL z = r / D, NONE z = r, PH rs = sg r (input of the
// triangular products, precision TZ).  Partials of |r|^2 and (PL/NONE) r'z.
template <typename T, typename TZ, int PC>
__global__ void __launch_bounds__(kVecThreads) pcg_alpha_kernel(int m, PcgState* st, const double* pq_part,
                                                                int npq, T* __restrict__ x, T* __restrict__ r,
                                                                const T* __restrict__ p, const T* __restrict__ q,
                                                                T* __restrict__ z, const T* __restrict__ dinv,
                                                                TZ* __restrict__ rs, const TZ* __restrict__ sg,
                                                                double* rr_part, double* rz_part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    if (st->done) return;
    const double pq = reduce_partials<kVecThreads>(pq_part, npq, sh);
    const double rz0 = st->rz_cur;
    if (!(pq > 0.0) || !isfinite(pq)) {   // breakdown: keep the last iterate, stop
        if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 3;
        return;
    }
    const double alpha = rz0 / pq;
    const T a = (T)alpha;
    double rr = 0.0, rz = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads) {
        x[i] = fma(a, p[i], x[i]);
        const T ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        rr += (double)ri * (double)ri;
        if (PC == PC_L_K) { const T zi = ri * dinv[i]; z[i] = zi; rz += (double)ri * (double)zi; }
        if (PC == PC_NONE_K) { z[i] = ri; rz += (double)ri * (double)ri; }
        if (PC == PC_H_K) { rs[i] = (TZ)((double)ri * (double)sg[i]); }
    }
    rr = block_sum<kVecThreads>(rr, sh);
    rz = block_sum<kVecThreads>(rz, sh);
    if (threadIdx.x == 0) {
        rr_part[blockIdx.x] = rr;
        if (PC != PC_H_K) rz_part[blockIdx.x] = rz;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rz_prev = rz0;
        st->alpha = alpha;
        st->iter_next = st->iter + 1;
    }
}

// beta = r'z_new / r'z_old;  p = z + beta p;  convergence test |r| <= tol |rhs|.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) pcg_beta_kernel(int m, PcgState* st, const T* __restrict__ z,
                                                               T* __restrict__ p, const double* rz_part, int nrz,
                                                               const double* rr_part, int nrr) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    if (st->done) return;
    const double rz = reduce_partials<kVecThreads>(rz_part, nrz, sh);
    const double rr = reduce_partials<kVecThreads>(rr_part, nrr, sh);
    const int it = st->iter_next;
    const bool finite = isfinite(rr) && isfinite(rz);
    const bool conv = finite && rr <= st->tol2;
    const bool stop = conv || !finite || it >= st->maxit;
    if (!stop) {
        const T beta = (T)(rz / st->rz_prev);
        for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads)
            p[i] = fma(beta, p[i], z[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->rz_cur = rz;
        st->rr = rr;
        st->iter = it;
        int dn = stop ? (conv ? 1 : (!finite ? 3 : 2)) : 0;
        // Stagnation (finite-precision limit of the recursive residual): no 4x
        // decrease of the best residual for `stall` iterations.  Decided by this
        // thread alone; other blocks may already have updated p, which no longer
        // matters once the loop ends.
        if (rr < 0.0625 * st->best_rr) { st->best_rr = rr; st->best_it = it; }
        if (!dn && st->stall > 0 && it - st->best_it >= st->stall) dn = 4;
        if (dn) st->done = dn;
    }
}

// ------------------------------------------------------------ generic vectors
// y = a x + b y  (any T)
template <typename TX, typename TY>
__global__ void axpby_kernel(int n, double a, const TX* __restrict__ x, double b, TY* __restrict__ y) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = a * (double)x[i];
        if (b != 0.0) v += b * (double)y[i];
        y[i] = (TY)v;
    }
}

template <typename TX, typename TY>
inline void axpby(int n, double a, const TX* x, double b, TY* y, cudaStream_t s) {
    if (n <= 0) return;
    axpby_kernel<TX, TY><<<vec_grid(n), kVecThreads, 0, s>>>(n, a, x, b, y);
}

// Partials of sum(v^2) and max|v| (FP64).
__global__ void norms_kernel(int n, const double* __restrict__ v, double* sq_part, double* max_part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    double sq = 0.0, mx = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads) {
        const double t = v[i];
        sq += t * t;
        mx = fmax(mx, fabs(t));
    }
    sq = block_sum<kVecThreads>(sq, sh);
    mx = block_max<kVecThreads>(mx, sh);
    if (threadIdx.x == 0) { sq_part[blockIdx.x] = sq; max_part[blockIdx.x] = mx; }
}

// Partials of sum(a_i * b_i) (FP64).
__global__ void dot_kernel(int n, const double* __restrict__ a, const double* __restrict__ b, double* part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    double s = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads)
        s += a[i] * b[i];
    s = block_sum<kVecThreads>(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One block folds partial arrays into scalars: out[k] = op_k(parts_k[0..cnt_k)).
struct ReduceJob {
    const double* part[8];
    int cnt[8];
    int op[8];   // 0 sum, 1 max, 2 min
    int njobs;
};

__global__ void reduce_jobs_kernel(ReduceJob job, double* out) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    for (int k = 0; k < job.njobs; ++k) {
        double v = job.op[k] == 0 ? 0.0 : (job.op[k] == 1 ? -1.0e308 : 1.0e308);
        for (int i = threadIdx.x; i < job.cnt[k]; i += kVecThreads) {
            const double t = job.part[k][i];
            v = job.op[k] == 0 ? v + t : (job.op[k] == 1 ? fmax(v, t) : fmin(v, t));
        }
        if (job.op[k] == 0) v = block_sum<kVecThreads>(v, sh);
        else if (job.op[k] == 1) v = block_max<kVecThreads>(v, sh);
        else v = block_min<kVecThreads>(v, sh);
        if (threadIdx.x == 0) out[k] = v;
        __syncthreads();
    }
}

// ---------------------------------------------------------- IPM elementwise
// r_c = s nu + (corr ? ds_a dnu_a : 0) - sigma_mu;  r_a = r_i + r_c / nu
// (eq. [rhs-KKT4] and r_a of eq. [augmented]); D = s / nu (eq. [diag-d]).
__global__ void ipm_rc_kernel(int m, const double* __restrict__ s, const double* __restrict__ nu,
                              const double* __restrict__ r_i, const double* __restrict__ ds_a,
                              const double* __restrict__ dn_a, double sigma_mu, double* __restrict__ r_c,
                              double* __restrict__ r_a, double* __restrict__ D) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double rc = s[i] * nu[i] - sigma_mu;
        if (ds_a) rc += ds_a[i] * dn_a[i];
        r_c[i] = rc;
        r_a[i] = r_i[i] + rc / nu[i];
        if (D) D[i] = s[i] / nu[i];
    }
}

// ds = -r_c / nu - D dnu  (eq. [delz])
__global__ void ipm_ds_kernel(int m, const double* __restrict__ r_c, const double* __restrict__ nu,
                              const double* __restrict__ D, const double* __restrict__ dnu,
                              double* __restrict__ ds) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        ds[i] = -r_c[i] / nu[i] - D[i] * dnu[i];
}

// Partials of the largest step keeping s, nu >= 0: min over negative components.
__global__ void ipm_maxstep_kernel(int m, const double* __restrict__ s, const double* __restrict__ ds,
                                   const double* __restrict__ nu, const double* __restrict__ dnu,
                                   double* part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    double a = 1.0e308;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads) {
        if (ds[i] < 0.0) a = fmin(a, -s[i] / ds[i]);
        if (dnu[i] < 0.0) a = fmin(a, -nu[i] / dnu[i]);
    }
    a = block_min<kVecThreads>(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// Partials of (s + a ds)'(nu + a dnu).
__global__ void ipm_muaff_kernel(int m, const double* __restrict__ s, const double* __restrict__ ds,
                                 const double* __restrict__ nu, const double* __restrict__ dnu, double a,
                                 double* part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    double t = 0.0;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < m; i += gridDim.x * kVecThreads)
        t += (s[i] + a * ds[i]) * (nu[i] + a * dnu[i]);
    t = block_sum<kVecThreads>(t, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// s0 = max(C x0 - d, 1), nu0 = 1 (start point).
__global__ void ipm_start_kernel(int m, const double* __restrict__ cx_minus_d, double* __restrict__ s,
                                 double* __restrict__ nu) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        s[i] = fmax(cx_minus_d[i], 1.0);
        nu[i] = 1.0;
    }
}

// out = (TO) (scale * in)
template <typename TI, typename TO>
__global__ void convert1d_kernel(int n, const TI* __restrict__ in, double scale, TO* __restrict__ out) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (TO)(scale * (double)in[i]);
}

template <typename TI, typename TO>
inline void convert1d(int n, const TI* in, double scale, TO* out, cudaStream_t s) {
    if (n <= 0) return;
    convert1d_kernel<TI, TO><<<vec_grid(n), kVecThreads, 0, s>>>(n, in, scale, out);
}

// Elementwise reciprocal (FP64 in, T out): out = 1 / in.
template <typename T>
__global__ void recip_kernel(int n, const double* __restrict__ in, T* __restrict__ out) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (T)(1.0 / in[i]);
}

// hs_j = 1 / sqrt(H_jj)  (column scaling of the diag(H)^{-1} variant of P_H)
__global__ void diag_rsqrt_kernel(int n, const double* __restrict__ H, long long ld, double* __restrict__ hs) {
    PCG_COUNT_KERNEL();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        hs[i] = 1.0 / sqrt(H[i * ld + i]);
}

// Dense expansion of a CSR matrix into a zeroed row-major array (one thread per
// row, entries added in storage order, so repeated columns are summed the same
// way every time).  A bad row pointer or column index sets *bad.
__global__ void csr_scatter_kernel(int rows, int cols, long long nnz, const int* __restrict__ rowptr,
                                   const int* __restrict__ colidx, const double* __restrict__ val,
                                   double* __restrict__ M, long long ld, int* bad) {
    PCG_COUNT_KERNEL();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const long long k0 = rowptr[i], k1 = rowptr[i + 1];
    if ((i == 0 && k0 != 0) || k0 < 0 || k1 < k0 || k1 > nnz) {
        atomicAdd(bad, 1);
        return;
    }
    for (long long k = k0; k < k1; ++k) {
        const int j = colidx[k];
        if (j < 0 || j >= cols) {
            atomicAdd(bad, 1);
            continue;
        }
        M[(long long)i * ld + j] += val[k];
    }
}

// Count of non-finite entries (for input validation), added to *bad.
__global__ void nonfinite_kernel(long long n, const double* __restrict__ v, int* bad) {
    PCG_COUNT_KERNEL();
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        c += !isfinite(v[i]);
    if (c) atomicAdd(bad, c);
}

// max |H_ij - H_ji| / max(|H_ij|, 1) over the lower triangle, folded into *out (as int bits of a
// non-negative float via atomicMax on the float's bit pattern).
__global__ void asym_kernel(int n, const double* __restrict__ H, long long ld, unsigned int* out) {
    PCG_COUNT_KERNEL();
    float worst = 0.f;
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (j >= i) continue;
        const double a = H[i * ld + j], b = H[j * ld + i];
        const double sc = fmax(fmax(fabs(a), fabs(b)), 1e-300);
        worst = fmaxf(worst, (float)(fabs(a - b) / sc));
    }
    atomicMax(out, __float_as_uint(worst));
}

// Row sums of |H| partial max: max_i sum_j |H_ij| (one warp per row).
__global__ void absrowsum_max_kernel(int n, const double* __restrict__ H, long long ld, double* part) {
    PCG_COUNT_KERNEL();
    __shared__ double sh[40];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double best = 0.0;
    for (int row = blockIdx.x * 8 + warp; row < n; row += gridDim.x * 8) {
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += fabs(H[row * ld + j]);
        s = warp_sum(s);
        best = fmax(best, s);
    }
    best = block_max<kVecThreads>(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

}  // namespace pcgipm
