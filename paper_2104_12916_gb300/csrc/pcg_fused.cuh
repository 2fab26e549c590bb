// pcg_fused.cuh -- the PCG hot loop (a6-a10) as one persistent cooperative kernel.
//
// One launch runs every iteration of one PCG solve on K_F dnu = r_nu.  An
// iteration is a chain of row-major matrix-vector phases (C' p, R^{-T} u,
// Gt z1, Gt' z2, R^{-1} t, C y, then for P_H the two triangles of the inverse
// factor of P~), separated by a grid barrier.
//
// Layout of the work: a matrix is cut into chunks of 32 lanes x 8 x 16 bytes
// (1024 FP32 or 512 FP64 elements) of one row; warps of the whole grid take
// chunks round-robin and each lane keeps 8 independent 16-byte loads in flight.
// Each chunk writes one partial sum; the next phase, while staging its input
// vector into shared memory, adds a row's chunk partials in a fixed order and
// applies the elementwise part of the method (D p, z1 + ..., the Jacobi
// scaling, the PCG updates).  The PCG dot products (p'q, |r|^2, r'z) are summed
// by every CTA over the whole vector in the same fixed order, so every CTA holds
// bit-identical scalars without a reduction barrier.  Vectors read and written in
// one phase (r, p) are double-buffered; each CTA writes only its own slice.
//
// Chunks that lie entirely outside a triangle are skipped (no load, no
// partial); inside a chunk, the zeros the triangle stores in memory are read.
//
// Every barrier wait is bounded: after kSpinLimit polls a block records
// QP_ETIMEOUT in the barrier word and returns, and every other block returns at
// its next barrier.
#pragma once

#include "common.cuh"
#include "dense.cuh"
#include "vec.cuh"

namespace pcgipm {

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr unsigned long long kSpinLimit = 1ull << 25;   // ~ seconds with the 64 ns back-off

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

// Accumulation type of the staging sums and PCG scalars inside the fused kernel:
// the working precision itself.  (GB300's FP64 pipe issues two FMAs per clock per
// SM, so an FP32 path must not touch FP64 arithmetic in its inner loops.)
template <typename T> struct Acc { using type = T; };

// Elements of one chunk for matrix element type T.
template <typename T> struct Chunk { static constexpr int n = 32 * 8 * (16 / sizeof(T)); };

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier: thread 0 of each block arrives with a release add on the counter;
// the last arrival resets it and publishes the next generation with a release add;
// the others poll the generation with acquire loads (bounded, see kSpinLimit).
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire(&b->gen);
        unsigned arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&b->count) : "memory");
        if (arrived + 1u == nblocks) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&b->count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&b->gen) : "memory");
        } else {
            unsigned long long spins = 0;
            while (ld_acquire(&b->gen) == g) {
                if (++spins > kSpinLimit) {
                    atomicExch(&b->err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        *s_flag = *((volatile int*)&b->err);
    }
    __syncthreads();
    return *s_flag == 0;
}

// Items of a chunked GEMV phase: (row, chunk) pairs, chunk-column-major, with
// the chunks that lie entirely outside a triangle left out so that the work is
// spread evenly over the warps.  Chunk column c holds rows [r0(c), r1(c)):
// all rows (TRI_NONE), rows >= c*CH (lower), rows < (c+1)*CH (upper).
template <int TRI>
__device__ __forceinline__ void chunk_rows(int c, int CH, int rows, int& r0, int& r1) {
    r0 = 0;
    r1 = rows;
    if (TRI == TRI_LOWER) r0 = min(rows, c * CH);
    if (TRI == TRI_UPPER) r1 = min(rows, (c + 1) * CH);
}

template <int TRI>
__device__ __forceinline__ long long chunk_items(int rows, int cols, int CH) {
    const int nc = (cols + CH - 1) / CH;
    if (TRI == TRI_NONE) return (long long)rows * nc;
    long long t = 0;
    for (int c = 0; c < nc; ++c) {
        int r0, r1;
        chunk_rows<TRI>(c, CH, rows, r0, r1);
        t += r1 - r0;
    }
    return t;
}

// Item index -> (row, chunk).  `c`/`base` carry the last chunk column found so a
// warp walking increasing item indices moves forward through the columns.
template <int TRI>
__device__ __forceinline__ void item_at(long long it, int rows, int nc, int CH, int& c, long long& base,
                                        int& row) {
    if constexpr (TRI == TRI_NONE) {
        c = (int)(it / rows);
        row = (int)(it - (long long)c * rows);
        return;
    }
    while (true) {
        int r0, r1;
        chunk_rows<TRI>(c, CH, rows, r0, r1);
        if (it < base + (r1 - r0) || c == nc - 1) {
            row = r0 + (int)(it - base);
            return;
        }
        base += r1 - r0;
        ++c;
    }
}

// Hint the 4 KB chunk (row, c) into L2 (one 128-byte line per lane).
template <typename TM>
__device__ __forceinline__ void prefetch_chunk(const TM* M, long long ld, int row, int c, int cols) {
    constexpr int CH = Chunk<TM>::n;
    const int lane = threadIdx.x & 31;
    const long long e = (long long)c * CH + (long long)lane * (128 / sizeof(TM));
    if (e < ld) {
        const TM* addr = M + (long long)row * ld + e;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(addr));
    }
}

// L2 hint of this warp's first item of a coming phase (issued before a barrier),
// with the item assignment of gemv_chunks.
template <typename TM, int TRI>
__device__ __forceinline__ void prefetch_first(const TM* M, int rows, int cols, long long ld, int flags = 0) {
    constexpr int CH = Chunk<TM>::n;
    const int warp = threadIdx.x >> 5;
    const int nc = (cols + CH - 1) / CH;
    const long long nitems = chunk_items<TRI>(rows, cols, CH);
    long long first, last;
    if (flags & 2) {
        first = blockIdx.x * kFusedWarps + warp;
        last = nitems;
    } else {
        const long long per = (nitems + gridDim.x - 1) / gridDim.x;
        first = (long long)blockIdx.x * per + warp;
        last = min(nitems, (long long)blockIdx.x * per + per);
    }
    if (first >= last || (flags & 4)) return;
    int c = 0, row = 0;
    long long base = 0;
    item_at<TRI>(first, rows, nc, CH, c, base, row);
    prefetch_chunk<TM>(M, ld, row, c, cols);
}

// Chunked GEMV phase: part[c * pld + row] = sum over chunk c of row `row` of M . xs
// (chunk-major, so that the consumer's per-row sums load coalesced).
// TRI: TRI_NONE / TRI_LOWER (square) / TRI_UPPER (square).
// Each block takes a contiguous range of items (rows next to each other in one
// chunk column: few pages, sequential DRAM rows) and its warps interleave
// within it.  flags bit 0: no L2 prefetch of the next item; bit 1: round-robin
// items over all warps of the grid instead.
template <typename TM, int TRI>
__device__ __forceinline__ void gemv_chunks(const TM* __restrict__ M, int rows, int cols, long long ld,
                                            const TM* __restrict__ xs, TM* __restrict__ part, int pld,
                                            int flags = 0) {
    using VT = Vec16<TM>;
    using V = typename VT::type;
    constexpr int CH = Chunk<TM>::n;
    constexpr int VN = VT::n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = (cols + CH - 1) / CH;
    const long long nitems = chunk_items<TRI>(rows, cols, CH);
    long long first, step, last;
    if (flags & 2) {
        first = blockIdx.x * kFusedWarps + warp;
        step = (long long)gridDim.x * kFusedWarps;
        last = nitems;
    } else {
        const long long per = (nitems + gridDim.x - 1) / gridDim.x;
        const long long b0 = (long long)blockIdx.x * per;
        first = b0 + warp;
        step = kFusedWarps;
        last = min(nitems, b0 + per);
    }
    const V* xv = reinterpret_cast<const V*>(xs);
    int c = 0, row = 0;
    long long base = 0;
    if (first < last) item_at<TRI>(first, rows, nc, CH, c, base, row);
    for (long long it = first; it < last; it += step) {
        const int crow = row, cc = c;
        // locate (and L2-prefetch) the next item while this one loads
        if (it + step < last) {
            item_at<TRI>(it + step, rows, nc, CH, c, base, row);
            if (!(flags & 1)) prefetch_chunk<TM>(M, ld, row, c, cols);
        }
        const V* mr = reinterpret_cast<const V*>(M + (long long)crow * ld + (long long)cc * CH);
        const int vbase = cc * (CH / VN);
        const int vend = (int)(ld / VN) - vbase;   // vectors of this row left from the chunk start
        V a[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int v = lane + 32 * k;
            a[k] = (v < vend) ? __ldg(mr + v) : V{};
        }
        TM acc = TM(0);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = VT::dot(a[k], xv[vbase + lane + 32 * k], acc);
        acc = warp_sum(acc);
        if (lane == 0) part[(long long)cc * pld + crow] = acc;
    }
}

// Chunk sums of four rows j[0..3] at once (rows >= len give 0): for each row the
// chunks are added in increasing order (the same order as row_total), but the
// loads of all four rows and four consecutive chunks are issued together.
template <typename TM, int TRI, typename AT>
__device__ __forceinline__ void sum_chunks4(const TM* __restrict__ part, int pld, int cols, const int* j,
                                            int len, AT* out) {
    constexpr int CH = Chunk<TM>::n;
    const int nc = (cols + CH - 1) / CH;
    int c0[4], c1[4];
    int cmin = nc, cmax = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        c0[u] = 0;
        c1[u] = (j[u] < len) ? nc : 0;
        if (TRI == TRI_LOWER && j[u] < len) c1[u] = j[u] / CH + 1;
        if (TRI == TRI_UPPER && j[u] < len) c0[u] = j[u] / CH;
        out[u] = AT(0);
        if (c0[u] < c1[u]) {
            cmin = min(cmin, c0[u]);
            cmax = max(cmax, c1[u]);
        }
    }
    for (int c = cmin; c < cmax; c += 4) {
        TM v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int cc = c + k;
                v[u][k] = (cc >= c0[u] && cc < c1[u]) ? __ldcg(part + (long long)cc * pld + j[u]) : TM(0);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 4; ++k) out[u] += (AT)v[u][k];
    }
}

// Stage xs[j] for j < pad (zero from len on): rows are taken four per thread;
// f(j4, valid, s4, val4) turns the four chunk sums into the four values.
template <typename TX, typename TM, int TRI, class F>
__device__ __forceinline__ void stage_sum(TX* xs, const TM* part, int pld, int cols, int len, int pad, F f) {
    using AT = typename Acc<TM>::type;
    for (int j0 = threadIdx.x; j0 < pad; j0 += 4 * kFusedThreads) {
        int j[4];
        AT sm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = j0 + u * kFusedThreads;
        sum_chunks4<TM, TRI, AT>(part, pld, cols, j, len, sm);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j[u] < pad) xs[j[u]] = (j[u] < len) ? f(j[u], sm[u]) : TX(0);
    }
}

// Block-wide fixed-order sum, result broadcast to every thread.
template <typename AT>
__device__ __forceinline__ AT block_allsum(AT v, AT* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        AT r = (l < kFusedWarps) ? sh[l] : AT(0);
        r = warp_sum(r);
        if (l == 0) sh[32] = r;
    }
    __syncthreads();
    v = sh[32];
    __syncthreads();
    return v;
}

template <typename TO, typename TP>
struct FusedArgs {
    int n, m1, m2;
    // operator (precision TO)
    const TO *CWT, *WH, *Gt, *GtT, *WHT, *CW;
    long long ldCWT, ldWH, ldGt, ldGtT, ldWHT, ldCW;
    // preconditioner (precision TP)
    const TP *WPl, *WPu;
    long long ldWP;
    const TP* sg;
    // vectors
    const TO* D;
    const TO* Dinv;
    TO* x;
    TO *r0, *r1, *p0, *p1;
    // chunk partials
    TO *PU, *PZ1, *PZ2, *PT, *PY, *PQ;
    TP *PV, *PZ;
    int ldU, ldZ1, ldZ2, ldT, ldY, ldQ, ldV, ldZ;
    PcgState* st;      // entry: rz_cur, tol2, maxit, done (from pcg_init); exit: iter, rr, done
    GridBar* bar;
    size_t xs_bytes;   // bytes of the staged-vector region of shared memory (16-byte multiple)
    unsigned long long* tstamp;   // optional: %globaltimer at phase marks of the first 4 iterations
    int flags;                    // bit 0: no next-item L2 prefetch; bit 1: round-robin items; bit 2: no
                                  // prefetch of the next phase before a barrier
};

// kind: PC_L_K (z = r / D), PC_H_K (z = Sg W' W Sg r), PC_NONE_K (z = r).
// Entry state (from pcg_init): x = 0, r = r0 = rhs, p = p0 = z0, st->rz_cur = r'z,
// st->tol2 = tol^2 |rhs|^2, st->maxit.  Shared memory: the staged vector
// (xs_bytes) followed by three m2-vectors in TO: q = K_F p, r and p of the
// current iteration.
template <typename TO, typename TP, int PC>
__global__ void __launch_bounds__(kFusedThreads, 1) pcg_fused_kernel(const FusedArgs<TO, TP> a) {
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TO* xs = reinterpret_cast<TO*>(smem_raw);
    TP* xp = reinterpret_cast<TP*>(smem_raw);
    TO* qc = reinterpret_cast<TO*>(smem_raw + a.xs_bytes);
    TO* rc = qc + a.m2;
    TO* pcs = rc + a.m2;
    using AT = typename Acc<TO>::type;
    __shared__ AT sh[40];
    __shared__ int s_flag;
    const int n = a.n, m1 = a.m1, m2 = a.m2;
    const int tid = threadIdx.x;
    const unsigned nblocks = gridDim.x;
    // slice of the m2-vectors this block owns for writes
    const int per = (m2 + nblocks - 1) / nblocks;
    const int own0 = blockIdx.x * per, own1 = min(m2, own0 + per);
    constexpr int CHO = Chunk<TO>::n, CHP = Chunk<TP>::n;
    const int padO_n = ((n + CHO - 1) / CHO) * CHO, padO_m2 = ((m2 + CHO - 1) / CHO) * CHO;
    const int padO_m1 = ((m1 + CHO - 1) / CHO) * CHO, padP_m2 = ((m2 + CHP - 1) / CHP) * CHP;
    const bool stamp = a.tstamp != nullptr && blockIdx.x == 0 && tid == 0;
    auto mark = [&](int it, int ph) {
        if (stamp && it < 4) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            a.tstamp[it * 32 + ph] = t;
        }
    };

    if (__ldcg(&a.st->done)) return;
    AT rz = (AT)__ldcg(&a.st->rz_cur);
    const double tol2 = __ldcg(&a.st->tol2);
    const int maxit = __ldcg(&a.st->maxit);
    int it = 0;
    int done = 0;
    AT rr = AT(0);
    TO* pc = a.p0;  TO* pn = a.p1;
    TO* rcur = a.r0; TO* rnext = a.r1;

    // first iteration: p and r from the entry state; xs = p
    for (int j = tid; j < m2; j += kFusedThreads) {
        pcs[j] = __ldcg(pc + j);
        rc[j] = __ldcg(rcur + j);
    }
    __syncthreads();
    for (int j = tid; j < padO_m2; j += kFusedThreads) xs[j] = (j < m2) ? pcs[j] : TO(0);
    __syncthreads();

    while (true) {
        mark(it, 0);
        // ---- P1 (a6): u = C' p
        gemv_chunks<TO, TRI_NONE>(a.CWT, n, m2, a.ldCWT, xs, a.PU, a.ldU, a.flags);
        mark(it, 11);
        prefetch_first<TO, TRI_LOWER>(a.WH, n, n, a.ldWH, a.flags);
        if (!grid_sync(a.bar, nblocks, &s_flag)) return;
        mark(it, 1);
        // ---- P2 (a7): z1 = R^{-T} u
        stage_sum<TO, TO, TRI_NONE>(xs, a.PU, a.ldU, m2, n, padO_n, [&](int, AT v) { return (TO)v; });
        __syncthreads();
        mark(it, 12);
        gemv_chunks<TO, TRI_LOWER>(a.WH, n, n, a.ldWH, xs, a.PZ1, a.ldZ1, a.flags);
        mark(it, 13);
        if (m1 > 0) prefetch_first<TO, TRI_NONE>(a.Gt, m1, n, a.ldGt, a.flags);
        else prefetch_first<TO, TRI_UPPER>(a.WHT, n, n, a.ldWHT, a.flags);
        if (!grid_sync(a.bar, nblocks, &s_flag)) return;
        mark(it, 2);
        if (m1 > 0) {
            // ---- P3: z2 = -Gt z1
            stage_sum<TO, TO, TRI_LOWER>(xs, a.PZ1, a.ldZ1, n, n, padO_n, [&](int, AT v) { return (TO)v; });
            __syncthreads();
            gemv_chunks<TO, TRI_NONE>(a.Gt, m1, n, a.ldGt, xs, a.PZ2, a.ldZ2, a.flags);
            prefetch_first<TO, TRI_NONE>(a.GtT, n, m1, a.ldGtT, a.flags);
            if (!grid_sync(a.bar, nblocks, &s_flag)) return;
            mark(it, 3);
            // ---- P4: t = z1 + Gt' z2
            stage_sum<TO, TO, TRI_NONE>(xs, a.PZ2, a.ldZ2, n, m1, padO_m1, [&](int, AT v) { return (TO)(-v); });
            __syncthreads();
            gemv_chunks<TO, TRI_NONE>(a.GtT, n, m1, a.ldGtT, xs, a.PT, a.ldT, a.flags);
            prefetch_first<TO, TRI_UPPER>(a.WHT, n, n, a.ldWHT, a.flags);
            if (!grid_sync(a.bar, nblocks, &s_flag)) return;
            mark(it, 4);
        }
        // ---- P5: y = R^{-1} t
        // t = z1 + Gt' z2: the Gt' partials first (into xs), then z1 added on top
        if (m1 > 0) {
            stage_sum<TO, TO, TRI_NONE>(xs, a.PT, a.ldT, m1, n, padO_n, [&](int, AT v) { return (TO)v; });
            __syncthreads();
            stage_sum<TO, TO, TRI_LOWER>(xs, a.PZ1, a.ldZ1, n, n, padO_n,
                                         [&](int j, AT v) { return (TO)(v + (AT)xs[j]); });
        } else {
            stage_sum<TO, TO, TRI_LOWER>(xs, a.PZ1, a.ldZ1, n, n, padO_n, [&](int, AT v) { return (TO)v; });
        }
        __syncthreads();
        mark(it, 14);
        gemv_chunks<TO, TRI_UPPER>(a.WHT, n, n, a.ldWHT, xs, a.PY, a.ldY, a.flags);
        mark(it, 15);
        prefetch_first<TO, TRI_NONE>(a.CW, m2, n, a.ldCW, a.flags);
        if (!grid_sync(a.bar, nblocks, &s_flag)) return;
        mark(it, 5);
        // ---- P6 (a8): q = D p + C y
        stage_sum<TO, TO, TRI_UPPER>(xs, a.PY, a.ldY, n, n, padO_n, [&](int, AT v) { return (TO)v; });
        __syncthreads();
        mark(it, 16);
        gemv_chunks<TO, TRI_NONE>(a.CW, m2, n, a.ldCW, xs, a.PQ, a.ldQ, a.flags);
        mark(it, 17);
        if (PC == PC_H_K) prefetch_first<TP, TRI_LOWER>(a.WPl, m2, m2, a.ldWP, a.flags);
        else prefetch_first<TO, TRI_NONE>(a.CWT, n, m2, a.ldCWT, a.flags);
        if (!grid_sync(a.bar, nblocks, &s_flag)) return;
        mark(it, 6);

        // ---- P7 (a10): q = D p + C y (cached), alpha = r'z / p'q, x += alpha p, r -= alpha q
        stage_sum<TO, TO, TRI_NONE>(qc, a.PQ, a.ldQ, n, m2, m2,
                                    [&](int j, AT v) { return (TO)fma((AT)__ldg(a.D + j), (AT)pcs[j], v); });
        __syncthreads();
        AT pq = AT(0);
        for (int j = tid; j < m2; j += kFusedThreads) pq = fma((AT)pcs[j], (AT)qc[j], pq);
        pq = block_allsum(pq, sh);
        // breakdown (p'q <= 0 or not finite): stop with the last iterate untouched
        if (!(pq > AT(0)) || !isfinite(pq)) { done = 3; break; }
        const AT alpha = rz / pq;
        const TO al = (TO)alpha;
        AT rrp = AT(0), rzp = AT(0);
        for (int j = tid; j < padO_m2; j += kFusedThreads) {
            if (j >= m2) {
                if (PC == PC_H_K) { if (j < padP_m2) xp[j] = TP(0); } else xs[j] = TO(0);
                continue;
            }
            const TO rn = fma(-al, qc[j], rc[j]);
            rc[j] = rn;
            rrp = fma((AT)rn, (AT)rn, rrp);
            if (j >= own0 && j < own1) {
                a.x[j] = fma(al, pcs[j], a.x[j]);
                rnext[j] = rn;
            }
            if (PC == PC_H_K) {
                xp[j] = (TP)((AT)rn * (AT)__ldg(a.sg + j));
            } else {
                const TO z = (PC == PC_L_K) ? rn * __ldg(a.Dinv + j) : rn;
                rzp = fma((AT)rn, (AT)z, rzp);
            }
        }
        if (PC == PC_H_K)
            for (int j = padO_m2 + tid; j < padP_m2; j += kFusedThreads) xp[j] = TP(0);
        rr = block_allsum(rrp, sh);
        ++it;
        const bool finite = isfinite(rr) && isfinite(pq);
        if (!finite) { done = 3; break; }
        if ((double)rr <= tol2) { done = 1; break; }
        if (it >= maxit) { done = 2; break; }
        mark(it - 1, 7);

        AT rz_new;
        if (PC == PC_H_K) {
            __syncthreads();
            // ---- P8 (a9): v = W rs, z = Sg W' v
            gemv_chunks<TP, TRI_LOWER>(a.WPl, m2, m2, a.ldWP, xp, a.PV, a.ldV, a.flags);
            mark(it - 1, 18);
            prefetch_first<TP, TRI_UPPER>(a.WPu, m2, m2, a.ldWP, a.flags);
            if (!grid_sync(a.bar, nblocks, &s_flag)) return;
            mark(it - 1, 8);
            stage_sum<TP, TP, TRI_LOWER>(xp, a.PV, a.ldV, m2, m2, padP_m2, [&](int, typename Acc<TP>::type v) { return (TP)v; });
            __syncthreads();
            mark(it - 1, 19);
            gemv_chunks<TP, TRI_UPPER>(a.WPu, m2, m2, a.ldWP, xp, a.PZ, a.ldZ, a.flags);
            mark(it - 1, 20);
            prefetch_first<TO, TRI_NONE>(a.CWT, n, m2, a.ldCWT, a.flags);
            if (!grid_sync(a.bar, nblocks, &s_flag)) return;
            mark(it - 1, 9);
            // z into the q cache (q is no longer needed), then r'z
            stage_sum<TO, TP, TRI_UPPER>(qc, a.PZ, a.ldZ, m2, m2, m2,
                                         [&](int j, typename Acc<TP>::type v) { return (TO)((AT)__ldg(a.sg + j) * (AT)v); });
            __syncthreads();
            rzp = AT(0);
            for (int j = tid; j < m2; j += kFusedThreads) rzp = fma((AT)rc[j], (AT)qc[j], rzp);
            rz_new = block_allsum(rzp, sh);
        } else {
            rz_new = block_allsum(rzp, sh);
        }
        // ---- beta, p = z + beta p (staged as the next P1 input; shared-memory only)
        const AT beta = rz_new / rz;
        rz = rz_new;
        const TO be = (TO)beta;
        for (int j = tid; j < padO_m2; j += kFusedThreads) {
            TO v = TO(0);
            if (j < m2) {
                TO z;
                if (PC == PC_H_K) z = qc[j];
                else z = (PC == PC_L_K) ? rc[j] * __ldg(a.Dinv + j) : rc[j];
                v = fma(be, pcs[j], z);
                pcs[j] = v;
                if (j >= own0 && j < own1) pn[j] = v;
            }
            xs[j] = v;
        }
        __syncthreads();
        mark(it - 1, 10);
        // swap the double buffers (global copies; the shared caches already hold the new values)
        TO* t1 = pc; pc = pn; pn = t1;
        TO* t2 = rcur; rcur = rnext; rnext = t2;
    }
    if (blockIdx.x == 0 && tid == 0) {
        a.st->iter = it;
        a.st->rr = (double)rr;
        a.st->rz_cur = (double)rz;
        a.st->done = done;
    }
}

}  // namespace pcgipm
