// pcg_fused.cuh -- the PCG hot loop (a6-a10) as one persistent cooperative kernel.
//
// One launch runs every iteration of one PCG solve on K_F dnu = r_nu.  An
// iteration is a chain of row-major matrix-vector phases separated by grid
// barriers: u = C' p; the forward solve with the K0 factor L (stored as its
// inverse: z1 = R^{-T} u and z2 = -Et u together, Et = L_S^{-1} A H^{-1} the
// (2,1) block of L^{-1}); the back solve y = R^{-1} z1 + Et' z2; q = D p + C y;
// then for P_H the two triangles of the inverse factor of P~.
//
// Layout of the work: a matrix is cut into chunks of 4 KB of one row (1024 FP32
// or 512 FP64 elements).  Each block owns a contiguous range of the chunks of
// every phase (rows next to each other in one chunk column).  The matrices do
// not change during the solve, so their stream need not wait for the barriers:
// a producer warp copies the block's chunks, phase after phase and iteration
// after iteration, into a ring of shared-memory slots with bulk asynchronous
// copies (cp.async.bulk, completion counted on one mbarrier per slot), running
// ahead of the consumers by up to the ring's depth -- across the grid barriers,
// where a kernel that only loads after the barrier leaves HBM idle.  The 15
// consumer warps take the block's chunks in turn, dot them with the staged
// vector and write one partial sum per chunk; the next phase, while staging its
// input vector, adds a row's chunk partials in a fixed order and applies the
// elementwise part of the method (D p, z1 + ..., the Jacobi scaling, the PCG
// updates).  The PCG dot products (p'q, |r|^2, r'z) are summed by every block
// over the whole vector in the same fixed order, so every block holds
// bit-identical scalars without a reduction barrier.  Vectors read and written
// in one phase (r, p) are double-buffered; each block writes only its own slice.
//
// Chunks that lie entirely outside a triangle are skipped (no copy, no
// partial); inside a chunk, the zeros the triangle stores in memory are read.
//
// Every wait is bounded in time (kWaitNs on %globaltimer): a consumer that gives
// up records QP_ETIMEOUT in the barrier word and every block returns at its next
// grid barrier; the producer stops when the consumers stop (or its own wait
// gives up) and then waits, again bounded, for the copies it has in flight.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "dense.cuh"
#include "vec.cuh"

namespace pcgipm {

// Block sizes: 512 threads for a QP that spreads over the GPU (one block per SM),
// 256 for a small QP (two blocks per SM, so that blocks of different QPs hide one
// another's barrier waits).  The last warp of a block is the producer.
constexpr int kBigBlock = 512, kSmallBlock = 256;
template <int NT> struct Blk {
    static constexpr int threads = NT - 32;            // consumer threads
    static constexpr int warps = threads / 32;         // consumer warps
    static constexpr int max_slots = 3 * warps;        // ring depths are multiples of `warps`
    static constexpr int small_slots = 2 * warps;      // ring of a QP that shares the GPU
};
constexpr int kSlotBytes = 4096;
constexpr int kMaxClusterBlocks = 16;             // grids up to this size launch as one cluster
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any wait

struct GridBar {
    unsigned int count;   // monotonic arrival counter (zeroed before each launch)
    unsigned int gen;
    int err;
    int pad;
};

// Accumulation type of the staging sums and PCG scalars inside the fused kernel:
// the working precision itself.  (GB300's FP64 pipe issues two FMAs per clock per
// SM, so an FP32 path must not touch FP64 arithmetic in its inner loops.)
template <typename T> struct Acc { using type = T; };

// Elements of one chunk for matrix element type T (one 4 KB slot).
template <typename T> struct Chunk { static constexpr int n = kSlotBytes / (int)sizeof(T); };

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------- mbarriers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of the completion of the phase of parity `parity` of `b`.
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16);
// completion is counted in bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Waits for the completion of the phase of parity `parity` of `b`; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(b, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

// Ring of chunk slots in shared memory.  Slot s holds the chunks g with
// g % S == s; its fill number is g / S.  full[s] completes one phase per copy
// (producer arrival + transaction bytes), empty[s] one phase per consumption
// (one arrival of the consuming warp).  A parity wait names the phase it waits
// for exactly only while the waiter is at most one phase ahead, so every slot
// has one owner on each side and each owner handles its slot's fills in order:
//  - producer lane s % 32 issues every fill of slot s; before fill f it waits
//    for the consumption of fill f - 1, and it had waited for that of f - 2
//    before issuing f - 1;
//  - S is a multiple of the consumer warp count W and chunk g goes to consumer
//    warp g % W, so slot s is always consumed by warp s % W,
//    which has consumed fill f - 1 (hence seen it land) before it waits for f.
// Neither side waits on anything but earlier chunks, so the ring cannot
// deadlock.
struct Ring {
    unsigned char* buf;
    uint64_t* full;
    uint64_t* empty;
    int* last_fill;          // per slot: fill number of the last copy issued, or -1
    volatile int* stop;      // set by the consumers when they leave
    int S;
};

// Named barrier of the consumer threads (the producer warp never joins it).
template <int NT>
__device__ __forceinline__ void csync() { asm volatile("bar.sync 1, %0;" ::"n"(Blk<NT>::threads) : "memory"); }

// Grid barrier over the consumers: thread 0 of each block adds 1 to a monotonic
// counter (release) and polls it (acquire) until every block of this round has
// arrived; `target` advances by the block count per barrier.  A wait failure
// anywhere (`*err` of this block, a timeout here) is published in b->err and
// makes every block's barrier return false.  Bounded by kWaitNs.
template <int NT>
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks, unsigned& target, const int* err,
                                          int* s_flag) {
    csync<NT>();
    target += nblocks;
    if (nblocks == 1) {   // a one-block grid: the block barrier above is the whole barrier
        if (threadIdx.x == 0) {
            const int e = *((volatile const int*)err);
            if (e) atomicExch(&b->err, 2);
            *s_flag = e;
        }
        csync<NT>();
        return *s_flag == 0;
    }
    if (threadIdx.x == 0) {
        if (*((volatile const int*)err)) atomicExch(&b->err, 2);
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
        if ((int)(ld_acquire(&b->count) - target) < 0) {
            // poll with a short back-off: 152 blocks polling one word without it
            // slow down the arrivals they wait for
            const unsigned long long t0 = gtimer();
            unsigned polls = 0;
            while ((int)(ld_acquire(&b->count) - target) < 0) {
                __nanosleep(32);
                if ((++polls & 15) == 0 && gtimer() - t0 > kWaitNs) {
                    atomicExch(&b->err, 1);
                    break;
                }
            }
        }
        __threadfence();
        *s_flag = *((volatile int*)&b->err);
    }
    csync<NT>();
    return *s_flag == 0;
}

// Items of a chunked GEMV phase: (row, chunk) pairs, chunk-column-major, with
// the chunks that lie entirely outside a triangle left out so that the work is
// spread evenly.  Chunk column c holds rows [r0(c), r1(c)): all rows
// (TRI_NONE), rows >= c*CH (lower), rows < (c+1)*CH (upper).
template <int TRI>
__device__ __forceinline__ void chunk_rows(int c, int CH, int rows, int& r0, int& r1) {
    r0 = 0;
    r1 = rows;
    if (TRI == TRI_LOWER) r0 = min(rows, c * CH);
    if (TRI == TRI_UPPER) r1 = min(rows, (c + 1) * CH);
}

template <int TRI>
__device__ __forceinline__ int chunk_items(int rows, int cols, int CH) {
    const int nc = (cols + CH - 1) / CH;
    if (TRI == TRI_NONE) return rows * nc;
    int t = 0;
    for (int c = 0; c < nc; ++c) {
        int r0, r1;
        chunk_rows<TRI>(c, CH, rows, r0, r1);
        t += r1 - r0;
    }
    return t;
}

// This block's contiguous item range [b0, b0 + cnt) of a phase.
template <int TRI>
__device__ __forceinline__ void block_range(int rows, int cols, int CH, int& b0, int& cnt) {
    const int nitems = chunk_items<TRI>(rows, cols, CH);
    const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
    b0 = (int)blockIdx.x * per;
    cnt = max(0, min(nitems, b0 + per) - b0);
}

// (row, chunk column) of an item, walked forward from a starting item by
// non-negative steps: one division when it starts, additions after.
template <int TRI>
struct ItemWalk {
    int rows, nc, CH;
    int it = 0, c = 0, base = 0, r0 = 0, r1 = 0, row = 0;
    __device__ __forceinline__ ItemWalk(int rows_, int nc_, int CH_, int first) : rows(rows_), nc(nc_), CH(CH_) {
        if constexpr (TRI == TRI_NONE) {
            it = first;
            c = first / rows;
            row = first - c * rows;
        } else {
            chunk_rows<TRI>(0, CH, rows, r0, r1);
            step(first);
        }
    }
    __device__ __forceinline__ void step(int d) {
        it += d;
        if constexpr (TRI == TRI_NONE) {
            row += d;
            while (row >= rows) {
                row -= rows;
                ++c;
            }
        } else {
            while (it >= base + (r1 - r0) && c < nc - 1) {
                base += r1 - r0;
                ++c;
                chunk_rows<TRI>(c, CH, rows, r0, r1);
            }
            row = r0 + (it - base);
        }
    }
};

// Ring position of an item: its slot and fill number (sequence number fill * S + slot).
struct RingPos {
    int slot = 0, fill = 0;
    __device__ __forceinline__ void advance(int d, int S) {   // any d >= 0
        slot += d;
        if (slot >= S) {
            fill += slot / S;
            slot %= S;
        }
    }
};

// Producer side of one phase: each lane copies the items whose slot it owns
// (slots lane and lane + 32), in increasing order.  The lanes poll together (a
// non-blocking test of their slot's empty barrier per round), so a lane whose
// slot is still in use never holds up a lane whose slot is free.  `pos` is the
// ring position of the phase's first item (advanced past the phase).  Returns
// false (in every lane) once the consumers have stopped or the phase took
// longer than kWaitNs.
template <typename TM, int TRI>
__device__ __forceinline__ bool produce_phase(const TM* __restrict__ M, int rows, int cols, long long ld,
                                              const Ring& R, RingPos& pos) {
    constexpr int CH = Chunk<TM>::n;
    const int lane = threadIdx.x & 31;
    const int nc = (cols + CH - 1) / CH;
    const int S = R.S;
    int b0, cnt;
    block_range<TRI>(rows, cols, CH, b0, cnt);
    // owned slots, and the distance from one slot to another along the ring
    const int o1 = lane < S ? lane : -1, o2 = lane + 32 < S ? lane + 32 : -1;
    auto dist = [&](int from, int to) { return to >= from ? to - from : to + S - from; };
    int i = cnt;
    if (o1 >= 0) i = dist(pos.slot, o1);
    if (o2 >= 0) i = min(i, dist(pos.slot, o2));
    RingPos me = pos;
    me.advance(i < cnt ? i : 0, S);
    ItemWalk<TRI> w(rows, nc, CH, b0 + (i < cnt ? i : 0));
    bool ok = true;
    unsigned polls = 0;
    const unsigned long long t0 = gtimer();
    while (true) {
        const bool has = ok && i < cnt;
        if (!__any_sync(0xffffffffu, has)) break;
        if (has) {
            const int slot = me.slot, fill = me.fill;
            // the slot is free once its previous chunk has been consumed
            if (fill == 0 || mbar_test(&R.empty[slot], (unsigned)((fill - 1) & 1))) {
                const long long e0 = (long long)w.c * CH;
                const unsigned bytes = (unsigned)(min((long long)CH, ld - e0) * (long long)sizeof(TM));
                R.last_fill[slot] = fill;
                mbar_expect_tx(&R.full[slot], bytes);
                bulk_g2s(R.buf + (size_t)slot * kSlotBytes, M + (long long)w.row * ld + e0, bytes, &R.full[slot]);
                // next owned slot: the lane's other slot, else the same slot one lap later
                const int other = (slot == o1) ? o2 : o1;
                const int d = (other >= 0) ? dist(slot, other) : S;
                i += d;
                if (i < cnt) {
                    me.advance(d, S);
                    w.step(d);
                }
            }
        }
        if ((++polls & 63) == 0 && (*R.stop || gtimer() - t0 > kWaitNs)) ok = false;
    }
    pos.advance(cnt, S);
    return __all_sync(0xffffffffu, ok);
}

// Consumer side of one phase: part[c * pld + row] = chunk c of row `row` of M . xs
// (chunk-major, so that the next phase's per-row sums load coalesced).  Warp w
// takes the items whose slot is w modulo the consumer warp count (S is a
// multiple of it).
template <typename TM, int TRI, int NT>
__device__ __forceinline__ void gemv_ring(const Ring& R, RingPos& pos, int rows, int cols, long long ld,
                                          const TM* __restrict__ xs, TM* __restrict__ part, int pld,
                                          int* err) {
    using VT = Vec16<TM>;
    using V = typename VT::type;
    constexpr int CH = Chunk<TM>::n;
    constexpr int VN = VT::n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nc = (cols + CH - 1) / CH;
    const int S = R.S;
    int b0, cnt;
    block_range<TRI>(rows, cols, CH, b0, cnt);
    const V* xv = reinterpret_cast<const V*>(xs);
    constexpr int W = Blk<NT>::warps;
    const int first = (warp - pos.slot % W + W) % W;
    if (first < cnt) {
        RingPos me = pos;
        me.advance(first, S);
        ItemWalk<TRI> w(rows, nc, CH, b0 + first);
        for (int i = first; i < cnt; i += W) {
            const int vbase = w.c * (CH / VN);
            const int slot = me.slot;
            if (!mbar_wait(&R.full[slot], (unsigned)(me.fill & 1))) *err = 1;
            const V* sv = reinterpret_cast<const V*>(R.buf + (size_t)slot * kSlotBytes);
            const int vend = (int)(ld / VN) - vbase;   // vectors of this row from the chunk start
            TM acc = TM(0);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = lane + 32 * k;
                const V m = (v < vend) ? sv[v] : V{};
                acc = VT::dot(m, xv[vbase + v], acc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&R.empty[slot]);
            acc = warp_sum(acc);
            if (lane == 0) part[(long long)w.c * pld + w.row] = acc;
            if (i + W < cnt) {
                me.advance(W, S);
                w.step(W);
            }
        }
    }
    pos.advance(cnt, S);
}

// Chunk sums of four rows j[0..3] at once (rows >= len give 0): for each row the
// chunks are added in increasing order, the loads of all four rows and four
// consecutive chunks issued together.
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
// f(j, sum) turns a row's chunk sum into the staged value.
template <int NT, typename TX, typename TM, int TRI, class F>
__device__ __forceinline__ void stage_sum(TX* xs, const TM* part, int pld, int cols, int len, int pad, F f) {
    using AT = typename Acc<TM>::type;
    constexpr int T = Blk<NT>::threads;
    for (int j0 = threadIdx.x; j0 < pad; j0 += 4 * T) {
        int j[4];
        AT sm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) j[u] = j0 + u * T;
        sum_chunks4<TM, TRI, AT>(part, pld, cols, j, len, sm);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j[u] < pad) xs[j[u]] = (j[u] < len) ? f(j[u], sm[u]) : TX(0);
    }
}

// stage_sum with an operand loaded before the partials: pre(j) is issued for the
// four rows together with their partial loads, and f(j, sum, pre(j)) makes the
// staged value, so a loop-invariant vector costs no extra round trip.
template <int NT, typename TX, typename TM, int TRI, class P, class F>
__device__ __forceinline__ void stage_sum_pre(TX* xs, const TM* part, int pld, int cols, int len, int pad, P pre,
                                              F f) {
    using AT = typename Acc<TM>::type;
    constexpr int T = Blk<NT>::threads;
    for (int j0 = threadIdx.x; j0 < pad; j0 += 4 * T) {
        int j[4];
        AT sm[4];
        decltype(pre(0)) pv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = j0 + u * T;
            pv[u] = (j[u] < len) ? pre(j[u]) : decltype(pre(0))(0);
        }
        sum_chunks4<TM, TRI, AT>(part, pld, cols, j, len, sm);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (j[u] < pad) xs[j[u]] = (j[u] < len) ? f(j[u], sm[u], pv[u]) : TX(0);
    }
}

// Consumer-wide fixed-order sum, result broadcast to every consumer thread.
template <int NT, typename AT>
__device__ __forceinline__ AT block_allsum(AT v, AT* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    csync<NT>();
    if (threadIdx.x < 32) {
        AT r = (l < Blk<NT>::warps) ? sh[l] : AT(0);
        r = warp_sum(r);
        if (l == 0) sh[32] = r;
    }
    csync<NT>();
    v = sh[32];
    csync<NT>();
    return v;
}

template <typename TO, typename TP>
struct FusedArgs {
    int n, m1, m2;
    // operator (precision TO)
    const TO *CWT, *WH, *Et, *EtT, *WHT, *CW;
    long long ldCWT, ldWH, ldEt, ldEtT, ldWHT, ldCW;
    // pcg_form 1: B = L^{-1}[C'; 0] ((n+m1) x m2) and B', partials of B p
    int wform;
    const TO *BW, *BWT;
    long long ldBW, ldBWT;
    TO* PW;
    int ldPW;
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
    GridBar* bar;      // zeroed before the launch
    size_t xs_bytes;   // bytes of the staged-vector region of shared memory (16-byte multiple)
    size_t ring_off;   // byte offset of the slot ring (128-byte aligned)
    int slots;         // ring depth S
    unsigned long long* tstamp;   // optional: %globaltimer at phase marks of the first 4 iterations
    int leave_early;              // failure-detection test: block 0 leaves before its first grid barrier
};

// Shared-memory layout of the persistent kernel: staged vector, three m2-vector
// caches, then the ring (slots, full and empty mbarriers, last-fill words, stop flag).
template <typename TO>
inline size_t fused_ring_offset(size_t xs_bytes, int m2) {
    const size_t o = xs_bytes + 3 * (size_t)m2 * sizeof(TO);
    return (o + 127) / 128 * 128;
}
inline size_t fused_smem_bytes(size_t ring_off, int slots) {
    return ring_off + (size_t)slots * (kSlotBytes + 2 * sizeof(uint64_t) + sizeof(int)) + 16;
}

// The producer's sequence of phases, the consumers' loop below in the same order.
template <typename TO, typename TP, int PC>
__device__ void pcg_producer(const FusedArgs<TO, TP>& a, const Ring& R) {
    const int n = a.n, m1 = a.m1, m2 = a.m2;
    RingPos g;
    while (!*R.stop) {   // (a block may own no chunk of any phase: it polls the stop flag here)
        if (a.wform) {
            if (!produce_phase<TO, TRI_NONE>(a.BW, n + m1, m2, a.ldBW, R, g)) break;
            if (!produce_phase<TO, TRI_NONE>(a.BWT, m2, n + m1, a.ldBWT, R, g)) break;
        } else {
            if (!produce_phase<TO, TRI_NONE>(a.CWT, n, m2, a.ldCWT, R, g)) break;
            if (!produce_phase<TO, TRI_LOWER>(a.WH, n, n, a.ldWH, R, g)) break;
            if (m1 > 0 && !produce_phase<TO, TRI_NONE>(a.Et, m1, n, a.ldEt, R, g)) break;
            if (!produce_phase<TO, TRI_UPPER>(a.WHT, n, n, a.ldWHT, R, g)) break;
            if (m1 > 0 && !produce_phase<TO, TRI_NONE>(a.EtT, n, m1, a.ldEtT, R, g)) break;
            if (!produce_phase<TO, TRI_NONE>(a.CW, m2, n, a.ldCW, R, g)) break;
        }
        if (PC == PC_H_K) {
            if (!produce_phase<TP, TRI_LOWER>(a.WPl, m2, m2, a.ldWP, R, g)) break;
            if (!produce_phase<TP, TRI_UPPER>(a.WPu, m2, m2, a.ldWP, R, g)) break;
        }
    }
    // drain: every copy issued lands before the block's shared memory goes away
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (int sl = lane; sl < R.S; sl += 32) {
        const int f = R.last_fill[sl];
        if (f >= 0) mbar_wait(&R.full[sl], (unsigned)(f & 1));
    }
}

// kind: PC_L_K (z = r / D), PC_H_K (z = Sg W' W Sg r), PC_NONE_K (z = r).
// Entry state (from pcg_init): x = 0, r = r0 = rhs, p = p0 = z0, st->rz_cur = r'z,
// st->tol2 = tol^2 |rhs|^2, st->maxit.  Shared memory: the staged vector
// (xs_bytes), three m2-vectors in TO (q = K_F p, r and p of the current
// iteration), then the ring.
template <typename TO, typename TP, int PC, int NT>
__global__ void __launch_bounds__(NT, NT == kSmallBlock ? 2 : 1) pcg_fused_kernel(const FusedArgs<TO, TP> a) {
    constexpr int kFusedThreads = Blk<NT>::threads;
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(128) unsigned char pcg_smem[];
    TO* xs = reinterpret_cast<TO*>(pcg_smem);
    TP* xp = reinterpret_cast<TP*>(pcg_smem);
    TO* qc = reinterpret_cast<TO*>(pcg_smem + a.xs_bytes);
    TO* rc = qc + a.m2;
    TO* pcs = rc + a.m2;
    Ring R;
    R.S = a.slots;
    R.buf = pcg_smem + a.ring_off;
    R.full = reinterpret_cast<uint64_t*>(R.buf + (size_t)R.S * kSlotBytes);
    R.empty = R.full + R.S;
    R.last_fill = reinterpret_cast<int*>(R.empty + R.S);
    R.stop = reinterpret_cast<volatile int*>(R.last_fill + R.S);
    using AT = typename Acc<TO>::type;
    __shared__ AT sh[40];
    __shared__ int s_flag;
    __shared__ int s_err;
    const int n = a.n, m1 = a.m1, m2 = a.m2;
    const int tid = threadIdx.x;
    const unsigned nblocks = gridDim.x;

    if (__ldcg(&a.st->done)) return;
    if (tid == 0) {
        for (int sl = 0; sl < R.S; ++sl) {
            mbar_init(&R.full[sl], 1);
            mbar_init(&R.empty[sl], 1);
            R.last_fill[sl] = -1;
        }
        *R.stop = 0;
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid >= kFusedThreads) {
        pcg_producer<TO, TP, PC>(a, R);
        return;
    }

    // ------------------------------------------------------------ consumers
    // slice of the m2-vectors this block owns for writes
    const int per = (m2 + nblocks - 1) / nblocks;
    const int own0 = blockIdx.x * per, own1 = min(m2, own0 + per);
    constexpr int CHO = Chunk<TO>::n, CHP = Chunk<TP>::n;
    const int padO_n = ((n + CHO - 1) / CHO) * CHO, padO_m2 = ((m2 + CHO - 1) / CHO) * CHO;
    const int padO_m1 = ((m1 + CHO - 1) / CHO) * CHO, padP_m2 = ((m2 + CHP - 1) / CHP) * CHP;
    TO* xs2 = xs + padO_n;   // z2, beside z1, for the back solve
    const int padO_nm1 = ((n + m1 + CHO - 1) / CHO) * CHO;
    const int qcols = a.wform ? n + m1 : n;   // columns of the matrix whose partials make C y
    const bool stamp = a.tstamp != nullptr && blockIdx.x == 0 && tid == 0;
    auto mark = [&](int it, int ph) {
        if (stamp && it < 4) a.tstamp[it * 32 + ph] = gtimer();
    };
    unsigned target = 0;
    RingPos g;   // ring position of the next chunk
    // every consumer exit passes here: the producer stops issuing and drains
    auto leave = [&]() {
        csync<NT>();
        if (tid == 0) {
            if (s_err) atomicExch(&a.bar->err, 2);
            *R.stop = 1;
        }
    };
    auto gsync = [&]() { return grid_sync<NT>(a.bar, nblocks, target, &s_err, &s_flag); };

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
    csync<NT>();
    for (int j = tid; j < padO_m2; j += kFusedThreads) xs[j] = (j < m2) ? pcs[j] : TO(0);
    csync<NT>();

    // failure-detection test: block 0 stops before the first grid barrier, as a block
    // that died would; every other block's bounded wait runs out and reports QP_ETIMEOUT
    if (a.leave_early && blockIdx.x == 0 && nblocks > 1) { leave(); return; }

    while (true) {
        mark(it, 0);
        if (a.wform) {
            // ---- W1 (a6-a7): w = B p, B = L^{-1}[C'; 0] (rows R^{-T} C', then Et C')
            gemv_ring<TO, TRI_NONE, NT>(R, g, n + m1, m2, a.ldBW, xs, a.PW, a.ldPW, &s_err);
            mark(it, 11);
            if (!gsync()) { leave(); return; }
            mark(it, 1);
            // ---- W2 (a7-a8): C y = B' J w with J = diag(I_n, -I_m1)
            stage_sum<NT, TO, TO, TRI_NONE>(xs, a.PW, a.ldPW, m2, n + m1, padO_nm1,
                                            [&](int j, AT v) { return (TO)(j < n ? v : -v); });
            csync<NT>();
            mark(it, 16);
            gemv_ring<TO, TRI_NONE, NT>(R, g, m2, n + m1, a.ldBWT, xs, a.PQ, a.ldQ, &s_err);
            mark(it, 17);
            if (!gsync()) { leave(); return; }
            mark(it, 6);
        } else {
            // ---- P1 (a6): u = C' p
            gemv_ring<TO, TRI_NONE, NT>(R, g, n, m2, a.ldCWT, xs, a.PU, a.ldU, &s_err);
            mark(it, 11);
            if (!gsync()) { leave(); return; }
            mark(it, 1);
            // ---- P2 (a7, forward solve with L): z1 = R^{-T} u, Et u (z2 = -Et u)
            stage_sum<NT, TO, TO, TRI_NONE>(xs, a.PU, a.ldU, m2, n, padO_n, [&](int, AT v) { return (TO)v; });
            csync<NT>();
            mark(it, 12);
            gemv_ring<TO, TRI_LOWER, NT>(R, g, n, n, a.ldWH, xs, a.PZ1, a.ldZ1, &s_err);
            if (m1 > 0) gemv_ring<TO, TRI_NONE, NT>(R, g, m1, n, a.ldEt, xs, a.PZ2, a.ldZ2, &s_err);
            mark(it, 13);
            if (!gsync()) { leave(); return; }
            mark(it, 2);
            // ---- P3 (a7, back solve with L'): y = R^{-1} z1 + Et' z2
            stage_sum<NT, TO, TO, TRI_LOWER>(xs, a.PZ1, a.ldZ1, n, n, padO_n, [&](int, AT v) { return (TO)v; });
            if (m1 > 0)
                stage_sum<NT, TO, TO, TRI_NONE>(xs2, a.PZ2, a.ldZ2, n, m1, padO_m1, [&](int, AT v) { return (TO)(-v); });
            csync<NT>();
            mark(it, 14);
            gemv_ring<TO, TRI_UPPER, NT>(R, g, n, n, a.ldWHT, xs, a.PY, a.ldY, &s_err);
            if (m1 > 0) gemv_ring<TO, TRI_NONE, NT>(R, g, n, m1, a.ldEtT, xs2, a.PT, a.ldT, &s_err);
            mark(it, 15);
            if (!gsync()) { leave(); return; }
            mark(it, 5);
            // ---- P4 (a8): q = D p + C y
            if (m1 > 0) {
                stage_sum<NT, TO, TO, TRI_NONE>(xs, a.PT, a.ldT, m1, n, padO_n, [&](int, AT v) { return (TO)v; });
                csync<NT>();
                stage_sum<NT, TO, TO, TRI_UPPER>(xs, a.PY, a.ldY, n, n, padO_n,
                                             [&](int j, AT v) { return (TO)(v + (AT)xs[j]); });
            } else {
                stage_sum<NT, TO, TO, TRI_UPPER>(xs, a.PY, a.ldY, n, n, padO_n, [&](int, AT v) { return (TO)v; });
            }
            csync<NT>();
            mark(it, 16);
            gemv_ring<TO, TRI_NONE, NT>(R, g, m2, n, a.ldCW, xs, a.PQ, a.ldQ, &s_err);
            mark(it, 17);
            if (!gsync()) { leave(); return; }
            mark(it, 6);
        }

        // ---- P5 (a10): q = D p + C y (cached), alpha = r'z / p'q, x += alpha p, r -= alpha q
        // (p'q is summed while q is staged: each thread takes its rows in increasing order)
        AT pq = AT(0);
        stage_sum_pre<NT, TO, TO, TRI_NONE>(qc, a.PQ, a.ldQ, qcols, m2, m2, [&](int j) { return __ldg(a.D + j); },
                                        [&](int j, AT v, TO dj) {
                                            const TO q = (TO)fma((AT)dj, (AT)pcs[j], v);
                                            pq = fma((AT)pcs[j], (AT)q, pq);
                                            return q;
                                        });
        pq = block_allsum<NT>(pq, sh);
        // breakdown (p'q <= 0 or not finite): stop with the last iterate untouched
        if (!(pq > AT(0)) || !isfinite(pq)) { done = 3; break; }
        const AT alpha = rz / pq;
        const TO al = (TO)alpha;
        AT rrp = AT(0), rzp = AT(0);
#pragma unroll 4
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
        rr = block_allsum<NT>(rrp, sh);
        ++it;
        const bool finite = isfinite(rr) && isfinite(pq);
        if (!finite) { done = 3; break; }
        if ((double)rr <= tol2) { done = 1; break; }
        if (it >= maxit) { done = 2; break; }
        mark(it - 1, 7);

        AT rz_new;
        if (PC == PC_H_K) {
            csync<NT>();
            // ---- P6 (a9): v = W rs, z = Sg W' v
            gemv_ring<TP, TRI_LOWER, NT>(R, g, m2, m2, a.ldWP, xp, a.PV, a.ldV, &s_err);
            mark(it - 1, 18);
            if (!gsync()) { leave(); return; }
            mark(it - 1, 8);
            stage_sum<NT, TP, TP, TRI_LOWER>(xp, a.PV, a.ldV, m2, m2, padP_m2, [&](int, typename Acc<TP>::type v) { return (TP)v; });
            csync<NT>();
            mark(it - 1, 19);
            gemv_ring<TP, TRI_UPPER, NT>(R, g, m2, m2, a.ldWP, xp, a.PZ, a.ldZ, &s_err);
            mark(it - 1, 20);
            if (!gsync()) { leave(); return; }
            mark(it - 1, 9);
            // z into the q cache (q is no longer needed), then r'z
            // (r'z is summed while z is staged, rows in increasing order per thread)
            rzp = AT(0);
            stage_sum_pre<NT, TO, TP, TRI_UPPER>(qc, a.PZ, a.ldZ, m2, m2, m2, [&](int j) { return __ldg(a.sg + j); },
                                             [&](int j, typename Acc<TP>::type v, TP sj) {
                                                 const TO z = (TO)((AT)sj * (AT)v);
                                                 rzp = fma((AT)rc[j], (AT)z, rzp);
                                                 return z;
                                             });
            rz_new = block_allsum<NT>(rzp, sh);
        } else {
            rz_new = block_allsum<NT>(rzp, sh);
        }
        // ---- beta, p = z + beta p (staged as the next P1 input; shared-memory only)
        const AT beta = rz_new / rz;
        rz = rz_new;
        const TO be = (TO)beta;
#pragma unroll 4
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
        csync<NT>();
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
    leave();
}

}  // namespace pcgipm
