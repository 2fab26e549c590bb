// pcg_fused.cuh -- the PCG hot loop (a6-a10) as one persistent cooperative kernel.
//
// One launch runs every iteration of one PCG solve on K_F dnu = r_nu.  An
// iteration is a short chain of row-major matrix-vector phases separated by
// grid barriers.  With the default form (pcg_form 0):
//   u = C' p;  y = M0 u with M0 = [K0^{-1}]_11 = R^{-1} R^{-T} - Et' Et, the
//   (1,1) block of the inverse of the K0 factorization (the forward and the
//   back solve of Sec. 5.2's second step in one product, formed once per QP);
//   q = D p + C y;  and for P_H, v = P~^{-1} (Sg r) with P~^{-1} = W' W the
//   inverse of the Jacobi-scaled P_H from its Cholesky factor W^{-1}.
// pcg_form 2 keeps the two triangular solves with the stored inverse factor
// ([R^{-T}; Et] u, then [R^{-1} | Et'] [z1; -z2]); pcg_form 1 applies
// K_F through B = L^{-1}[C'; 0] (two phases).
//
// Layout of the work.  A matrix is cut into chunks of one row of at most one
// ring slot (16 KB for a QP spread over the GPU, 4 KB for a small one); chunks
// that lie entirely outside a stored triangle are left out.  (Bulk copies of
// 4 KB stream at about half the HBM rate of 16 KB ones: the copy engine's rate
// per copy, not the ring depth, bounds them.)  Each block owns a contiguous range of whole rows of
// every phase (balanced by chunk count on the host), so a row's result is
// summed by one block in a fixed order and written once: the next phase stages
// its input with one load per element.  The matrices do not change during the
// solve, so their stream does not wait for the barriers: a producer warp
// copies the block's chunks, phase after phase and iteration after iteration,
// into a ring of shared-memory slots with bulk asynchronous copies
// (cp.async.bulk, completion counted on one mbarrier per slot), running ahead
// of the consumers by up to the ring's depth -- across the grid barriers, where
// a kernel that only loaded after the barrier would leave HBM idle.  Consumer
// warps dot the chunks with the staged vector and keep one partial per chunk
// in shared memory; after the phase each owned row is summed in chunk order.
// The PCG scalars (p'q, |r|^2, r'z) are summed by every block over the whole
// vectors in the same fixed order, so every block holds bit-identical scalars
// without a reduction barrier, and the vector updates are done redundantly in
// shared memory (each block writes only its own slice of x).
//
// Every wait is bounded in time (kWaitNs on %globaltimer): a consumer that gives
// up sets the error bit of the barrier word and every block returns at its next
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
};
constexpr int kBigSlotBytes = 16384;              // ring slot of a QP spread over the GPU
constexpr int kSmallSlotBytes = 4096;             // ring slot of a small QP (its rows are short)
static_assert((kBigSlotBytes & (kBigSlotBytes - 1)) == 0 && (kSmallSlotBytes & (kSmallSlotBytes - 1)) == 0,
              "slot sizes are powers of two (chdiv)");
constexpr int kMaxSlots = 64;                     // two slots per producer lane at most
constexpr int kSmallRingSlots = 14;               // ring of a QP whose grid covers a small part of the GPU
constexpr int kMaxClusterBlocks = 16;             // grids up to this size launch as one cluster
constexpr int kMaxPhases = 6;                     // operator phases (pcg_form 2: four) + P_H (one or two)
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any wait
constexpr unsigned kBarErr = 0x40000000u;         // error bit of the barrier counter
constexpr int kNU = 16;                           // m2-vector elements per thread held in registers
constexpr int kSeg = 64;                          // sliced FP64 update: elements per partial sum

// Grid barrier word: a monotonic arrival counter (zeroed before each launch)
// whose bit 30 records a failure anywhere, so one acquire load tells a polling
// block both that the round is complete and whether to leave.
struct GridBar {
    unsigned count;
    unsigned pad[31];
};

// Accumulation type of the chunk dots and PCG scalars inside the fused kernel:
// the working precision itself.  (GB300's FP64 pipe issues two FMAs per clock per
// SM, so an FP32 path must not touch FP64 arithmetic in its inner loops.)
template <typename T> struct Acc { using type = T; };

// One matrix of a phase: it contributes to phase rows [r0, r1), its columns are
// dotted with the staged vector from offset xoff.  Dense (row-major, streamed
// through the ring; chunks outside its stored triangle, relative to its own rows
// i = r - r0, are skipped) or CSR (rp, ci and the values M; no ring items: the
// owning block's thread of a row sums its nonzeros after the dense chunks).
struct Part {
    const void* M;
    long long ld;     // row stride in elements (a multiple of 32: rows start 128-byte aligned)
    int r0, r1;
    int cols;
    int tri;          // TRI_NONE, TRI_LOWER (row i: chunks up to i's), TRI_UPPER (from i's)
    int xoff;
    const int* rp;    // CSR row pointers (rows r1 - r0 + 1) and column indices, or null (dense)
    const int* ci;
};

// A phase: up to two parts (stacked rows, or side by side on the same rows),
// and how its input is staged from the previous phase's output:
// xs[j] = out[j] (j < in_len1), xs[in_off2 + j] = in_s2 * out[in_len1 + j] (j < in_len2),
// zeros elsewhere up to in_pad.
struct Phase {
    Part p[2];
    int np;
    int rows;
    int ncmax;        // most chunks of one row (stride of the per-row partials)
    int tbl;          // offset of this phase's (first row, first item) table: grid + 1 entries
    int in_len1, in_off2, in_len2, in_pad;
    float in_s2;
    int flat;         // 1: one dense untriangular matrix on rows [0, rows): a block's rows are one
                      // contiguous range of memory, cut into full-slot chunks that may cross rows
};

// Rows of a flat phase: row r spans elements [r ld, (r + 1) ld) of the matrix,
// chunk c spans [c CH, (c + 1) CH) (global offsets, so that the segments of a row
// -- and every sum -- are the same for any grid); a block copies the chunks that
// meet its rows, clipped to them.
// x / CH for x >= 0: CH, the elements of one ring slot (4 or 16 KB of 4- or 8-byte
// elements), is a power of two, so the quotient is a shift.
__host__ __device__ __forceinline__ long long chdiv(long long x, int CH) {
#ifdef __CUDA_ARCH__
    return x >> (__ffs(CH) - 1);
#else
    return x >> __builtin_ctz((unsigned)CH);
#endif
}
__host__ __device__ inline int flat_first_chunk(long long r, long long ld, int CH) { return (int)chdiv(r * ld, CH); }
__host__ __device__ inline int flat_row_chunks(long long r, long long ld, int CH) {
    return (int)chdiv((r + 1) * ld - 1, CH) - (int)chdiv(r * ld, CH) + 1;
}
// chunks meeting rows [rb0, rb1)
__host__ __device__ inline int flat_items(long long rb0, long long rb1, long long ld, int CH) {
    if (rb1 <= rb0) return 0;
    return (int)chdiv(rb1 * ld + CH - 1, CH) - (int)chdiv(rb0 * ld, CH);
}

__host__ __device__ inline void part_chunks(const Part& P, int CH, int r, int& c0, int& c1) {
    c0 = c1 = 0;
    if (r < P.r0 || r >= P.r1 || P.rp) return;
    const int nc = (int)chdiv(P.cols + CH - 1, CH);
    const int i = r - P.r0;
    const int ic = (int)chdiv(i, CH);
    c1 = nc;
    if (P.tri == TRI_LOWER) c1 = (ic + 1 < nc) ? ic + 1 : nc;
    if (P.tri == TRI_UPPER) c0 = (ic < nc) ? ic : nc;
}

__host__ __device__ inline int row_items(const Phase& ph, int CH, int r) {
    int t = 0;
    for (int q = 0; q < ph.np; ++q) {
        int c0, c1;
        part_chunks(ph.p[q], CH, r, c0, c1);
        t += c1 - c0;
    }
    return t;
}

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

// Ring of chunk slots in shared memory.  The block's chunks are numbered in one
// sequence over phases and iterations; chunk g goes to slot g % S, its fill
// number is g / S.  full[s] completes one phase per copy (producer arrival +
// transaction bytes), empty[s] one phase per consumption (one arrival of the
// consuming warp).  A parity wait names the phase it waits for exactly only
// while the waiter is at most one phase ahead, so every slot has one owner on
// each side and each owner handles its slot's fills in order:
//  - producer lane s % 32 issues every fill of slot s; before fill f it waits
//    for the consumption of fill f - 1, and it had waited for that of f - 2
//    before issuing f - 1;
//  - consumer warp s % W consumes every fill of slot s (W consumer warps), in
//    order, so it has consumed fill f - 1 (hence seen it land) before it waits
//    for fill f.
// Neither side waits on anything but earlier chunks, so the ring cannot
// deadlock.
struct Ring {
    unsigned char* buf;
    int slot_bytes;
    uint64_t* full;
    uint64_t* empty;
    int* last_fill;          // per slot: fill number of the last copy issued, or -1
    volatile int* stop;      // set by the consumers when they leave
    int S;
    // diagnostics (block 0, PCGIPM_PHASE_TIMES): %globaltimer at issue, landing and
    // release of the chunks with ring sequence numbers [trace0, trace0 + kTrace)
    unsigned long long* trace;
    int trace0;
};
constexpr int kTrace = 512;
__device__ __forceinline__ void trace_mark(const Ring& R, int which, int fill, int slot) {
    if (R.trace) {
        const int q = fill * R.S + slot - R.trace0;
        if (q >= 0 && q < kTrace) R.trace[which * kTrace + q] = gtimer();
    }
}

// Named barrier of the consumer threads (the producer warp never joins it).
template <int NT>
__device__ __forceinline__ void csync() { asm volatile("bar.sync 1, %0;" ::"n"(Blk<NT>::threads) : "memory"); }

// Grid barrier over the consumers: thread 0 of each block adds 1 to the
// monotonic counter (release; the block barrier before it orders the block's
// writes) and spins on it (acquire) until every block of this round has
// arrived; `target` advances by the block count per barrier.  A failure of
// this block (*err) or a timeout here sets the error bit, which ends every
// block's wait and makes every block's barrier return false.  Bounded by kWaitNs.
template <int NT>
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned nblocks, unsigned& target, const int* err,
                                          int* s_flag) {
    csync<NT>();
    target += nblocks;
    if (nblocks == 1) {   // a one-block grid: the block barrier above is the whole barrier
        if (threadIdx.x == 0) {
            const int e = *((volatile const int*)err);
            if (e) atomicOr(&b->count, kBarErr);
            *s_flag = e;
        }
        csync<NT>();
        return *s_flag == 0;
    }
    if (threadIdx.x == 0) {
        if (*((volatile const int*)err)) atomicOr(&b->count, kBarErr);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&b->count) : "memory");
        unsigned v = ld_acquire(&b->count);
        if (!(v & kBarErr) && (int)((v & ~kBarErr) - target) < 0) {
            const unsigned long long t0 = gtimer();
            unsigned polls = 0;
            while (true) {
                v = ld_acquire(&b->count);
                if ((v & kBarErr) || (int)((v & ~kBarErr) - target) >= 0) break;
                if ((++polls & 1023) == 0 && gtimer() - t0 > kWaitNs) {
                    atomicOr(&b->count, kBarErr);
                    v = kBarErr;
                    break;
                }
            }
        }
        *s_flag = (v & kBarErr) ? 1 : 0;
    }
    csync<NT>();
    return *s_flag == 0;
}

// Position in a block's item sequence of one phase: (row, part, chunk) and the
// chunk's index k within its row; steps forward over rows in O(rows skipped).
// CH: elements of one chunk.
struct Walk {
    int CH;
    int row, p, c, c1, k;
    __host__ __device__ __forceinline__ void first_of_row(const Phase& ph, int r) {
        row = r;
        k = 0;
        p = -1;
        next_part(ph);
    }
    // the next (row, part) with chunks, from part p + 1 of `row` on
    __host__ __device__ __forceinline__ void next_part(const Phase& ph) {
        while (true) {
            if (++p >= ph.np) {
                if (++row >= ph.rows) { c = c1 = 0; return; }
                p = -1;
                k = 0;
                continue;
            }
            int c0;
            part_chunks(ph.p[p], CH, row, c0, c1);
            if (c0 < c1) { c = c0; return; }
        }
    }
    __host__ __device__ __forceinline__ void step(const Phase& ph, int d) {
        while (d > 0) {
            const int rem = c1 - c - 1;   // items after the current one in this (row, part)
            if (d <= rem) { c += d; k += d; return; }
            d -= rem + 1;
            k += rem + 1;
            next_part(ph);
        }
    }
};

// Ring position of an item: its slot and fill number (sequence number fill * S + slot).
struct RingPos {
    int slot = 0, fill = 0;
    __device__ __forceinline__ void advance(int d, int S) {   // any d >= 0
        slot += d;
        if (slot >= S) {
            if (slot < 2 * S) {
                slot -= S;
                ++fill;
            } else {
                fill += slot / S;
                slot %= S;
            }
        }
    }
};

// Distance along the ring from slot `from` to slot `to` (0..S-1).
__device__ __forceinline__ int ring_dist(int from, int to, int S) { return to >= from ? to - from : to + S - from; }

// This block's rows [rb0, rb1) and item count of a phase (host-balanced table).
struct BlockRange {
    int rb0, rb1, cnt;
};
__device__ __forceinline__ BlockRange block_range(const int2* __restrict__ tbl, const Phase& ph) {
    const int2 a = tbl[ph.tbl + blockIdx.x], b = tbl[ph.tbl + blockIdx.x + 1];
    return BlockRange{a.x, b.x, b.y - a.y};
}

// Producer side of one phase: each lane copies the items whose slots it owns
// (slots lane and lane + 32), in increasing order.  The lanes poll together (a
// non-blocking test of their slot's empty barrier per round), so a lane whose
// slot is still in use never holds up a lane whose slot is free.  `pos` is the
// ring position of the phase's first item (advanced past the phase).  Returns
// false (in every lane) once the consumers have stopped or the phase took
// longer than kWaitNs.
template <typename TM>
__device__ __forceinline__ bool produce_phase(const Phase& ph, const BlockRange br, const Ring& R, RingPos& pos) {
    const int CH = R.slot_bytes / (int)sizeof(TM);
    const int lane = threadIdx.x & 31;
    const int S = R.S;
    const int cnt = br.cnt;
    const int o1 = lane < S ? lane : -1, o2 = lane + 32 < S ? lane + 32 : -1;
    int i = cnt;
    if (o1 >= 0) i = ring_dist(pos.slot, o1, S);
    if (o2 >= 0) i = min(i, ring_dist(pos.slot, o2, S));
    RingPos me = pos;
    Walk w;
    w.CH = CH;
    const bool flat = ph.flat != 0;
    const Part& P0 = ph.p[0];
    const TM* fbase = static_cast<const TM*>(P0.M);                   // flat: global element offsets
    const long long fbeg = (long long)br.rb0 * P0.ld, fend = (long long)br.rb1 * P0.ld;
    const long long fc0 = chdiv(fbeg, CH);                                    // first chunk meeting the rows
    if (i < cnt) {
        me.advance(i, S);
        if (!flat) {
            w.first_of_row(ph, br.rb0);
            w.step(ph, i);
        }
    }
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
                const TM* src;
                unsigned bytes;
                if (flat) {
                    const long long e0 = max(fbeg, (fc0 + i) * CH), e1 = min(fend, (fc0 + i + 1) * CH);
                    src = fbase + e0;
                    bytes = (unsigned)((e1 - e0) * (long long)sizeof(TM));
                } else {
                    const Part& P = ph.p[w.p];
                    const long long e0 = (long long)w.c * CH;
                    bytes = (unsigned)(min((long long)CH, P.ld - e0) * (long long)sizeof(TM));
                    src = static_cast<const TM*>(P.M) + (long long)(w.row - P.r0) * P.ld + e0;
                }
                R.last_fill[slot] = fill;
                trace_mark(R, 0, fill, slot);
                mbar_expect_tx(&R.full[slot], bytes);
                bulk_g2s(R.buf + (size_t)slot * R.slot_bytes, src, bytes, &R.full[slot]);
                // next owned slot: the lane's other slot, else the same slot one lap later
                const int other = (slot == o1) ? o2 : o1;
                const int d = (other >= 0) ? ring_dist(slot, other, S) : S;
                i += d;
                if (i < cnt) {
                    me.advance(d, S);
                    if (!flat) w.step(ph, d);
                }
            }
        }
        if ((++polls & 63) == 0 && (*R.stop || gtimer() - t0 > kWaitNs)) ok = false;
    }
    pos.advance(cnt, S);
    return __all_sync(0xffffffffu, ok);
}

// Consumer side of one phase: spart[lrow * ncmax + k] = chunk k of local row
// lrow dotted with the staged vector xs.  Warp w takes the items of the slots
// w, w + W, w + 2W, ... (below S).
template <typename TM, int NT>
__device__ __forceinline__ void consume_phase(const Phase& ph, const BlockRange br, const Ring& R, RingPos& pos,
                                              const TM* __restrict__ xs, TM* __restrict__ spart, int* err) {
    using VT = Vec16<TM>;
    using V = typename VT::type;
    constexpr int VN = VT::n;
    constexpr int W = Blk<NT>::warps;
    const int CH = R.slot_bytes / (int)sizeof(TM);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int S = R.S;
    const int cnt = br.cnt;
    // owned slots: warp, warp + W, ... (below S); the one after slot s is s + W, or
    // `warp` on the next lap.  The first owned item is the nearest owned slot.
    int i = cnt;
    for (int s = warp; s < S; s += W) i = min(i, ring_dist(pos.slot, s, S));
    if (i < cnt && ph.flat) {
        // flat chunks: split each chunk at the row boundaries it crosses
        const long long ld = ph.p[0].ld;
        const long long fbeg = (long long)br.rb0 * ld, fend = (long long)br.rb1 * ld;
        const long long fc0 = chdiv(fbeg, CH);
        RingPos me = pos;
        me.advance(i, S);
        while (true) {
            const int slot = me.slot;
            if (!mbar_wait(&R.full[slot], (unsigned)(me.fill & 1))) *err = 1;
            if (lane == 0) trace_mark(R, 1, me.fill, slot);
            const V* sv = reinterpret_cast<const V*>(R.buf + (size_t)slot * R.slot_bytes);
            const long long c = fc0 + i;                         // global chunk
            const long long e0 = max(fbeg, c * CH), e1 = min(fend, (c + 1) * CH);
            // global row (a 32-bit quotient where the offsets allow: 64-bit division is slow)
            long long rl = (e0 <= 0x7fffffffLL) ? (long long)((unsigned)e0 / (unsigned)ld) : e0 / ld;
            const V* xv = reinterpret_cast<const V*>(xs);
            // Row segments four at a time: their dots are independent, and one round of
            // shuffles reduces all four (a chunk of a short-row matrix holds many rows).
            // A row that starts inside chunk c has c as its first chunk (k = 0); only the
            // chunk's first segment may continue a row begun in an earlier chunk.
            for (long long e = e0; e < e1;) {
                TM acc[4];
                long long rg = rl;
                int nr = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[t] = TM(0);
                    if (e < e1) {                                // (the same in every lane)
                        const long long se = min(e1, (rl + 1) * ld);
                        const int v0 = (int)((e - e0) / VN), v1 = (int)((se - e0) / VN);
                        // slot vector v holds columns (e0 - rl ld) / VN + v of row rl (both multiples of VN)
                        const int xo = (int)((e0 - rl * ld) / VN);
                        TM a0 = TM(0), a1 = TM(0);
                        int v = v0 + lane;
#pragma unroll 2
                        for (; v + 32 < v1; v += 64) {
                            a0 = VT::dot(sv[v], xv[xo + v], a0);
                            a1 = VT::dot(sv[v + 32], xv[xo + v + 32], a1);
                        }
                        if (v < v1) a0 = VT::dot(sv[v], xv[xo + v], a0);
                        acc[t] = a0 + a1;
                        e = se;
                        ++rl;
                        ++nr;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                }
                if (lane == 0) {
                    for (int t = 0; t < nr; ++t) {
                        const long long r = rg + t;
                        const int k = (r * ld >= c * CH) ? 0 : (int)(c - flat_first_chunk(r, ld, CH));
                        spart[(r - br.rb0) * ph.ncmax + k] = acc[t];
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&R.empty[slot]);
                trace_mark(R, 2, me.fill, slot);
            }
            const int d = (slot + W < S) ? W : warp + S - slot;
            if (i + d >= cnt) break;
            i += d;
            me.advance(d, S);
        }
    } else if (i < cnt) {
        RingPos me = pos;
        me.advance(i, S);
        Walk w;
        w.CH = CH;
        w.first_of_row(ph, br.rb0);
        w.step(ph, i);
        while (true) {
            const Part& P = ph.p[w.p];
            const int slot = me.slot;
            if (!mbar_wait(&R.full[slot], (unsigned)(me.fill & 1))) *err = 1;
            if (lane == 0) trace_mark(R, 1, me.fill, slot);
            const V* sv = reinterpret_cast<const V*>(R.buf + (size_t)slot * R.slot_bytes);
            const V* xv = reinterpret_cast<const V*>(xs + P.xoff + w.c * CH);
            // vectors copied into the slot (the row's padding columns are zeros)
            const int vend = (int)(min((long long)CH, P.ld - (long long)w.c * CH) / VN);
            TM a0 = TM(0), a1 = TM(0);
            int v = lane;
#pragma unroll 2
            for (; v + 32 < vend; v += 64) {
                a0 = VT::dot(sv[v], xv[v], a0);
                a1 = VT::dot(sv[v + 32], xv[v + 32], a1);
            }
            if (v < vend) a0 = VT::dot(sv[v], xv[v], a0);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&R.empty[slot]);
                trace_mark(R, 2, me.fill, slot);
            }
            TM acc = warp_sum(a0 + a1);
            if (lane == 0) spart[(w.row - br.rb0) * ph.ncmax + w.k] = acc;
            const int d = (slot + W < S) ? W : warp + S - slot;
            if (i + d >= cnt) break;
            i += d;
            me.advance(d, S);
            w.step(ph, d);
        }
    }
    pos.advance(cnt, S);
}

// Sum each owned row's chunk partials in chunk order, add the row's CSR
// contributions (nonzeros in storage order), and write it to out[row].
template <typename TM, int NT>
__device__ __forceinline__ void row_sums(const Phase& ph, const BlockRange br, const TM* __restrict__ spart,
                                         TM* __restrict__ out, int slot_bytes, const TM* __restrict__ xs) {
    const int CH = slot_bytes / (int)sizeof(TM);
    for (int r = br.rb0 + (int)threadIdx.x; r < br.rb1; r += Blk<NT>::threads) {
        const int nk = ph.flat ? flat_row_chunks(r, ph.p[0].ld, CH) : row_items(ph, CH, r);
        const TM* sp = spart + (r - br.rb0) * ph.ncmax;
        TM s = TM(0);
        for (int k = 0; k < nk; ++k) s += sp[k];
        for (int q = 0; q < ph.np; ++q) {
            const Part& P = ph.p[q];
            if (!P.rp || r < P.r0 || r >= P.r1) continue;
            const TM* val = static_cast<const TM*>(P.M);
            const int k1 = __ldg(P.rp + (r - P.r0) + 1);
            for (int k = __ldg(P.rp + (r - P.r0)); k < k1; ++k) s = fma(__ldg(val + k), xs[P.xoff + __ldg(P.ci + k)], s);
        }
        out[r] = s;
    }
}

// Stage a phase's input from the previous phase's output (see Phase).  Loads are
// issued four per thread before any is used.
template <int NT, typename TX>
__device__ __forceinline__ void stage_input(const Phase& ph, TX* __restrict__ xs, const TX* __restrict__ out) {
    constexpr int T = Blk<NT>::threads;
    for (int j0 = threadIdx.x; j0 < ph.in_pad; j0 += 4 * T) {
        TX v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * T;
            v[u] = TX(0);
            if (j < ph.in_len1) {
                v[u] = __ldcg(out + j);
            } else if (ph.in_len2 > 0 && j >= ph.in_off2 && j < ph.in_off2 + ph.in_len2) {
                v[u] = (TX)ph.in_s2 * __ldcg(out + ph.in_len1 + (j - ph.in_off2));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * T;
            if (j < ph.in_pad) xs[j] = v[u];
        }
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

// Two fixed-order sums at once.
template <int NT, typename AT>
__device__ __forceinline__ void block_allsum2(AT& a, AT& b, AT* sh) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[w] = a; sh[16 + w] = b; }
    csync<NT>();
    if (threadIdx.x < 32) {
        AT ra = (l < Blk<NT>::warps) ? sh[l] : AT(0);
        AT rb = (l < Blk<NT>::warps) ? sh[16 + l] : AT(0);
        ra = warp_sum(ra);
        rb = warp_sum(rb);
        if (l == 0) { sh[32] = ra; sh[33] = rb; }
    }
    csync<NT>();
    a = sh[32];
    b = sh[33];
    csync<NT>();
}

template <typename TO, typename TP>
struct FusedArgs {
    int n, m1, m2;
    Phase ph[kMaxPhases];   // operator phases 0..nop-1, then the P_H phases nop..nop+npc-1
    int nop, npc;           // npc: 1 (the symmetric inverse P~^{-1}) or 2 (its two triangular factors)
    const int2* tbl;        // (first row, first item) of every block, per phase
    TO* out[kMaxPhases];    // output vectors of the operator phases
    TP* outP[2];            // outputs of the P_H phases
    const TP* sg;           // Jacobi scaling of P_H
    const TO* D;
    const TO* Dinv;
    TO* x;
    const TO* r_in;         // entry residual (= rhs) and search direction (= z0)
    const TO* p_in;
    PcgState* st;      // entry: rz_cur, tol2, maxit, done (from pcg_init); exit: iter, rr, done
    GridBar* bar;      // zeroed before the launch
    size_t xs_bytes;   // bytes of the staged-vector region of shared memory (16-byte multiple)
    size_t spart_off;  // byte offset of the per-row chunk partials
    size_t xo_off;     // byte offset of the block's slice of x (ceil(m2 / grid) elements)
    size_t ring_off;   // byte offset of the slot ring (128-byte aligned)
    int slots;         // ring depth S
    int slot_bytes;    // bytes of one slot (a multiple of 16)
    unsigned long long* tstamp;   // optional: %globaltimer marks of block 0 (4 iterations x 32) and
                                  // every block's phase ends of iteration 2 (8 x grid, after 128)
    int leave_early;              // failure-detection test: block 0 leaves before its first grid barrier
    int trace0;                   // first ring sequence number of block 0's chunk trace (see Ring)
    double* segp;                 // sliced FP64 update: per-segment partials of r'r (first nseg) and r'z
    TO* zbuf;                     // sliced FP64 update: z = P_L^{-1} r, every block's slice
    int nseg;                     // ceil(m2 / kSeg)
    int qcache;                   // 1: q (and P_H's z) cached in shared memory between passes;
                                  // 0: recomputed from global memory (same arithmetic), which
                                  // leaves room for the ring when m2-vectors of TO are large
};

// Shared-memory layout of the persistent kernel: staged vector, the m2-vector
// caches (r, p, and with qcache q or z, in TO), the per-row chunk partials, then
// the ring (slots, full and empty mbarriers, last-fill words, stop flag).
template <typename TO>
inline size_t fused_spart_offset(size_t xs_bytes, int m2, int qcache) {
    const size_t o = xs_bytes + (size_t)(2 + (qcache ? 1 : 0)) * (size_t)m2 * sizeof(TO);
    return (o + 15) / 16 * 16;
}
inline size_t fused_ring_offset(size_t spart_off, size_t spart_bytes) {
    const size_t o = spart_off + spart_bytes;
    return (o + 127) / 128 * 128;
}
inline size_t fused_smem_bytes(size_t ring_off, int slots, int slot_bytes) {
    return ring_off + (size_t)slots * (slot_bytes + 2 * sizeof(uint64_t) + sizeof(int)) + 16;
}

// The producer's sequence of phases, the consumers' loop below in the same order.
template <typename TO, typename TP, int PC>
__device__ void pcg_producer(const FusedArgs<TO, TP>& a, const BlockRange* brs, const Ring& R) {
    RingPos g;
    const int nph = a.nop + (PC == PC_H_K ? a.npc : 0);
    while (!*R.stop) {   // (a block may own no chunk of any phase: it polls the stop flag here)
        bool ok = true;
        for (int k = 0; k < nph && ok; ++k)
            ok = (k < a.nop) ? produce_phase<TO>(a.ph[k], brs[k], R, g) : produce_phase<TP>(a.ph[k], brs[k], R, g);
        if (!ok) break;
    }
    // drain: every copy issued lands before the block's shared memory goes away
    __syncwarp();
    const int lane = threadIdx.x & 31;
    for (int sl = lane; sl < R.S; sl += 32) {
        const int f = R.last_fill[sl];
        if (f >= 0) mbar_wait(&R.full[sl], (unsigned)(f & 1));
    }
}

// kind: PC_L_K (z = r / D), PC_H_K (z = Sg P~^{-1} Sg r), PC_NONE_K (z = r).
// Entry state (from pcg_init): x = 0, r = rhs, p = z0, st->rz_cur = r'z,
// st->tol2 = tol^2 |rhs|^2, st->maxit.
template <typename TO, typename TP, int PC, int NT>
__global__ void __launch_bounds__(NT, NT == kSmallBlock ? 2 : 1)
    pcg_fused_kernel(const __grid_constant__ FusedArgs<TO, TP> a) {
    constexpr int T = Blk<NT>::threads;
    PCG_COUNT_KERNEL();
    extern __shared__ __align__(128) unsigned char pcg_smem[];
    TO* xs = reinterpret_cast<TO*>(pcg_smem);
    TP* xp = reinterpret_cast<TP*>(pcg_smem);
    TO* rc = reinterpret_cast<TO*>(pcg_smem + a.xs_bytes);
    TO* pcs = rc + a.m2;
    TO* qc = pcs + a.m2;             // (only with a.qcache)
    const bool qcache = a.qcache != 0;
    Ring R;
    R.S = a.slots;
    R.slot_bytes = a.slot_bytes;
    R.buf = pcg_smem + a.ring_off;
    R.full = reinterpret_cast<uint64_t*>(R.buf + (size_t)R.S * a.slot_bytes);
    R.empty = R.full + R.S;
    R.last_fill = reinterpret_cast<int*>(R.empty + R.S);
    R.stop = reinterpret_cast<volatile int*>(R.last_fill + R.S);
    R.trace = (a.tstamp != nullptr && blockIdx.x == 0) ? a.tstamp + 128 + 8 * 1024 : nullptr;
    R.trace0 = a.trace0;
    using AT = typename Acc<TO>::type;
    using ATP = typename Acc<TP>::type;
    __shared__ AT sh[40];
    __shared__ int s_flag;
    __shared__ int s_err;
    __shared__ BlockRange s_br[kMaxPhases];
    const int m2 = a.m2;
    const int tid = threadIdx.x;
    const unsigned nblocks = gridDim.x;
    const int nph = a.nop + (PC == PC_H_K ? a.npc : 0);

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
    if (tid < nph) s_br[tid] = block_range(a.tbl, a.ph[tid]);
    __syncthreads();
    if (tid >= T) {
        pcg_producer<TO, TP, PC>(a, s_br, R);
        return;
    }

    // ------------------------------------------------------------ consumers
    TO* spart = reinterpret_cast<TO*>(pcg_smem + a.spart_off);
    TP* spartP = reinterpret_cast<TP*>(pcg_smem + a.spart_off);
    // slice of x this block owns: accumulated in shared memory (x = 0 at entry),
    // written to global memory when the solve ends
    // With an FP64 operator and P_L (or no preconditioner) the r, x and z updates are
    // sliced: block b updates only the elements of segments [sb, se) (kSeg elements
    // each), publishes z and the segments' partial sums of r'r and r'z, and after one
    // more grid barrier every block adds the partials in segment order.  The update's
    // 5 FP64 operations per element then run once on the GPU instead of once per block
    // (the FP64 pipe issues 2 per clock per SM), and every sum keeps an order that does
    // not depend on the grid.
    constexpr bool SL = std::is_same<TO, double>::value && PC != PC_H_K;
    const int warp = tid >> 5, lane = tid & 31;
    const int sb = (int)((long long)a.nseg * blockIdx.x / nblocks);
    const int se = (int)((long long)a.nseg * (blockIdx.x + 1) / nblocks);
    const int per = (m2 + nblocks - 1) / nblocks;
    const int own0 = SL ? min(m2, sb * kSeg) : (int)blockIdx.x * per;
    const int own1 = SL ? min(m2, se * kSeg) : min(m2, own0 + per);
    TO* xo = reinterpret_cast<TO*>(pcg_smem + a.xo_off);
    for (int j = tid; j < own1 - own0; j += T) xo[j] = TO(0);
    // staged m2-vectors are padded to 32 elements (the leading dimension of C' and P~^{-1})
    const int padO_m2 = ((m2 + 31) / 32) * 32, padP_m2 = padO_m2;
    const bool stamp = a.tstamp != nullptr && blockIdx.x == 0 && tid == 0;
    auto mark = [&](int it, int ph) {
        if (stamp && it < 4) a.tstamp[it * 32 + ph] = gtimer();
    };
    // every block's phase end (before its barrier arrival) in iteration 2
    auto mark_all = [&](int it, int ph) {
        if (a.tstamp != nullptr && tid == 0 && it == 2 && ph < 8)
            a.tstamp[128 + ph * nblocks + blockIdx.x] = gtimer();
    };
    unsigned target = 0;
    RingPos g;   // ring position of the next chunk
    // every consumer exit passes here: the producer stops issuing and drains
    auto leave = [&]() {
        csync<NT>();
        if (tid == 0) {
            if (s_err) atomicOr(&a.bar->count, kBarErr);
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

    // first iteration: p and r from the entry state; xs = p
    for (int j = tid; j < m2; j += T) {
        pcs[j] = __ldcg(a.p_in + j);
        rc[j] = __ldcg(a.r_in + j);
    }
    csync<NT>();
    for (int j = tid; j < padO_m2; j += T) xs[j] = (j < m2) ? pcs[j] : TO(0);
    csync<NT>();

    // failure-detection test: block 0 stops before the first grid barrier, as a block
    // that died would; every other block's bounded wait runs out and reports QP_ETIMEOUT
    if (a.leave_early && blockIdx.x == 0 && nblocks > 1) { leave(); return; }

    while (true) {
        mark(it, 0);
        // ---- operator phases (a6-a8): K_F p = D p + C y, y from C'p and the K0 solve
        for (int k = 0; k < a.nop; ++k) {
            const Phase& ph = a.ph[k];
            if (k > 0) {
                stage_input<NT, TO>(ph, xs, a.out[k - 1]);
                csync<NT>();
                mark(it, 10 + k);
            }
            consume_phase<TO, NT>(ph, s_br[k], R, g, xs, spart, &s_err);
            csync<NT>();
            row_sums<TO, NT>(ph, s_br[k], spart, a.out[k], a.slot_bytes, xs);
            mark(it, 15 + k);
            mark_all(it, k);
            if (!gsync()) { leave(); return; }
            mark(it, 1 + k);
        }

        // ---- (a10) q = D p + w (cached), alpha = r'z / p'q, x += alpha p, r -= alpha q
        // Each thread takes the elements j = tid + u T, all of a pass's global loads issued
        // before any is used (one round of latency per pass); sums in increasing u.
        AT pq = AT(0);
        const TO* w = a.out[a.nop - 1];
        // the next pass's 1/D (P_L), loaded here so that its latency overlaps this pass
        TO zv[kNU];
#pragma unroll
        for (int u = 0; u < kNU; ++u) {
            const int j = tid + u * T;
            zv[u] = (PC == PC_L_K && j < m2) ? __ldg(a.Dinv + j) : TO(1);
        }
        {
            TO wv[kNU], dv[kNU];
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int j = tid + u * T;
                wv[u] = j < m2 ? __ldcg(w + j) : TO(0);
                dv[u] = j < m2 ? __ldg(a.D + j) : TO(0);
            }
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int j = tid + u * T;
                if (j < m2) {
                    const TO q = (TO)fma((AT)dv[u], (AT)pcs[j], (AT)wv[u]);
                    if (qcache) qc[j] = q;
                    pq = fma((AT)pcs[j], (AT)q, pq);
                }
            }
            for (int j = tid + kNU * T; j < m2; j += T) {
                const TO q = (TO)fma((AT)__ldg(a.D + j), (AT)pcs[j], (AT)__ldcg(w + j));
                if (qcache) qc[j] = q;
                pq = fma((AT)pcs[j], (AT)q, pq);
            }
        }
        pq = block_allsum<NT>(pq, sh);
        mark(it, 6);
        // breakdown (p'q <= 0 or not finite): stop with the last iterate untouched
        if (!(pq > AT(0)) || !isfinite(pq)) { done = 3; break; }
        const AT alpha = rz / pq;
        const TO al = (TO)alpha;
        AT rrp = AT(0), rzp = AT(0);
        if (SL) {
            // this block's segments: one warp per segment, lanes on elements k * 32 + lane
            for (int sg = sb + warp; sg < se; sg += Blk<NT>::warps) {
                AT prr = AT(0), prz = AT(0);
#pragma unroll
                for (int k = 0; k < kSeg / 32; ++k) {
                    const int j = sg * kSeg + k * 32 + lane;
                    if (j < m2) {
                        const TO qj = qcache ? qc[j] : (TO)fma((AT)__ldg(a.D + j), (AT)pcs[j], (AT)__ldcg(w + j));
                        const TO rn = fma(-al, qj, rc[j]);
                        rc[j] = rn;
                        prr = fma((AT)rn, (AT)rn, prr);
                        xo[j - own0] = fma(al, pcs[j], xo[j - own0]);
                        const TO z = (PC == PC_L_K) ? rn * __ldg(a.Dinv + j) : rn;
                        a.zbuf[j] = z;
                        prz = fma((AT)rn, (AT)z, prz);
                    }
                }
                prr = warp_sum(prr);
                prz = warp_sum(prz);
                if (lane == 0) {
                    a.segp[sg] = (double)prr;
                    a.segp[a.nseg + sg] = (double)prz;
                }
            }
            if (!gsync()) { leave(); return; }
            if (warp == 0) {
                AT srr = AT(0), srz = AT(0);
                for (int sg = lane; sg < a.nseg; sg += 32) {
                    srr += (AT)__ldcg(a.segp + sg);
                    srz += (AT)__ldcg(a.segp + a.nseg + sg);
                }
                srr = warp_sum(srr);
                srz = warp_sum(srz);
                if (lane == 0) { sh[32] = srr; sh[33] = srz; }
            }
            csync<NT>();
            rrp = sh[32];
            rzp = sh[33];
            csync<NT>();
        } else {
            // the preconditioner's diagonal factor: 1/D (P_L) or the Jacobi scaling Sg (P_H)
            const TO* dz = (PC == PC_L_K) ? a.Dinv : nullptr;
            TP gv[kNU];
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int j = tid + u * T;
                gv[u] = (PC == PC_H_K && j < m2) ? __ldg(a.sg + j) : TP(0);
            }
            auto update = [&](int j, TO dzj, TP sgj) {
                const TO qj = qcache ? qc[j] : (TO)fma((AT)__ldg(a.D + j), (AT)pcs[j], (AT)__ldcg(w + j));
                const TO rn = fma(-al, qj, rc[j]);
                rc[j] = rn;
                rrp = fma((AT)rn, (AT)rn, rrp);
                if (j >= own0 && j < own1) xo[j - own0] = fma(al, pcs[j], xo[j - own0]);
                if (PC == PC_H_K) {
                    xp[j] = (TP)((AT)rn * (AT)sgj);
                } else {
                    const TO z = rn * dzj;   // (dzj = 1 without a preconditioner)
                    xs[j] = z;               // z for the p update below (xs is free until then)
                    rzp = fma((AT)rn, (AT)z, rzp);
                }
            };
#pragma unroll
            for (int u = 0; u < kNU; ++u) {
                const int j = tid + u * T;
                if (j < m2) update(j, zv[u], gv[u]);
            }
            for (int j = tid + kNU * T; j < m2; j += T)
                update(j, (PC == PC_L_K) ? __ldg(dz + j) : TO(1), (PC == PC_H_K) ? __ldg(a.sg + j) : TP(0));
        }
        for (int j = m2 + tid; j < padO_m2; j += T) {
            if (PC == PC_H_K) xp[j] = TP(0); else xs[j] = TO(0);
        }
        if (SL) {
            rr = rrp;
        } else if (PC == PC_H_K) {
            rr = block_allsum<NT>(rrp, sh);
        } else {
            block_allsum2<NT>(rrp, rzp, sh);
            rr = rrp;
        }
        ++it;
        mark(it - 1, 7);
        const bool finite = isfinite(rr) && isfinite(pq);
        if (!finite) { done = 3; break; }
        if ((double)rr <= tol2) { done = 1; break; }
        if (it >= maxit) { done = 2; break; }

        AT rz_new;
        const TP* vout = a.outP[a.npc > 0 ? a.npc - 1 : 0];
        if (PC == PC_H_K) {
            // ---- (a9) v = P~^{-1} (Sg r) (one symmetric phase, or W then W'), z = Sg v
            for (int k = 0; k < a.npc; ++k) {
                const Phase& ph = a.ph[a.nop + k];
                if (k > 0) {
                    stage_input<NT, TP>(ph, xp, a.outP[k - 1]);
                    csync<NT>();
                }
                consume_phase<TP, NT>(ph, s_br[a.nop + k], R, g, xp, spartP, &s_err);
                csync<NT>();
                row_sums<TP, NT>(ph, s_br[a.nop + k], spartP, a.outP[k], a.slot_bytes, xp);
                mark(it - 1, 19 + k);
                mark_all(it - 1, a.nop + k);
                if (!gsync()) { leave(); return; }
            }
            mark(it - 1, 8);
            // z into the q cache (q is no longer needed), then r'z
            rzp = AT(0);
            {
                TP vv[kNU], sv[kNU];
#pragma unroll
                for (int u = 0; u < kNU; ++u) {
                    const int j = tid + u * T;
                    vv[u] = j < m2 ? __ldcg(vout + j) : TP(0);
                    sv[u] = j < m2 ? __ldg(a.sg + j) : TP(0);
                }
#pragma unroll
                for (int u = 0; u < kNU; ++u) {
                    const int j = tid + u * T;
                    if (j < m2) {
                        const TO z = (TO)((ATP)sv[u] * (ATP)vv[u]);
                        if (qcache) qc[j] = z;
                        rzp = fma((AT)rc[j], (AT)z, rzp);
                    }
                }
                for (int j = tid + kNU * T; j < m2; j += T) {
                    const TO z = (TO)((ATP)__ldg(a.sg + j) * (ATP)__ldcg(vout + j));
                    if (qcache) qc[j] = z;
                    rzp = fma((AT)rc[j], (AT)z, rzp);
                }
            }
            rz_new = block_allsum<NT>(rzp, sh);
        } else {
            rz_new = rzp;
        }
        // ---- beta, p = z + beta p (staged as the next first-phase input; shared-memory only)
        const AT beta = rz_new / rz;
        rz = rz_new;
        const TO be = (TO)beta;
#pragma unroll 4
        for (int j = tid; j < padO_m2; j += T) {
            TO v = TO(0);
            if (j < m2) {
                TO z;
                if (PC == PC_H_K) z = qcache ? qc[j] : (TO)((ATP)__ldg(a.sg + j) * (ATP)__ldcg(vout + j));
                else z = SL ? __ldcg(a.zbuf + j) : xs[j];
                v = fma(be, pcs[j], z);
                pcs[j] = v;
            }
            xs[j] = v;
        }
        csync<NT>();
        mark(it - 1, 9);
    }
    csync<NT>();
    for (int j = own0 + tid; j < own1; j += T) a.x[j] = xo[j - own0];
    if (blockIdx.x == 0 && tid == 0) {
        a.st->iter = it;
        a.st->rr = (double)rr;
        a.st->rz_cur = (double)rz;
        a.st->done = done;
    }
    leave();
}

}  // namespace pcgipm
