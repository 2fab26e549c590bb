// tc_gemm.cuh -- dense contractions of the factorizations on the tcgen05 tensor cores.
//
//   C[i, j] = alpha * sum_k A[i, k] B[j, k] + beta * C[i, j]      (FP32 in and out)
//
// A (M x K) and B (N x K) are row-major with k contiguous ("K-major"), the form
// of every product the factorizations take: the trailing update A22 -= L21 L21'
// of a blocked Cholesky, T = (C R^{-1})(C R^{-1})', P~^{-1} = W'W, M0.
//
// The tensor cores take TF32 operands (10 explicit mantissa bits).  With
// `split` each operand is written as hi + lo (hi = the operand rounded to TF32,
// lo = the exact FP32 remainder) and the product is accumulated as
// hi*hi + hi*lo + lo*hi in FP32 (the lo*lo term, below 2^-21 relative, is left
// out): an FP32-accurate product at a third of the TF32 rate.  Without it, one
// TF32 product.
//
// One CTA computes one 128 x 128 tile of C: a producer warp loads 32-wide K
// slices of A and B into a ring of shared-memory stages with TMA
// (cp.async.bulk.tensor, 128-byte swizzle, zero fill outside the matrices); one
// thread of the MMA warp issues tcgen05.mma (kind::tf32, M = 128, N = 128, K = 8
// per instruction) into FP32 accumulators in tensor memory and releases each
// stage with tcgen05.commit.  K slice kt goes to accumulator kt mod kTcAcc, so
// each accumulator sums a quarter of the products: the tensor core's FP32
// accumulation does not round to nearest, and its error grows with the number
// of terms summed in one accumulator (one accumulator over K = 4000 made the
// explicit P~^{-1} = W'W indefinite enough to stall PCG).  Four epilogue warps
// read the accumulators back with tcgen05.ld (each warp its 32-lane quarter: one
// row of C per thread), add them in a fixed order, apply alpha, and pass each
// 32 x 32 piece through shared memory so that every store (and the beta read)
// covers a row segment of 32 consecutive elements.  With `lower_out` only tiles
// on or below the diagonal run and only elements j <= i are written.
//
// Every wait is bounded (kTcWaitNs of %globaltimer): a wait that gives up sets
// *err, the kernel skips the remaining work, waits (bounded) for its issued
// copies and MMAs, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace pcgipm {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 32;        // tile; BK = one 128-byte swizzle row of FP32
constexpr int kTcThreads = 192;                            // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr unsigned long long kTcWaitNs = 2000000000ull;     // 2 s bound on any wait
constexpr int kTcTileBytes = kTcBM * kTcBK * 4;            // 16 KB per operand slice
constexpr int kTcAcc = 4;                                  // accumulators (128 TMEM columns each)

__device__ __forceinline__ unsigned long long tc_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned tc_smem(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void tc_mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc_smem(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false after kTcWaitNs.
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* b, unsigned parity) {
    if (tc_mbar_try(b, parity)) return true;
    const unsigned long long t0 = tc_gtimer();
    while (!tc_mbar_try(b, parity))
        if (tc_gtimer() - t0 > kTcWaitNs) return false;
    return true;
}
__device__ __forceinline__ void tc_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(b)), "r"(bytes) : "memory");
}
// 2-D TMA load of the box at (x = column, y = row) into shared memory; completion in bytes on `bar`.
__device__ __forceinline__ void tc_tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            tc_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tc_smem(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand slice of 128 rows x 128
// bytes written by TMA with the 128-byte swizzle: rows of 128 bytes, groups of
// 8 rows 1024 bytes apart (stride byte offset), leading byte offset unused by
// swizzled K-major layouts (1), descriptor version 1, layout 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t tc_desc_sw128(const void* smem_tile) {
    const uint64_t addr = tc_smem(smem_tile);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;                 // start address
    d |= (uint64_t)1 << 16;                       // leading byte offset (unused)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                       // version
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4)                  // D format: F32
           | (2u << 7)                // A format: TF32
           | (2u << 10)               // B format: TF32
           | ((uint32_t)(N >> 3) << 17)
           | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
                 : "memory");
}

struct TcGemmParams {
    int M, N, K;
    float alpha, beta;
    float* C;
    long long ldc;
    int split;        // 1: A and B come as hi and lo maps (hi*hi + hi*lo + lo*hi)
    int lower_out;    // only tiles with a column block <= the row block; only j <= i written
    int* err;         // set to 1 when a wait gives up
};

// Kernel: one 128 x 128 tile of C per CTA.  Stage layout: [A hi][B hi]([A lo][B lo]).
template <int STAGES>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapBh,
                   const __grid_constant__ CUtensorMap mapAl, const __grid_constant__ CUtensorMap mapBl,
                   const TcGemmParams p) {
    PCG_COUNT_KERNEL();
    const int tm = blockIdx.y, tn = blockIdx.x;
    if (p.lower_out && tn > tm) return;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte alignment of the stages (the 128-byte swizzle repeats every 8 rows)
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nops = p.split ? 4 : 2;
    const int stage_bytes = nops * kTcTileBytes;
    __shared__ uint64_t full[STAGES], empty[STAGES], accum;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ktiles = (p.K + kTcBK - 1) / kTcBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc_mbar_init(&full[s], 1);
            tc_mbar_init(&empty[s], 1);
        }
        tc_mbar_init(&accum, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {   // tensor memory: 128 lanes x kTcAcc * 128 FP32 columns (the accumulators)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_base)),
                     "r"(kTcAcc * kTcBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ---- producer: one lane issues the TMA loads of every K slice
        if (lane == 0) {
            int issued = 0;
            for (int kt = 0; kt < ktiles; ++kt) {
                const int s = kt % STAGES;
                const int round = kt / STAGES;
                if (round > 0 && !tc_mbar_wait(&empty[s], (unsigned)((round - 1) & 1))) {
                    s_fail = 1;
                    atomicExch(p.err, 1);
                    break;
                }
                if (*(volatile int*)&s_fail) break;
                issued = kt + 1;
                unsigned char* st = base + (size_t)s * stage_bytes;
                tc_expect_tx(&full[s], (unsigned)stage_bytes);
                const int x = kt * kTcBK;
                tc_tma_load(st, &mapAh, x, tm * kTcBM, &full[s]);
                tc_tma_load(st + kTcTileBytes, &mapBh, x, tn * kTcBN, &full[s]);
                if (p.split) {
                    tc_tma_load(st + 2 * kTcTileBytes, &mapAl, x, tm * kTcBM, &full[s]);
                    tc_tma_load(st + 3 * kTcTileBytes, &mapBl, x, tn * kTcBN, &full[s]);
                }
            }
            // after a failure, the copies still in flight land before the CTA exits
            if (*(volatile int*)&s_fail)
                for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
                    tc_mbar_wait(&full[kt % STAGES], (unsigned)((kt / STAGES) & 1));
        }
    } else if (warp == 1) {
        // ---- MMA issuer: one lane
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc_tf32(kTcBM, kTcBN);
            bool ok = true;
            for (int kt = 0; kt < ktiles && ok; ++kt) {
                const int s = kt % STAGES;
                if (!tc_mbar_wait(&full[s], (unsigned)((kt / STAGES) & 1))) {
                    ok = false;
                    s_fail = 1;
                    atomicExch(p.err, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = base + (size_t)s * stage_bytes;
                const uint64_t ah = tc_desc_sw128(st), bh = tc_desc_sw128(st + kTcTileBytes);
                const uint64_t al = tc_desc_sw128(st + 2 * kTcTileBytes), bl = tc_desc_sw128(st + 3 * kTcTileBytes);
                const uint32_t d = tmem + (uint32_t)((kt % kTcAcc) * kTcBN);
#pragma unroll
                for (int kk = 0; kk < kTcBK / 8; ++kk) {
                    // K = 8 TF32 = 32 bytes per instruction: advance the start address by 2 (x 16 B)
                    const uint64_t o = (uint64_t)(kk * 2);
                    const int acc = (kt >= kTcAcc || kk > 0) ? 1 : 0;
                    tc_mma_tf32(d, ah + o, bh + o, idesc, acc);
                    if (p.split) {
                        tc_mma_tf32(d, ah + o, bl + o, idesc, 1);
                        tc_mma_tf32(d, al + o, bh + o, idesc, 1);
                    }
                }
                tc_commit(&empty[s]);   // the stage is free once these MMAs have read it
            }
            tc_commit(&accum);          // the accumulator is complete (or abandoned)
        }
    } else {
        // ---- epilogue: warps 2..5, TMEM lane quarter (warp % 4), one row per thread
        const int q = warp & 3;
        const bool ok = tc_mbar_wait(&accum, 0u);
        if (!ok) atomicExch(p.err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // every MMA has completed (or none will run): the stages are free for the
        // 32 x 33 staging piece of each epilogue warp
        const bool write = __all_sync(0xffffffffu, ok && ktiles > 0 && !*(volatile int*)&s_fail);
        float* stg = reinterpret_cast<float*>(base) + q * 32 * 33;
        const int nacc = ktiles < kTcAcc ? ktiles : kTcAcc;
        const int row0 = tm * kTcBM + q * 32;
#pragma unroll 1
        for (int c0 = 0; c0 < kTcBN; c0 += 32) {
            float acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
#pragma unroll 1
            for (int a = 0; a < nacc; ++a) {   // (nacc is the same in every lane)
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * kTcBN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] += __uint_as_float(v[j]);
            }
            if (write) {
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = p.alpha * acc[j];
                __syncwarp();
                const int col = tn * kTcBN + c0 + lane;
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
                    const int row = row0 + r;
                    if (row < p.M && col < p.N && (!p.lower_out || col <= row)) {
                        float* cp = p.C + (long long)row * p.ldc + col;
                        float x = stg[r * 33 + lane];
                        if (p.beta != 0.0f) x = fmaf(p.beta, *cp, x);
                        *cp = x;
                    }
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcAcc * kTcBN)
                     : "memory");
    }
}

// hi = x rounded to TF32 (round to nearest, ties away), lo = x - hi (exact in FP32).
__global__ void tc_split_kernel(const float* __restrict__ x, long long ldx, int rows, int cols, float* __restrict__ hi,
                                float* __restrict__ lo, long long ldo) {
    PCG_COUNT_KERNEL();
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        const float v = x[i * ldx + j];
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
        const float hv = __uint_as_float(h);
        hi[i * ldo + j] = hv;
        if (lo) lo[i * ldo + j] = v - hv;
    }
}

// ----------------------------------------------------------------- host side
using PFN_encodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline PFN_encodeTiled tc_encode_fn() {
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a row-major FP32 matrix (rows x cols, leading dimension ld
// elements) read in boxes of 128 rows x 32 columns with the 128-byte swizzle;
// coordinates outside the matrix read zeros.  False if the map cannot be made
// (base not 16-byte aligned, ld * 4 not a multiple of 16, no driver entry point).
inline bool tc_make_map(CUtensorMap* m, const float* base, int rows, int cols, long long ld) {
    PFN_encodeTiled fn = tc_encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15) || rows <= 0 || cols <= 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcBM};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kTcStagesSplit = 3, kTcStagesPlain = 5;
inline size_t tc_smem_bytes(bool split) {
    return (size_t)(split ? kTcStagesSplit * 4 : kTcStagesPlain * 2) * kTcTileBytes + 1024;
}

// C = alpha A B' + beta C on the tensor cores.  A (M x K, lda), B (N x K, ldb)
// row-major FP32 (or, with `split`, their hi/lo parts Ah, Al, Bh, Bl as written
// by tc_split_kernel).  Returns false (nothing launched) if a tensor map cannot
// be made.
inline bool tc_gemm(int M, int N, int K, float alpha, const float* Ah, const float* Al, long long lda,
                    const float* Bh, const float* Bl, long long ldb, float beta, float* C, long long ldc,
                    bool split, bool lower_out, int* d_err, cudaStream_t s) {
    if (M <= 0 || N <= 0) return true;
    CUtensorMap mah, mbh, mal, mbl;
    if (!tc_make_map(&mah, Ah, M, K, lda) || !tc_make_map(&mbh, Bh, N, K, ldb)) return false;
    if (split) {
        if (!tc_make_map(&mal, Al, M, K, lda) || !tc_make_map(&mbl, Bl, N, K, ldb)) return false;
    } else {
        mal = mah;
        mbl = mbh;
    }
    TcGemmParams p{M, N, K, alpha, beta, C, ldc, split ? 1 : 0, lower_out ? 1 : 0, d_err};
    dim3 grid((N + kTcBN - 1) / kTcBN, (M + kTcBM - 1) / kTcBM);
    const size_t smem = tc_smem_bytes(split);
    if (split) {
        static const cudaError_t a = cudaFuncSetAttribute(tc_gemm_kernel<kTcStagesSplit>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (a != cudaSuccess) return false;
        tc_gemm_kernel<kTcStagesSplit><<<grid, kTcThreads, smem, s>>>(mah, mbh, mal, mbl, p);
    } else {
        static const cudaError_t a = cudaFuncSetAttribute(tc_gemm_kernel<kTcStagesPlain>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (a != cudaSuccess) return false;
        tc_gemm_kernel<kTcStagesPlain><<<grid, kTcThreads, smem, s>>>(mah, mbh, mal, mbl, p);
    }
    return true;
}

}  // namespace pcgipm
