// engine.cuh -- one QP on one GPU: setup factorization, the implicit K_F
// product, graph-captured PCG, reduced Newton solves with FP64 refinement and
// the primal-dual IPM loop.
//
// Precisions.  The operator of the hot path (C, C' and the stored K0 factor,
// with the PCG vectors) runs in TO; the factored preconditioner P_H in TP;
// everything the IPM decides with (residuals, refinement residuals, step
// lengths, centrality) is FP64.
//   QP_PREC_FP64: TO = TP = double.
//   QP_PREC_FP32: TP = float; TO starts as float and a QP switches to TO =
//   double (a second, FP64 factor of K0) once FP64 refinement of a Newton
//   direction contracts too slowly -- the FP32 operator's error is amplified by
//   the conditioning of K_F on the active set late in the IPM.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/pcgipm.h"
#include "common.cuh"
#include "dense.cuh"
#include "dense_bk.cuh"
#include "gemv.cuh"
#include "pcg_fused.cuh"
#include "vec.cuh"

namespace pcgipm {

struct CudaError {
    cudaError_t e;
    int line;
};
struct NoMem {};
struct QpError { int code; };

#define PCG_CK(x)                                                       \
    do {                                                                \
        cudaError_t _e = (x);                                           \
        if (_e != cudaSuccess) throw ::pcgipm::CudaError{_e, __LINE__}; \
    } while (0)

// Owns every device allocation of one handle (zero-initialised on the handle's
// stream, so that the zeroing is ordered before the handle's own kernels: the
// legacy default stream does not order against a non-blocking stream).
class DevArena {
public:
    ~DevArena() { release(); }
    cudaStream_t stream = nullptr;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        const size_t bytes = count * sizeof(T) + 256;
        if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            if (std::getenv("PCGIPM_VERBOSE")) std::fprintf(stderr, "  device allocation of %zu bytes failed\n", bytes);
            throw NoMem{};
        }
        PCG_CK(cudaMemsetAsync(p, 0, bytes, stream));
        ptrs_.push_back(p);
        bytes_ += bytes;
        return static_cast<T*>(p);
    }
    // Stream-ordered frees: no device-wide synchronisation (cudaFree would wait for
    // every stream, stalling other QPs solved concurrently).
    void release() {
        for (void* p : ptrs_) cudaFreeAsync(p, stream);
        ptrs_.clear();
    }
    size_t bytes() const { return bytes_; }

private:
    std::vector<void*> ptrs_;
    size_t bytes_ = 0;
};

template <typename T>
struct Mat {
    T* p = nullptr;
    int rows = 0, cols = 0;
    long long ld = 0;
    void alloc(DevArena& a, int r, int c) {
        rows = r;
        cols = c;
        ld = pad_ld(c > 0 ? c : 1);
        p = a.alloc<T>((size_t)(r > 0 ? r : 1) * ld);
    }
};

// y_i = a acc + b z_i + c w_i + e dv_i dx_i  (optional terms skipped when null)
template <typename T>
struct EpiLin {
    T* y;
    T a;
    const T* z; T b;
    const T* w; T c;
    const T* dv; const T* dx; T e;
    __device__ __forceinline__ double operator()(int i, T acc) const {
        T v = a * acc;
        if (z) v += b * z[i];
        if (w) v += c * w[i];
        if (dv) v += e * dv[i] * dx[i];
        y[i] = v;
        return 0.0;
    }
};

template <typename T>
inline EpiLin<T> lin(T* y, T a = T(1), const T* z = nullptr, T b = T(0), const T* w = nullptr, T c = T(0),
                     const T* dv = nullptr, const T* dx = nullptr, T e = T(0)) {
    return EpiLin<T>{y, a, z, b, w, c, dv, dx, e};
}

inline int resolve_pc(int pc, int n, int m1) {
    if (pc == QP_PC_AUTO) return (2 * m1 >= n) ? QP_PC_PL : QP_PC_PH_EXACT;
    return pc;
}

inline int pc_kind(int pc) {
    if (pc == QP_PC_PL) return PC_L_K;
    if (pc == QP_PC_PH_EXACT || pc == QP_PC_PH_DIAG) return PC_H_K;
    return PC_NONE_K;
}

// Operator of the hot path in precision TO: C, C', the inverted K0 factor, and
// the PCG / K0-solve vectors.
template <typename TO>
struct Op {
    Mat<TO> CW, CWT;   // C and C'
    Mat<TO> WH, WHT;   // R^{-T} = L_H^{-1} (lower) and R^{-1} (upper), H = R'R
    Mat<TO> Gt, GtT;   // L_S^{-1} A R^{-1} and its transpose, L_S L_S' = A H^{-1} A'
    Mat<TO> Et, EtT;   // Gt R^{-T} = L_S^{-1} A H^{-1} (the (2,1) block of L^{-1}) and its transpose
    Mat<TO> WS, WST;   // L_S^{-1} (lower) and L_S^{-T} (upper)
    Mat<TO> BW, BWT;   // pcg_form 1: B = L^{-1}[C'; 0] = [R^{-T} C'; Et C'] ((n+m1) x m2) and B'
    Mat<TO> M0;        // [K0^{-1}]_11 = R^{-1} R^{-T} - Et' Et (n x n, symmetric), pcg_form 0 and 3
    Mat<TO> LV, LVT;   // pcg_form 3: V = C Z (m2 x r) and V', M0 = Z Z', r = rank(M0) = n - m1
    int lr = 0;        // pcg_form 3: r
    const TO *cval = nullptr, *ctval = nullptr;   // CSR values of C and C' (QPs created with a CSR C)
    TO *oU = nullptr, *oY, *oZ, *oW;   // persistent kernel: outputs of the operator phases
    TO *px = nullptr, *pr, *pz, *pp, *pq, *pu, *pz1, *pz2, *pt, *py, *prhs, *pD, *pDinv;
    TO* zb = nullptr;          // persistent kernel, sliced FP64 update: z
    double* segp = nullptr;    // persistent kernel, sliced FP64 update: per-segment partial sums
    TO *ku, *kw, *ke, *kz1, *kz2, *kt, *ka, *kmb, *wa, *wg;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    int graph_k[3] = {0, 0, 0};
    bool factored = false;
};

// Factored preconditioner P_H in precision TP.
template <typename TP>
struct Pc {
    Mat<TP> Tm, Pm, WPl, WPu;   // T = C H^{-1} C' (or C diag(H)^{-1} C'), P~, L^{-1}, L^{-T}
    Mat<TP> PI;                 // P~^{-1} = L^{-T} L^{-1} (m2 x m2, symmetric; FP32 P_H)
    TP *sg = nullptr, *rs, *pv, *Dp;
    TP *oV[2] = {nullptr, nullptr};   // persistent kernel: outputs of the P_H phases
    int t_kind = 0;
    double shift = 0.0;
};

class Engine {
public:
    int n = 0, m1 = 0, m2 = 0;
    qp_opts opt{};
    cudaStream_t s = nullptr;
    bool own_stream = false;
    bool factored = false;
    bool f64 = false;       // QP_PREC_FP64
    bool all64 = false;     // QP_PREC_FP32 whose K0 factor needed FP64 pivots: the QP runs in FP64
    bool use64 = false;     // operator currently in FP64
    bool pc64 = false;      // preconditioner currently in FP64
    DevArena arena;
    qp_stats stats{};
    double* stage[4] = {nullptr, nullptr, nullptr, nullptr};
    bool verbose = false;
    int ipm_k = 0;

    // FP64 problem data (masters for residuals and refinement)
    Mat<double> H, A, AT, C, CT;
    // C in CSR form (qp_create_csr): C (m2 rows) and C' (n rows), indices and FP64 values
    int *crp = nullptr, *cci = nullptr, *ctrp = nullptr, *ctci = nullptr;
    double *cval64 = nullptr, *ctval64 = nullptr;
    long long nnz = 0;
    double *c = nullptr, *b = nullptr, *d = nullptr;
    double h_norm_inf = 0, b_inf = 0, c_inf = 0, d_inf = 0;

    Op<float> o32;
    Op<double> o64;
    Pc<float> p32;
    Pc<double> p64;

    double *part_pq, *part_rr, *part_rz, *part_bb, *part_a, *part_b, *part_c, *part_d, *part_e, *part_f, *diag0;
    PcgState* st = nullptr;
    PcgState* hst = nullptr;   // pinned, 2 slots
    double* d_scal = nullptr;
    double* h_scal = nullptr;  // pinned
    int* d_info = nullptr;
    int* h_info = nullptr;     // pinned
    cudaEvent_t ev0, ev1, evA, evB, evW;
    int cap_rows = 0;
    int last_pcg_done = 0;
    double last_pcg_rel = 0.0;
    double cur_tol = 0.0;       // tolerance of the PCG solve being run
    GridBar* bar = nullptr;
    bool allow_pc64 = true;
    int ipm_pc = 0;             // preconditioner of the IPM solve in progress (enum qp_precond)
    const void* cl_key = nullptr;   // last cluster-launch check: kernel, grid, shared memory, result
    int cl_grid = 0;
    size_t cl_smem = 0;
    bool cl_ok = false;
    bool phase_times = false;
    bool leave_early = false;   // PCGIPM_TEST_LEAVE_EARLY=1: failure-detection test of the bounded waits
    unsigned long long* tstamp = nullptr;

    // FP64 IPM vectors
    double *x, *lam, *nu, *sl, *hx, *rg, *re, *ri, *rc, *ra, *D64;
    double *dx, *dl, *dn, *ds, *dxa, *dla, *dna, *dsa;
    double *fg, *fe, *fa, *rho_g, *rho_e, *rho_a, *tx, *tl, *tn;

    template <typename TO> Op<TO>& op() {
        if constexpr (std::is_same<TO, float>::value) return o32; else return o64;
    }
    template <typename TP> Pc<TP>& pcd() {
        if constexpr (std::is_same<TP, float>::value) return p32; else return p64;
    }

    Engine(int n_, int m1_, int m2_, const qp_opts& o, bool csr_c = false) {
        n = n_; m1 = m1_; m2 = m2_; opt = o;
        form_auto = (opt.pcg_form == QP_FORM_AUTO);
        opt.pcg_form = resolve_form(opt.pcg_form, n, m1, m2, csr_c);
        stats.pcg_form_used = opt.pcg_form;
        stats.k0_inertia_pos = stats.k0_inertia_neg = stats.k0_pivots_2x2 = -1;
        f64 = (opt.precision == QP_PREC_FP64);
        use64 = f64;
        pc64 = f64;
        if (opt.stream) {
            s = static_cast<cudaStream_t>(opt.stream);
        } else {
            PCG_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            own_stream = true;
        }
        arena.stream = s;
        // blocking_wait: host waits yield the CPU (many QPs in flight, more host threads than cores)
        const unsigned evf = opt.blocking_wait ? cudaEventBlockingSync : cudaEventDefault;
        PCG_CK(cudaEventCreateWithFlags(&ev0, evf));
        PCG_CK(cudaEventCreateWithFlags(&ev1, evf));
        PCG_CK(cudaEventCreateWithFlags(&evA, evf));
        PCG_CK(cudaEventCreateWithFlags(&evB, evf));
        PCG_CK(cudaEventCreateWithFlags(&evW, evf | cudaEventDisableTiming));
        cap_rows = std::max(std::max(n, m2), std::max(m1, 512)) + 64;   // >= every partials grid
        const char* v = std::getenv("PCGIPM_VERBOSE");
        verbose = v && v[0] == '1';
        const char* pt = std::getenv("PCGIPM_PHASE_TIMES");
        phase_times = pt && pt[0] == '1';
        const char* le = std::getenv("PCGIPM_TEST_LEAVE_EARLY");
        leave_early = le && le[0] == '1';
        allow_pc64 = opt.mixed_fallback != 0;
    }

    template <typename TO>
    void destroy_graphs(Op<TO>& o) {
        for (auto& g : o.graph)
            if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    }

    ~Engine() {
        if (tc_scr) cudaFreeAsync(tc_scr, s);
        destroy_graphs(o32);
        destroy_graphs(o64);
        if (hst) cudaFreeHost(hst);
        if (h_scal) cudaFreeHost(h_scal);
        if (h_info) cudaFreeHost(h_info);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        cudaEventDestroy(evA);
        cudaEventDestroy(evB);
        cudaEventDestroy(evW);
        arena.release();
        cudaStreamSynchronize(s);
        if (own_stream) cudaStreamDestroy(s);
    }

    template <typename X>
    X* vec(int len) { return arena.alloc<X>((size_t)pad_ld(len > 0 ? len : 1)); }

    // Upper bound on the device bytes a handle of these sizes holds at any time:
    // every arena allocation below plus the setup scratch (the factor's working
    // copies, the C R^{-1} product of T), counted at their padded sizes with the
    // arena's 256-byte slack, for each precision and preconditioner the options
    // allow the solve to reach (FP32 may move to FP64; AUTO may move to P_H).
    // QP_FORM_AUTO with a dense C: the low-rank form (K_F = D + V V', V = C Z,
    // M0 = Z Z') when V streams at most half the elements of C', M0 and C
    // (2 m2 r <= (2 m2 n + n^2) / 2, r = n - m1) and r <= 1024 (Z costs r steps of a
    // pivoted Cholesky, one grid barrier each, once per QP); otherwise the M0 form.
    // With C in CSR the M0 form (its C products are sparse row sums; V would be dense).
    static int resolve_form(int form, int n, int m1, int m2, bool csr) {
        if (form != QP_FORM_AUTO) return form;
        const double r = n - m1;
        const double lowrank = 2.0 * m2 * r, m0form = 2.0 * m2 * n + (double)n * n;
        return (!csr && r >= 1 && r <= 1024 && lowrank <= 0.5 * m0form) ? 3 : 0;
    }

    static size_t bytes_bound(int n, int m1, int m2, const qp_opts& oin) {
        qp_opts o = oin;
        o.pcg_form = resolve_form(o.pcg_form, n, m1, m2, false);   // (a CSR handle never holds more)
        auto mat = [](int r, int c, size_t es) {
            return (size_t)std::max(r, 1) * (size_t)pad_ld(std::max(c, 1)) * es + 256;
        };
        auto v = [](int len, size_t es) { return (size_t)pad_ld(std::max(len, 1)) * es + 256; };
        const int cap = std::max(std::max(n, m2), std::max(m1, 512)) + 64;
        size_t b = 0;
        // FP64 problem copies, IPM / refinement vectors, partials, staging, scalars
        b += mat(n, n, 8) + mat(m1, n, 8) + mat(n, m1, 8) + mat(m2, n, 8) + mat(n, m2, 8);
        b += 64 * v(cap, 8) + 4096;
        auto op = [&](size_t es, bool copyC) {
            size_t t = 32 * v(cap, es) + 2 * v(n + m1, es);
            if (copyC) t += mat(m2, n, es) + mat(n, m2, es);
            t += 2 * mat(n, n, es);
            if (o.pcg_form == 0 || o.pcg_form == 3) t += mat(n, n, es);   // M0
            if (o.pcg_form == 3) t += mat(m2, std::max(n - m1, 1), es) + mat(std::max(n - m1, 1), m2, es) + mat(n - m1 + 1, n, es) + v(n, es);
            if (m1) t += 2 * mat(m1, m1, es) + 2 * mat(m1, n, es) + 2 * mat(n, m1, es);
            if (o.pcg_form == 1) t += mat(n + m1, m2, es) + mat(m2, n + m1, es);
            t += mat(n, n, es) + 2 * mat(m1, n, es) + mat(m1, m1, es);   // factor scratch
            return t;
        };
        auto pc = [&](size_t es) {
            size_t t = 4 * mat(m2, m2, es) + 6 * v(m2, es) + mat(m2, n, es);
            if (es == 4) t += mat(m2, m2, es) + tc_scratch_floats(n, m2) * 4 + 1024;   // P~^{-1}, tensor-core scratch
            return t;
        };
        const bool fp32 = (o.precision == QP_PREC_FP32);
        const bool ph = o.precond != QP_PC_PL && o.precond != QP_PC_NONE;
        b += (size_t)kMaxPhases * kTblStride * 8 + 256 + (128 + 8 * 1024) * 8 + 256;
        b += op(8, false);                       // the factor is formed in FP64
        if (o.factor_bk && (o.pcg_form == 0 || o.pcg_form == 3))   // K0 in full, Z and D^{-1} Z, pivot data
            b += mat(n + m1, n + m1, 8) + 2 * mat(n + m1, n, 8) + 8 * v(n + m1, 8) + 8 * v(2048, 8);
        if (fp32) {
            b += op(4, true);
            if (ph) b += pc(4) + (o.mixed_fallback ? pc(8) : 0);
        } else {
            if (ph) b += pc(8);
        }
        return b;
    }

    // Wait for the solver stream (spinning, or yielding with blocking_wait).
    void wait_stream() {
        if (opt.blocking_wait) {
            PCG_CK(cudaEventRecord(evW, s));
            PCG_CK(cudaEventSynchronize(evW));
        } else {
            PCG_CK(cudaStreamSynchronize(s));
        }
    }

    void sync_check() {
        wait_stream();
        PCG_CK(cudaGetLastError());
    }

    // ------------------------------------------------------------------ create
    // C is dense (Ch) or CSR (csr != null; C arrives zeroed from the arena and the
    // pattern is expanded into it on the device).
    struct CsrIn {
        const int* rowptr;
        const int* colidx;
        const double* val;
    };
    void load(const double* Hh, const double* ch, const double* Ah, const double* bh, const double* Ch,
              const double* dh, int ptr_kind, const CsrIn* csr = nullptr) {
        const cudaMemcpyKind kind = (ptr_kind == QP_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        H.alloc(arena, n, n);
        A.alloc(arena, m1, n);
        AT.alloc(arena, n, m1);
        C.alloc(arena, m2, n);
        CT.alloc(arena, n, m2);
        c = vec<double>(n); b = vec<double>(m1); d = vec<double>(m2);
        PCG_CK(cudaMemcpy2DAsync(H.p, H.ld * 8, Hh, (size_t)n * 8, (size_t)n * 8, n, kind, s));
        if (m1) PCG_CK(cudaMemcpy2DAsync(A.p, A.ld * 8, Ah, (size_t)n * 8, (size_t)n * 8, m1, kind, s));
        int* csr_bad = nullptr;
        if (csr) {
            int last = 0;
            if (ptr_kind == QP_PTR_HOST) {
                last = csr->rowptr[m2];
            } else {
                PCG_CK(cudaMemcpyAsync(&last, csr->rowptr + m2, sizeof(int), cudaMemcpyDeviceToHost, s));
                wait_stream();
            }
            if (last < 0) throw QpError{QP_EINVAL};
            const long long nnz = last;
            csr_bad = arena.alloc<int>(1);
            const int* rp = csr->rowptr;
            const int* ci = csr->colidx;
            const double* cv = csr->val;
            void* tmp = nullptr;
            if (ptr_kind == QP_PTR_HOST) {
                const size_t bytes = (size_t)(m2 + 1) * 4 + (size_t)nnz * 4 + (size_t)nnz * 8 + 64;
                if (cudaMallocAsync(&tmp, bytes, s) != cudaSuccess) { cudaGetLastError(); throw NoMem{}; }
                char* t = static_cast<char*>(tmp);
                double* dv = reinterpret_cast<double*>(t);
                int* dr = reinterpret_cast<int*>(t + (size_t)nnz * 8);
                int* dc = dr + (m2 + 1);
                if (nnz) PCG_CK(cudaMemcpyAsync(dv, cv, (size_t)nnz * 8, kind, s));
                PCG_CK(cudaMemcpyAsync(dr, rp, (size_t)(m2 + 1) * 4, kind, s));
                if (nnz) PCG_CK(cudaMemcpyAsync(dc, ci, (size_t)nnz * 4, kind, s));
                rp = dr; ci = dc; cv = dv;
            }
            csr_scatter_kernel<<<(m2 + 255) / 256, 256, 0, s>>>(m2, n, nnz, rp, ci, cv, C.p, C.ld, csr_bad);
            // host copies for the C' pattern (built once the pattern is checked)
            h_rp.resize(m2 + 1);
            h_ci.resize(nnz);
            h_cv.resize(nnz);
            const cudaMemcpyKind back = (ptr_kind == QP_PTR_DEVICE || tmp) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
            PCG_CK(cudaMemcpyAsync(h_rp.data(), rp, (size_t)(m2 + 1) * 4, back, s));
            if (nnz) PCG_CK(cudaMemcpyAsync(h_ci.data(), ci, (size_t)nnz * 4, back, s));
            if (nnz) PCG_CK(cudaMemcpyAsync(h_cv.data(), cv, (size_t)nnz * 8, back, s));
            wait_stream();
            if (tmp) cudaFreeAsync(tmp, s);
        } else {
            PCG_CK(cudaMemcpy2DAsync(C.p, C.ld * 8, Ch, (size_t)n * 8, (size_t)n * 8, m2, kind, s));
        }
        PCG_CK(cudaMemcpyAsync(c, ch, (size_t)n * 8, kind, s));
        if (m1) PCG_CK(cudaMemcpyAsync(b, bh, (size_t)m1 * 8, kind, s));
        PCG_CK(cudaMemcpyAsync(d, dh, (size_t)m2 * 8, kind, s));
        transpose<double>(A.p, A.ld, AT.p, AT.ld, m1, n, s);
        transpose<double>(C.p, C.ld, CT.p, CT.ld, m2, n, s);

        part_pq = vec<double>(cap_rows); part_rr = vec<double>(cap_rows); part_rz = vec<double>(cap_rows);
        part_bb = vec<double>(cap_rows); part_a = vec<double>(cap_rows); part_b = vec<double>(cap_rows);
        part_c = vec<double>(cap_rows); part_d = vec<double>(cap_rows); part_e = vec<double>(cap_rows);
        part_f = vec<double>(cap_rows); diag0 = vec<double>(cap_rows);
        st = arena.alloc<PcgState>(1);
        bar = arena.alloc<GridBar>(1);
        tstamp = arena.alloc<unsigned long long>(128 + 8 * 1024 + 3 * kTrace);
        d_tcerr = arena.alloc<int>(1);
        d_tbl = arena.alloc<int2>((size_t)kMaxPhases * kTblStride);
        d_scal = vec<double>(16);
        d_info = arena.alloc<int>(8);
        PCG_CK(cudaMallocHost(&hst, 2 * sizeof(PcgState)));
        PCG_CK(cudaMallocHost(&h_scal, 16 * sizeof(double)));
        PCG_CK(cudaMallocHost(&h_info, 8 * sizeof(int)));
        for (auto& p : stage) p = vec<double>(cap_rows);

        // validation: finiteness and symmetry of H
        PCG_CK(cudaMemsetAsync(d_info, 0, 8 * sizeof(int), s));
        nonfinite_kernel<<<304, 256, 0, s>>>((long long)n * H.ld, H.p, d_info);
        if (m1) nonfinite_kernel<<<304, 256, 0, s>>>((long long)m1 * A.ld, A.p, d_info);
        nonfinite_kernel<<<304, 256, 0, s>>>((long long)m2 * C.ld, C.p, d_info);
        nonfinite_kernel<<<64, 256, 0, s>>>(n, c, d_info);
        if (m1) nonfinite_kernel<<<64, 256, 0, s>>>(m1, b, d_info);
        nonfinite_kernel<<<64, 256, 0, s>>>(m2, d, d_info);
        asym_kernel<<<304, 256, 0, s>>>(n, H.p, H.ld, reinterpret_cast<unsigned int*>(d_info + 1));
        // norms used by the stopping rule
        absrowsum_max_kernel<<<152, 256, 0, s>>>(n, H.p, H.ld, part_a);
        norms_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, c, part_b, part_c);
        norms_kernel<<<vec_grid(std::max(m1, 1)), kVecThreads, 0, s>>>(m1, b, part_b, part_d);
        norms_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, d, part_b, part_e);
        ReduceJob job{};
        job.part[0] = part_a; job.cnt[0] = 152; job.op[0] = 1;
        job.part[1] = part_c; job.cnt[1] = vec_grid(n); job.op[1] = 1;
        job.part[2] = part_d; job.cnt[2] = vec_grid(std::max(m1, 1)); job.op[2] = 1;
        job.part[3] = part_e; job.cnt[3] = vec_grid(m2); job.op[3] = 1;
        job.njobs = 4;
        reduce_jobs_kernel<<<1, kVecThreads, 0, s>>>(job, d_scal);
        PCG_CK(cudaMemcpyAsync(h_scal, d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaMemcpyAsync(h_info, d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        if (csr_bad) PCG_CK(cudaMemcpyAsync(h_info + 2, csr_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        else h_info[2] = 0;
        sync_check();
        if (h_info[2] != 0) throw QpError{QP_EINVAL};
        if (csr) upload_csr();
        h_norm_inf = h_scal[0]; c_inf = h_scal[1]; b_inf = m1 ? h_scal[2] : 0.0; d_inf = h_scal[3];
        float asym;
        std::memcpy(&asym, &h_info[1], sizeof(float));
        if (h_info[0] != 0 || !(asym <= 1e-12f)) throw QpError{QP_EINVAL};

        // IPM vectors
        x = vec<double>(n); lam = vec<double>(m1); nu = vec<double>(m2); sl = vec<double>(m2);
        hx = vec<double>(n); rg = vec<double>(n); re = vec<double>(m1); ri = vec<double>(m2);
        rc = vec<double>(m2); ra = vec<double>(m2); D64 = vec<double>(m2);
        dx = vec<double>(n); dl = vec<double>(m1); dn = vec<double>(m2); ds = vec<double>(m2);
        dxa = vec<double>(n); dla = vec<double>(m1); dna = vec<double>(m2); dsa = vec<double>(m2);
        fg = vec<double>(n); fe = vec<double>(m1); fa = vec<double>(m2);
        rho_g = vec<double>(n); rho_e = vec<double>(m1); rho_a = vec<double>(m2);
        tx = vec<double>(n); tl = vec<double>(m1); tn = vec<double>(m2);
        sync_check();
    }

    // C and C' in CSR form on the device (the pattern is checked; C' by a counting
    // sort on the host: each column's entries in increasing row order).
    std::vector<int> h_rp, h_ci;
    std::vector<double> h_cv;
    void upload_csr() {
        nnz = (long long)h_ci.size();
        std::vector<int> trp(n + 1, 0), tci(nnz);
        std::vector<double> tv(nnz);
        for (long long k = 0; k < nnz; ++k) ++trp[h_ci[k] + 1];
        for (int j = 0; j < n; ++j) trp[j + 1] += trp[j];
        std::vector<int> fill(trp.begin(), trp.end() - 1);
        for (int i = 0; i < m2; ++i)
            for (int k = h_rp[i]; k < h_rp[i + 1]; ++k) {
                const int pos = fill[h_ci[k]]++;
                tci[pos] = i;
                tv[pos] = h_cv[k];
            }
        const size_t nz = (size_t)std::max(nnz, 1LL);
        crp = arena.alloc<int>(m2 + 1); cci = arena.alloc<int>(nz);
        ctrp = arena.alloc<int>(n + 1); ctci = arena.alloc<int>(nz);
        cval64 = arena.alloc<double>(nz); ctval64 = arena.alloc<double>(nz);
        PCG_CK(cudaMemcpyAsync(crp, h_rp.data(), (size_t)(m2 + 1) * 4, cudaMemcpyHostToDevice, s));
        PCG_CK(cudaMemcpyAsync(ctrp, trp.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s));
        if (nnz) {
            PCG_CK(cudaMemcpyAsync(cci, h_ci.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
            PCG_CK(cudaMemcpyAsync(ctci, tci.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
            PCG_CK(cudaMemcpyAsync(cval64, h_cv.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice, s));
            PCG_CK(cudaMemcpyAsync(ctval64, tv.data(), (size_t)nnz * 8, cudaMemcpyHostToDevice, s));
        }
        wait_stream();   // the host vectors go away below
        h_rp.clear(); h_ci.clear(); h_cv.clear();
        h_rp.shrink_to_fit(); h_ci.shrink_to_fit(); h_cv.shrink_to_fit();
    }

    // ------------------------------------------------------------------ factor
    // Setup phase (Sec. 4.1): K0 = [H A'; A 0] = L diag(I, -I) L' with
    // L = [R' 0; G L_S], R'R = H, G = A R^{-1}, L_S L_S' = G G' = A H^{-1} A'.
    // The factor is always formed in FP64 (pivots, triangular inverses and every
    // product); the FP32 operator holds its entries rounded once.  A pivot below
    // 1e-13 of the original diagonal entry means H is not positive definite
    // (QP_ENOTCONVEX) or A H^{-1} A' is singular (QP_ESINGULAR); pivots below
    // 1e-6 (FP32 resolution) are recorded in fp32_pivot_warn.
    // Also formed once per QP: M0 = [K0^{-1}]_11 = R^{-1} R^{-T} - Et' Et (the
    // persistent kernel's K0 solve, pcg_form 0) and, for pcg_form 1,
    // B = L^{-1}[C'; 0].
    template <typename TO>
    void alloc_op_vectors(Op<TO>& o) {
        o.px = vec<TO>(m2); o.pr = vec<TO>(m2); o.pz = vec<TO>(m2); o.pp = vec<TO>(m2); o.pq = vec<TO>(m2);
        o.pu = vec<TO>(n); o.pz1 = vec<TO>(n); o.pz2 = vec<TO>(m1); o.pt = vec<TO>(n); o.py = vec<TO>(n);
        o.prhs = vec<TO>(m2); o.pD = vec<TO>(m2); o.pDinv = vec<TO>(m2);
        if (std::is_same<TO, double>::value) {
            o.zb = vec<TO>(m2);
            o.segp = vec<double>(2 * ((m2 + kSeg - 1) / kSeg));
        }
        o.ku = vec<TO>(n); o.kw = vec<TO>(m1); o.ke = vec<TO>(m1); o.kz1 = vec<TO>(n); o.kz2 = vec<TO>(m1);
        o.kt = vec<TO>(n); o.ka = vec<TO>(n); o.kmb = vec<TO>(m1); o.wa = vec<TO>(m2); o.wg = vec<TO>(n);
        o.oU = vec<TO>(n); o.oY = vec<TO>(n); o.oZ = vec<TO>(n + m1); o.oW = vec<TO>(m2);
        if (opt.pcg_form == 1) {
            o.BW.alloc(arena, n + m1, m2);
            o.BWT.alloc(arena, m2, n + m1);
        }
        o.WH.alloc(arena, n, n);
        o.WHT.alloc(arena, n, n);
        if (opt.pcg_form == 0 || opt.pcg_form == 3) o.M0.alloc(arena, n, n);
        if (opt.pcg_form == 3) {
            o.lr = n - m1;
            o.LV.alloc(arena, m2, std::max(o.lr, 1));
            o.LVT.alloc(arena, std::max(o.lr, 1), m2);
        }
        if (m1) {
            o.WS.alloc(arena, m1, m1); o.WST.alloc(arena, m1, m1);
            o.Gt.alloc(arena, m1, n); o.GtT.alloc(arena, n, m1);
            o.Et.alloc(arena, m1, n); o.EtT.alloc(arena, n, m1);
        }
    }

    bool fp32_pivot_warn = false;

    // Bunch-Kaufman LDL' of K0 (qp_opts.factor_bk): inertia check and M0 = Z' D^{-1} Z.
    void bk_m0(double* M0, long long ldm0) {
        const int N = n + m1;
        const long long ldk = pad_ld(N), ldz = pad_ld(n);
        double *K = nullptr, *Z = nullptr, *Y = nullptr, *aux = nullptr;
        auto galloc = [&](double** p, size_t count) {
            if (cudaMallocAsync(p, count * sizeof(double) + 256, s) != cudaSuccess) {
                cudaGetLastError();
                if (K) cudaFreeAsync(K, s);
                if (Z) cudaFreeAsync(Z, s);
                if (Y) cudaFreeAsync(Y, s);
                throw NoMem{};
            }
        };
        galloc(&K, (size_t)N * ldk);
        galloc(&Z, (size_t)N * ldz);
        galloc(&Y, (size_t)N * ldz);
        galloc(&aux, (size_t)6 * ldk + 4096 + 64);
        double* w = aux;                                   // 2 N
        double* d = aux + 2 * ldk;                         // N
        double* e = aux + 3 * ldk;                         // N
        int* perm = reinterpret_cast<int*>(aux + 4 * ldk);                 // N ints
        int* ptype = reinterpret_cast<int*>(aux + 5 * ldk);                // N ints
        double* cval = aux + 6 * ldk;                      // 2 x 1024
        int* cidx = reinterpret_cast<int*>(cval + 2048);   // 2 x 1024 ints
        unsigned* pbar = reinterpret_cast<unsigned*>(cidx + 2048);
        int* perr = reinterpret_cast<int*>(pbar + 4);
        int* pstat = perr + 1;
        PCG_CK(cudaMemsetAsync(pbar, 0, 32, s));
        bk_build_k0_kernel<<<vec_grid(N), kVecThreads, 0, s>>>(H.p, H.ld, A.p, A.ld, n, m1, K, ldk, perm);
        int dev = 0, sms = 0;
        PCG_CK(cudaGetDevice(&dev));
        PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int G = std::max(1, std::min(std::min(sms, 1024), N / 16));
        BkArgs ba{K, ldk, N, w, cval, cidx, perm, d, e, ptype, pbar, perr, pstat};
        void* args[] = {(void*)&ba};
        PCG_CK(cudaLaunchCooperativeKernel((const void*)bk_factor_kernel, G, kBkThreads, args, 0, s));
        std::vector<double> hd(N), he(N);
        std::vector<int> ht(N);
        int flags[2] = {0, 0};
        PCG_CK(cudaMemcpyAsync(flags, perr, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaMemcpyAsync(hd.data(), d, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaMemcpyAsync(he.data(), e, N * sizeof(double), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaMemcpyAsync(ht.data(), ptype, N * sizeof(int), cudaMemcpyDeviceToHost, s));
        wait_stream();
        PCG_CK(cudaGetLastError());
        auto release = [&]() { cudaFreeAsync(K, s); cudaFreeAsync(Z, s); cudaFreeAsync(Y, s); cudaFreeAsync(aux, s); };
        if (flags[0]) { release(); throw QpError{QP_ETIMEOUT}; }
        if (flags[1]) { release(); throw QpError{QP_ESINGULAR}; }
        // inertia of D (Sylvester): 1x1 blocks by sign; a 2x2 block with det < 0 has one of each
        int pos = 0, neg = 0, two = 0;
        for (int i = 0; i < N; ++i) {
            if (ht[i] == 1) {
                (hd[i] > 0 ? pos : neg) += 1;
            } else if (ht[i] == 2) {
                const double det = hd[i] * hd[i + 1] - he[i] * he[i];
                ++two;
                if (det < 0) { ++pos; ++neg; }
                else if (hd[i] > 0) pos += 2;
                else neg += 2;
            }
        }
        stats.k0_inertia_pos = pos;
        stats.k0_inertia_neg = neg;
        stats.k0_pivots_2x2 = two;
        if (pos != n || neg != m1) {
            if (verbose) std::fprintf(stderr, "  K0 inertia (%d, %d), expected (%d, %d)\n", pos, neg, n, m1);
            release();
            throw QpError{QP_ENOTCONVEX};
        }
        // Z = L^{-1} P [I_n; 0] by 64-row blocks, Y = D^{-1} Z, M0 = Z' Y
        const long long total = (long long)N * ldz;
        bk_pe_kernel<<<(int)std::min<long long>((total + 255) / 256, 152LL * 16), 256, 0, s>>>(perm, N, n, Z, ldz);
        for (int k0 = 0; k0 < N; k0 += kBkRows) {
            const int kb = std::min(kBkRows, N - k0);
            if (k0 > 0) {
                GemmArgs<double> g{};
                g.M = kb; g.N = n; g.K = k0;
                g.A = K + (long long)k0 * ldk; g.sai = ldk; g.sak = 1;
                g.B = Z; g.sbk = ldz; g.sbj = 1;
                g.C = Z + (long long)k0 * ldz; g.ldc = ldz; g.alpha = -1.0; g.beta = 1.0;
                gemm<double>(g, s);
            }
            bk_trsm_block_kernel<<<(n + 127) / 128, 128, 0, s>>>(K, ldk, k0, kb, Z, ldz, n);
        }
        bk_dinv_kernel<<<(int)std::min<long long>(((long long)N * n + 255) / 256, 152LL * 16), 256, 0, s>>>(
            d, e, ptype, N, n, Z, Y, ldz);
        GemmArgs<double> h{};
        h.M = n; h.N = n; h.K = N;
        h.A = Z; h.sai = 1; h.sak = ldz;
        h.B = Y; h.sbk = ldz; h.sbj = 1;
        h.C = M0; h.ldc = ldm0; h.alpha = 1.0; h.beta = 0.0;
        gemm<double>(h, s);
        release();
        wait_stream();
        PCG_CK(cudaGetLastError());
    }
    bool form_auto = false;   // pcg_form was QP_FORM_AUTO

    // Scratch of the tensor-core products (TF32 hi/lo splits of their operands),
    // grown on demand and released with the handle.
    float* tc_scr = nullptr;
    size_t tc_cap = 0;
    int* d_tcerr = nullptr;
    float* tc_scratch(size_t floats) {
        if (floats > tc_cap) {
            if (tc_scr) cudaFreeAsync(tc_scr, s);
            tc_scr = nullptr;
            tc_cap = 0;
            if (cudaMallocAsync(&tc_scr, floats * sizeof(float) + 1024, s) != cudaSuccess) {
                cudaGetLastError();
                throw NoMem{};
            }
            tc_cap = floats;
        }
        return tc_scr;
    }
    void tc_check() {
        int e = 0;
        PCG_CK(cudaMemcpyAsync(&e, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
        wait_stream();
        if (e) throw QpError{QP_ETIMEOUT};
    }
    // Floats of tensor-core scratch of the FP32 P_H path: T's operands
    // (C and R^{-1}, then C R^{-1}), P~^{-1}'s operand W', and the blocked Cholesky.
    static size_t tc_scratch_floats(int n, int m2) {
        const size_t ldn = pad_ld(n), ldm = pad_ld(m2);
        const size_t t = 2 * (size_t)m2 * ldn + 2 * (size_t)n * ldn;
        const size_t pi = 2 * (size_t)m2 * ldm;
        return std::max(std::max(t, pi), chol_tc_scratch(m2));
    }

    // The FP32 operator's factor formed in FP32 storage with the dense contractions on
    // the tensor cores (FP32-accurate 3xTF32 splits) and FP64 pivots on the diagonal
    // blocks: H = R'R with its inverse (blocked, the trailing and inverse updates on
    // tcgen05), G = A R^{-1}, S = G G', L_S and its inverse, Gt = L_S^{-1} G,
    // Et = Gt R^{-T}, and M0 = R^{-1}R^{-T} - Et'Et.  Returns false (nothing kept) if a
    // pivot falls below FP32 resolution (1e-6 of its original diagonal entry) or a
    // tensor map cannot be made; the caller then rounds the FP64 factor instead.
    bool factor_tc32() {
        Op<float>& o = o32;
        const long long ldn = pad_ld(n), ldm = pad_ld(std::max(m1, 1));
        const double rel = 1e-6;
        chol_inv_prepare<float, double>();
        float *Hw = nullptr, *Aw = nullptr, *G = nullptr, *GT = nullptr, *S = nullptr;
        auto galloc = [&](float** p, size_t count) {
            if (cudaMallocAsync(p, count * sizeof(float) + 256, s) != cudaSuccess) { cudaGetLastError(); throw NoMem{}; }
            PCG_CK(cudaMemsetAsync(*p, 0, count * sizeof(float) + 256, s));
        };
        // scratch: hi/lo splits of two operands of up to n x ldn, and the blocked Cholesky
        float* sc = tc_scratch(std::max<size_t>(4 * (size_t)n * (size_t)ldn, chol_tc_scratch(n)));
        float *ah = sc, *al = ah + (size_t)n * ldn, *bh = al + (size_t)n * ldn, *bl = bh + (size_t)n * ldn;
        bool ok = true;
        auto split = [&](const float* x, long long ldx, int rows, int cols, float* hi, float* lo) {
            tc_split(x, ldx, rows, cols, hi, lo, ldx, s);
        };
        // C = alpha X Y' + beta C with X (M x K), Y (N x K) K-major, both split first
        auto tcmm = [&](int M, int N, int K, float alpha, const float* X, long long ldx, const float* Y, long long ldy,
                        float beta, float* Cm, long long ldc, bool lower) {
            if (!ok || M <= 0 || N <= 0) return;
            split(X, ldx, M, K, ah, al);
            split(Y, ldy, N, K, bh, bl);
            ok = tc_gemm(M, N, K, alpha, ah, al, ldx, bh, bl, ldy, beta, Cm, ldc, true, lower, d_tcerr, s);
            if (!ok) cudaGetLastError();
        };
        PCG_CK(cudaMemsetAsync(d_tcerr, 0, sizeof(int), s));
        PCG_CK(cudaMemsetAsync(d_info, 0, 8 * sizeof(int), s));
        galloc(&Hw, (size_t)n * ldn);
        PCG_CK(cudaMemsetAsync(o.WH.p, 0, (size_t)n * o.WH.ld * sizeof(float), s));
        convert2d<double, float>(H.p, H.ld, Hw, ldn, n, n, s);
        chol_inv_tc<double>(Hw, ldn, o.WH.p, o.WH.ld, n, 0, rel, d_info, s, tc_scratch(0), d_tcerr, diag0);
        transpose<float>(o.WH.p, o.WH.ld, o.WHT.p, o.WHT.ld, n, n, s);
        if (m1) {
            galloc(&Aw, (size_t)m1 * ldn);
            galloc(&G, (size_t)m1 * ldn);
            galloc(&GT, (size_t)n * ldm);
            galloc(&S, (size_t)m1 * ldm);
            PCG_CK(cudaMemsetAsync(o.WS.p, 0, (size_t)m1 * o.WS.ld * sizeof(float), s));
            convert2d<double, float>(A.p, A.ld, Aw, ldn, m1, n, s);
            tcmm(m1, n, n, 1.0f, Aw, ldn, o.WH.p, o.WH.ld, 0.0f, G, ldn, false);        // G = A R^{-1} = A WH'
            tcmm(m1, m1, n, 1.0f, G, ldn, G, ldn, 0.0f, S, ldm, true);                  // S = G G' (lower)
            if (ok) chol_inv_tc<double>(S, ldm, o.WS.p, o.WS.ld, m1, 0, rel, d_info + 2, s, tc_scratch(0), d_tcerr, diag0);
            transpose<float>(G, ldn, GT, ldm, m1, n, s);
            tcmm(m1, n, m1, 1.0f, o.WS.p, o.WS.ld, GT, ldm, 0.0f, o.Gt.p, o.Gt.ld, false);   // Gt = L_S^{-1} G
            transpose<float>(o.Gt.p, o.Gt.ld, o.GtT.p, o.GtT.ld, m1, n, s);
            transpose<float>(o.WS.p, o.WS.ld, o.WST.p, o.WST.ld, m1, m1, s);
            tcmm(m1, n, n, 1.0f, o.Gt.p, o.Gt.ld, o.WHT.p, o.WHT.ld, 0.0f, o.Et.p, o.Et.ld, false);   // Et = Gt WH
            transpose<float>(o.Et.p, o.Et.ld, o.EtT.p, o.EtT.ld, m1, n, s);
        }
        if (o.M0.p) {
            tcmm(n, n, n, 1.0f, o.WHT.p, o.WHT.ld, o.WHT.p, o.WHT.ld, 0.0f, o.M0.p, o.M0.ld, false);   // R^{-1}R^{-T}
            if (m1) tcmm(n, n, m1, -1.0f, o.EtT.p, o.EtT.ld, o.EtT.p, o.EtT.ld, 1.0f, o.M0.p, o.M0.ld, false);
        }
        convert2d<double, float>(C.p, C.ld, o.CW.p, o.CW.ld, m2, n, s);
        convert2d<double, float>(CT.p, CT.ld, o.CWT.p, o.CWT.ld, n, m2, s);
        if (crp && !o.cval) {
            float* v = arena.alloc<float>((size_t)std::max(nnz, 1LL));
            float* vt = arena.alloc<float>((size_t)std::max(nnz, 1LL));
            convert1d<double, float>((int)nnz, cval64, 1.0, v, s);
            convert1d<double, float>((int)nnz, ctval64, 1.0, vt, s);
            o.cval = v;
            o.ctval = vt;
        }
        PCG_CK(cudaMemcpyAsync(h_info, d_info, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        cudaFreeAsync(Hw, s);
        if (Aw) cudaFreeAsync(Aw, s);
        if (G) cudaFreeAsync(G, s);
        if (GT) cudaFreeAsync(GT, s);
        if (S) cudaFreeAsync(S, s);
        wait_stream();
        PCG_CK(cudaGetLastError());
        tc_check();
        if (!ok || h_info[0] != 0 || h_info[2] != 0) {
            if (verbose) std::fprintf(stderr, "  tensor-core FP32 factor declined (tc %d, pivots %d %d): FP64 factor\n",
                                      (int)ok, h_info[0], h_info[2]);
            return false;
        }
        stats.factor_tc = 1;
        return true;
    }

    template <typename TO>
    void factor_op() {
        Op<TO>& o = op<TO>();
        if (o.factored) return;
        constexpr bool is64 = std::is_same<TO, double>::value;
        if constexpr (!is64) {
            if (!o.px) {
                alloc_op_vectors(o);
                o.CW.alloc(arena, m2, n);
                o.CWT.alloc(arena, n, m2);
            }
            // qp_opts.factor_tc: the FP32 factor itself on the tensor cores (forms 0 and 2)
            if (opt.factor_tc && (opt.pcg_form == 0 || opt.pcg_form == 2) && factor_tc32()) {
                o.factored = true;
                return;
            }
            // FP32 operator: the FP64 factor rounded once (an FP32 factorization would
            // add about cond(R) u32 to every entry; rounding adds u32 of the entry)
            factor_op<double>();
            convert2d<double, TO>(C.p, C.ld, o.CW.p, o.CW.ld, m2, n, s);
            convert2d<double, TO>(CT.p, CT.ld, o.CWT.p, o.CWT.ld, n, m2, s);
            auto rnd = [&](const Mat<double>& a, Mat<TO>& b) {
                if (a.p && b.p) convert2d<double, TO>(a.p, a.ld, b.p, b.ld, a.rows, a.cols, s);
            };
            rnd(o64.WH, o.WH); rnd(o64.WHT, o.WHT); rnd(o64.M0, o.M0);
            if (opt.pcg_form == 3) {
                o.lr = o64.lr;
                rnd(o64.LV, o.LV);
                rnd(o64.LVT, o.LVT);
            }
            rnd(o64.WS, o.WS); rnd(o64.WST, o.WST); rnd(o64.Gt, o.Gt); rnd(o64.GtT, o.GtT);
            rnd(o64.Et, o.Et); rnd(o64.EtT, o.EtT);
            if (crp && !o.cval) {
                TO* v = arena.alloc<TO>((size_t)std::max(nnz, 1LL));
                TO* vt = arena.alloc<TO>((size_t)std::max(nnz, 1LL));
                convert1d<double, TO>((int)nnz, cval64, 1.0, v, s);
                convert1d<double, TO>((int)nnz, ctval64, 1.0, vt, s);
                o.cval = v;
                o.ctval = vt;
            }
            if (opt.pcg_form == 1) {
                // B is formed from the FP64 factor and rounded once to FP32, so its entries
                // carry only their final rounding
                rnd(o64.BW, o.BW);
                transpose<TO>(o.BW.p, o.BW.ld, o.BWT.p, o.BWT.ld, n + m1, m2, s);
            }
            wait_stream();
            PCG_CK(cudaGetLastError());
            o.factored = true;
            return;
        } else {
        const double rel = 1e-13, warn = 1e-6;
        chol_inv_prepare<TO, double>();
        if (!o.px) {
            alloc_op_vectors(o);
            o.CW.p = C.p; o.CW.rows = m2; o.CW.cols = n; o.CW.ld = C.ld;
            o.CWT.p = CT.p; o.CWT.rows = n; o.CWT.cols = m2; o.CWT.ld = CT.ld;
            o.cval = cval64;
            o.ctval = ctval64;
        }
        // scratch of the factorization (freed at the end)
        TO *Hw = nullptr, *Aw = nullptr, *G = nullptr, *S = nullptr;
        const long long ldn = pad_ld(n), ldm = pad_ld(std::max(m1, 1));
        auto galloc = [&](TO** p, size_t count) {
            if (cudaMallocAsync(p, count * sizeof(TO) + 256, s) != cudaSuccess) { cudaGetLastError(); throw NoMem{}; }
            PCG_CK(cudaMemsetAsync(*p, 0, count * sizeof(TO) + 256, s));
        };
        galloc(&Hw, (size_t)n * ldn);
        PCG_CK(cudaMemsetAsync(o.WH.p, 0, (size_t)n * o.WH.ld * sizeof(TO), s));
        convert2d<double, TO>(H.p, H.ld, Hw, ldn, n, n, s);
        PCG_CK(cudaMemsetAsync(d_info, 0, 8 * sizeof(int), s));
        chol_inv<TO, double>(Hw, ldn, o.WH.p, o.WH.ld, n, 0, rel, d_info, s, diag0, warn, d_info + 1);
        transpose<TO>(o.WH.p, o.WH.ld, o.WHT.p, o.WHT.ld, n, n, s);
        if (m1) {
            galloc(&Aw, (size_t)m1 * ldn);
            galloc(&G, (size_t)m1 * ldn);
            galloc(&S, (size_t)m1 * ldm);
            PCG_CK(cudaMemsetAsync(o.WS.p, 0, (size_t)m1 * o.WS.ld * sizeof(TO), s));
            convert2d<double, TO>(A.p, A.ld, Aw, ldn, m1, n, s);
            GemmArgs<TO> g{};
            // G = A R^{-1} = A WH'   (opB(k,j) = WH[j,k], zero for k > j)
            g.M = m1; g.N = n; g.K = n;
            g.A = Aw; g.sai = ldn; g.sak = 1;
            g.B = o.WH.p; g.sbk = 1; g.sbj = o.WH.ld; g.b_tri = TRI_UPPER;
            g.C = G; g.ldc = ldn; g.alpha = TO(1); g.beta = TO(0);
            gemm<TO>(g, s);
            // S = G G'
            GemmArgs<TO> h{};
            h.M = m1; h.N = m1; h.K = n;
            h.A = G; h.sai = ldn; h.sak = 1;
            h.B = G; h.sbk = 1; h.sbj = ldn;
            h.C = S; h.ldc = ldm; h.alpha = TO(1); h.beta = TO(0); h.lower_out = 1;
            gemm<TO>(h, s);
            chol_inv<TO, double>(S, ldm, o.WS.p, o.WS.ld, m1, 0, rel, d_info + 2, s, diag0, warn, d_info + 3);
            // Gt = L_S^{-1} G
            GemmArgs<TO> k{};
            k.M = m1; k.N = n; k.K = m1;
            k.A = o.WS.p; k.sai = o.WS.ld; k.sak = 1; k.a_tri = TRI_LOWER;
            k.B = G; k.sbk = ldn; k.sbj = 1;
            k.C = o.Gt.p; k.ldc = o.Gt.ld; k.alpha = TO(1); k.beta = TO(0);
            gemm<TO>(k, s);
            transpose<TO>(o.Gt.p, o.Gt.ld, o.GtT.p, o.GtT.ld, m1, n, s);
            transpose<TO>(o.WS.p, o.WS.ld, o.WST.p, o.WST.ld, m1, m1, s);
            // Et = Gt R^{-T}: with it the forward solve with L maps u to [R^{-T} u; -Et u]
            // in one product, and the back solve is y = R^{-1} z1 + Et' z2 (z2 = -Et u)
            GemmArgs<TO> e{};
            e.M = m1; e.N = n; e.K = n;
            e.A = o.Gt.p; e.sai = o.Gt.ld; e.sak = 1;
            e.B = o.WH.p; e.sbk = o.WH.ld; e.sbj = 1; e.b_tri = TRI_LOWER;
            e.C = o.Et.p; e.ldc = o.Et.ld; e.alpha = TO(1); e.beta = TO(0);
            gemm<TO>(e, s);
            transpose<TO>(o.Et.p, o.Et.ld, o.EtT.p, o.EtT.ld, m1, n, s);
        }
        if (o.M0.p) {
            // M0 = R^{-1} R^{-T} - Et' Et = H^{-1} - H^{-1} A' (A H^{-1} A')^{-1} A H^{-1}
            // (opA(i,k) = WH[k,i], zero for k < i; opB(k,j) = WH[k,j], zero for k < j)
            GemmArgs<TO> g{};
            g.M = n; g.N = n; g.K = n;
            g.A = o.WH.p; g.sai = 1; g.sak = o.WH.ld; g.a_tri = TRI_UPPER;
            g.B = o.WH.p; g.sbk = o.WH.ld; g.sbj = 1; g.b_tri = TRI_LOWER;
            g.C = o.M0.p; g.ldc = o.M0.ld; g.alpha = TO(1); g.beta = TO(0);
            gemm<TO>(g, s);
            if (m1) {
                GemmArgs<TO> h{};
                h.M = n; h.N = n; h.K = m1;
                h.A = o.Et.p; h.sai = 1; h.sak = o.Et.ld;
                h.B = o.Et.p; h.sbk = o.Et.ld; h.sbj = 1;
                h.C = o.M0.p; h.ldc = o.M0.ld; h.alpha = TO(-1); h.beta = TO(1);
                gemm<TO>(h, s);
            }
        }
        if (opt.factor_bk && o.M0.p && std::is_same<TO, double>::value) bk_m0(reinterpret_cast<double*>(o.M0.p), o.M0.ld);
        if (opt.pcg_form == 3 && o.lr > 0) {
            // M0 = Z Z' with Z (n x r), r = n - m1 (M0 = R^{-1} (I - P) R^{-T}, P the orthogonal
            // projector onto the row space of A R^{-1}, of rank m1): pivoted Cholesky, then
            // V' = Z' C' (r x m2) and V = C Z, so K_F = D + V V' (Sec. 4.3, Lemma 2)
            const int r = o.lr;
            TO *Zt = nullptr, *dd = nullptr;
            galloc(&Zt, (size_t)r * ldn);
            galloc(&dd, (size_t)n + 2 * 1024 + 64);   // d, then the per-CTA candidates and the barrier words
            int dev = 0, sms = 0, per_sm = 0;
            PCG_CK(cudaGetDevice(&dev));
            PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            PCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pivoted_chol_grid_kernel, 256, 0));
            int G = std::min(std::min(sms * std::max(per_sm, 1), 1024), std::max(1, n / 16));
            double* cval = dd + n;
            int* cidx = reinterpret_cast<int*>(cval + 1024);
            unsigned* pbar = reinterpret_cast<unsigned*>(cidx + 1024);
            int* perr = reinterpret_cast<int*>(pbar + 4);
            PCG_CK(cudaMemsetAsync(pbar, 0, 32, s));
            const double* M0p = o.M0.p;
            long long ldm0 = o.M0.ld, ldz = ldn;
            double rel_floor = 1e-13;
            int* rank_out = d_info + 5;
            void* args[] = {(void*)&M0p, (void*)&ldm0, (void*)&n, (void*)&r, (void*)&Zt, (void*)&ldz, (void*)&dd,
                            (void*)&cval, (void*)&cidx, (void*)&pbar, (void*)&rel_floor, (void*)&rank_out, (void*)&perr};
            PCG_CK(cudaLaunchCooperativeKernel((const void*)pivoted_chol_grid_kernel, G, 256, args, 0, s));
            GemmArgs<TO> g{};
            g.M = r; g.N = m2; g.K = n;
            g.A = Zt; g.sai = ldn; g.sak = 1;
            g.B = C.p; g.sbk = 1; g.sbj = C.ld;
            g.C = o.LVT.p; g.ldc = o.LVT.ld; g.alpha = TO(1); g.beta = TO(0);
            gemm<TO>(g, s);
            transpose<TO>(o.LVT.p, o.LVT.ld, o.LV.p, o.LV.ld, r, m2, s);
            PCG_CK(cudaMemcpyAsync(h_info + 5, d_info + 5, sizeof(int), cudaMemcpyDeviceToHost, s));
            cudaFreeAsync(Zt, s);
            cudaFreeAsync(dd, s);
            wait_stream();
            if (h_info[5] != r) {
                if (verbose) std::fprintf(stderr, "  low-rank form: M0 has rank %d, expected %d\n", h_info[5], r);
                if (!form_auto) throw QpError{QP_ESINGULAR};
                opt.pcg_form = 0;            // chosen by QP_FORM_AUTO: the M0 form (M0 is held)
                stats.pcg_form_used = 0;
            }
        }
        if (opt.pcg_form == 1) {
            // B = L^{-1}[C'; 0]: B1 = R^{-T} C' (n x m2), B2 = Et C' (m1 x m2), and B'
            GemmArgs<TO> b1{};
            b1.M = n; b1.N = m2; b1.K = n;
            b1.A = o.WH.p; b1.sai = o.WH.ld; b1.sak = 1; b1.a_tri = TRI_LOWER;
            b1.B = o.CWT.p; b1.sbk = o.CWT.ld; b1.sbj = 1;
            b1.C = o.BW.p; b1.ldc = o.BW.ld; b1.alpha = TO(1); b1.beta = TO(0);
            gemm<TO>(b1, s);
            if (m1) {
                GemmArgs<TO> b2{};
                b2.M = m1; b2.N = m2; b2.K = n;
                b2.A = o.Et.p; b2.sai = o.Et.ld; b2.sak = 1;
                b2.B = o.CWT.p; b2.sbk = o.CWT.ld; b2.sbj = 1;
                b2.C = o.BW.p + (long long)n * o.BW.ld; b2.ldc = o.BW.ld; b2.alpha = TO(1); b2.beta = TO(0);
                gemm<TO>(b2, s);
            }
            transpose<TO>(o.BW.p, o.BW.ld, o.BWT.p, o.BWT.ld, n + m1, m2, s);
        }
        PCG_CK(cudaMemcpyAsync(h_info, d_info, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
        cudaFreeAsync(Hw, s);
        if (Aw) cudaFreeAsync(Aw, s);
        if (G) cudaFreeAsync(G, s);
        if (S) cudaFreeAsync(S, s);
        wait_stream();
        PCG_CK(cudaGetLastError());
        if (h_info[0] != 0) throw QpError{QP_ENOTCONVEX};
        if (h_info[2] != 0) throw QpError{QP_ESINGULAR};
        fp32_pivot_warn = (h_info[1] != 0) || (h_info[3] != 0);
        o.factored = true;
        }
    }

    void factor() {
        if (factored) return;
        PCG_CK(cudaEventRecord(evA, s));
        factor_op<double>();
        if (!f64) {
            if (fp32_pivot_warn && allow_pc64) {
                // A pivot of H or of A H^{-1} A' is below FP32 resolution relative to its
                // diagonal (ill-conditioned H or F_H): with mixed_fallback the QP is solved
                // with the FP64 operator from the start.
                if (verbose) std::fprintf(stderr, "  K0 pivots below FP32 resolution: FP64 from the start\n");
                all64 = true;
                use64 = pc64 = true;
            } else {
                factor_op<float>();
            }
        }
        const int pc = resolve_pc(opt.precond, n, m1);
        if (pc_kind(pc) == PC_H_K) {
            if (f64 || all64) ensure_T<double>(pc); else ensure_T<float>(pc);
        }
        PCG_CK(cudaEventRecord(evB, s));
        PCG_CK(cudaEventSynchronize(evB));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, evA, evB);
        stats.t_factor_ms = ms;
        factored = true;
    }

    // The persistent kernel applies an FP32 P_H factor as one symmetric product
    // P~^{-1} = W'W (formed each IPM iteration, m2^3 flops at FP32 rates) and an FP64
    // one as its two triangles W, then W' (one more phase, no FP64 product).
    // The FP32 Cholesky, its inverse and W'W run on the CUDA cores (round to
    // nearest): the tensor cores' FP32 accumulation is biased toward zero, and
    // W'W formed there (K = m2 terms) was indefinite enough in P~'s small
    // eigendirections that PCG stopped converging (5,600 instead of 200 PCG
    // iterations per Newton direction on the n=2000 workload).
    template <typename TP>
    static constexpr bool ph_one_phase() { return std::is_same<TP, float>::value; }

    // T = C H^{-1} C' = (C R^{-1})(C R^{-1})' (exact) or C diag(H)^{-1} C' (diag),
    // once per QP, from the operator factor of the same precision.
    template <typename TP>
    void ensure_T(int kind) {
        Pc<TP>& P = pcd<TP>();
        if (P.t_kind == kind) return;
        factor_op<TP>();
        Op<TP>& o = op<TP>();
        if (!P.Tm.p) {
            P.Tm.alloc(arena, m2, m2);
            P.Pm.alloc(arena, m2, m2);
            P.WPl.alloc(arena, m2, m2);
            P.WPu.alloc(arena, m2, m2);
            P.sg = vec<TP>(m2); P.rs = vec<TP>(m2); P.pv = vec<TP>(m2); P.Dp = vec<TP>(m2);
            P.oV[0] = vec<TP>(m2); P.oV[1] = vec<TP>(m2);
            if (ph_one_phase<TP>()) P.PI.alloc(arena, m2, m2);
            chol_inv_prepare<TP, TP>();
        }
        TP* Bp = nullptr;
        const long long ldb = pad_ld(n);
        if (cudaMallocAsync(&Bp, (size_t)m2 * ldb * sizeof(TP) + 256, s) != cudaSuccess) {
            cudaGetLastError();
            throw NoMem{};
        }
        bool tc = false;
        if constexpr (std::is_same<TP, float>::value) {
            // FP32: both products on the tensor cores (FP32-accurate 3xTF32 splits)
            float* sc = tc_scratch(tc_scratch_floats(n, m2));
            float *ch = sc, *cl = ch + (size_t)m2 * ldb, *wh = cl + (size_t)m2 * ldb, *wl = wh + (size_t)n * ldb;
            PCG_CK(cudaMemsetAsync(d_tcerr, 0, sizeof(int), s));
            tc = true;
            if (kind == QP_PC_PH_EXACT) {
                // B = C R^{-1} = C WH': (B)_ij = sum_k C_ik WH_jk
                tc_split(o.CW.p, o.CW.ld, m2, n, ch, cl, ldb, s);
                tc_split(o.WH.p, o.WH.ld, n, n, wh, wl, ldb, s);
                tc = tc_gemm(m2, n, n, 1.0f, ch, cl, ldb, wh, wl, ldb, 0.0f, Bp, ldb, true, false, d_tcerr, s);
            } else {
                double* hs = stage[3];
                diag_rsqrt_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, H.p, H.ld, hs);
                convert2d<double, TP>(C.p, C.ld, Bp, ldb, m2, n, s, hs);
            }
            if (tc) {
                // T = B B' (lower tiles)
                tc_split(Bp, ldb, m2, n, ch, cl, ldb, s);
                tc = tc_gemm(m2, m2, n, 1.0f, ch, cl, ldb, ch, cl, ldb, 0.0f, P.Tm.p, P.Tm.ld, true, true, d_tcerr, s);
            }
            if (!tc) cudaGetLastError();
        }
        if (!tc) {
            if (kind == QP_PC_PH_EXACT) {
                GemmArgs<TP> g{};
                g.M = m2; g.N = n; g.K = n;
                g.A = o.CW.p; g.sai = o.CW.ld; g.sak = 1;
                g.B = o.WH.p; g.sbk = 1; g.sbj = o.WH.ld; g.b_tri = TRI_UPPER;
                g.C = Bp; g.ldc = ldb; g.alpha = TP(1); g.beta = TP(0);
                gemm<TP>(g, s);
            } else {
                double* hs = stage[3];
                diag_rsqrt_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, H.p, H.ld, hs);
                convert2d<double, TP>(C.p, C.ld, Bp, ldb, m2, n, s, hs);
            }
            GemmArgs<TP> h{};
            h.M = m2; h.N = m2; h.K = n;
            h.A = Bp; h.sai = ldb; h.sak = 1;
            h.B = Bp; h.sbk = 1; h.sbj = ldb;
            h.C = P.Tm.p; h.ldc = P.Tm.ld; h.alpha = TP(1); h.beta = TP(0); h.lower_out = 1;
            gemm<TP>(h, s);
        }
        cudaFreeAsync(Bp, s);
        wait_stream();
        PCG_CK(cudaGetLastError());
        if (std::is_same<TP, float>::value) tc_check();
        P.t_kind = kind;
    }

    // P~ = Sg (D + T) Sg + shift I, Sg = diag(D + T)^{-1/2}; Cholesky and inverse
    // (Sec. 5.2 PH-KF: P_H factored at every IPM iteration).  P~ is SPD in exact
    // arithmetic, but late in the IPM its smallest eigenvalues (directions in
    // null(T) with small D) fall below the working precision and the Cholesky
    // meets pivots under the floor; it is then refactored with a diagonal shift
    // (a preconditioner only needs to be SPD: the shift changes PCG iteration
    // counts, never the solution).
    template <typename TP>
    double build_ph(const double* Dd) {
        Pc<TP>& P = pcd<TP>();
        constexpr bool is64 = std::is_same<TP, double>::value;
        const double floor = is64 ? 1e-12 : 1e-5;
        convert1d<double, TP>(m2, Dd, 1.0, P.Dp, s);
        double shift = 0.0;
        for (int attempt = 0; attempt < 6; ++attempt) {
            build_scaled_ph_kernel<TP><<<304 * 4, 256, 0, s>>>(P.Tm.p, P.Tm.ld, P.Dp, P.Pm.p, P.Pm.ld, P.sg, m2, shift);
            PCG_CK(cudaMemsetAsync(P.WPl.p, 0, (size_t)m2 * P.WPl.ld * sizeof(TP), s));
            PCG_CK(cudaMemsetAsync(d_info + 4, 0, sizeof(int), s));
            chol_inv<TP, TP>(P.Pm.p, P.Pm.ld, P.WPl.p, P.WPl.ld, m2, 1, floor, d_info + 4, s);
            PCG_CK(cudaMemcpyAsync(h_info + 4, d_info + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
            sync_check();
            if (h_info[4] == 0) break;
            shift = (shift == 0.0) ? (is64 ? 1e-10 : 1e-4) : shift * 10.0;
        }
        transpose<TP>(P.WPl.p, P.WPl.ld, P.WPu.p, P.WPu.ld, m2, m2, s);
        if (P.PI.p) {
            // P~^{-1} = W' W (W = L^{-1} lower): opA(i,k) = W[k,i], zero for k < i;
            // opB(k,j) = W[k,j], zero for k < j
            GemmArgs<TP> g{};
            g.M = m2; g.N = m2; g.K = m2;
            g.A = P.WPl.p; g.sai = 1; g.sak = P.WPl.ld; g.a_tri = TRI_UPPER;
            g.B = P.WPl.p; g.sbk = P.WPl.ld; g.sbj = 1; g.b_tri = TRI_LOWER;
            g.C = P.PI.p; g.ldc = P.PI.ld; g.alpha = TP(1); g.beta = TP(0);
            gemm<TP>(g, s);
        }
        P.shift = shift;
        if (verbose && shift > 0) std::fprintf(stderr, "  P_H shift %.1e\n", shift);
        return shift;
    }

    // ------------------------------------------------------- hot-path products
    // [a; b] = K0^{-1} [u; w] with z1 = R^{-T} u, z2 = L_S^{-1} w - Gt z1,
    // a = R^{-1}(z1 + Gt' z2), and mb = -b = L_S^{-T} z2 (forward solve, D^{-1},
    // back solve of the LDL' factor).
    template <typename TO>
    void k0_solve_dev(const TO* u, const TO* w, TO* a, TO* mb, const int* skip = nullptr) {
        Op<TO>& o = op<TO>();
        launch_gemv<TO, TRI_LOWER>(o.WH.p, n, n, o.WH.ld, u, lin<TO>(o.kz1), nullptr, skip, s);
        if (m1) {
            if (w) {
                launch_gemv<TO, TRI_LOWER>(o.WS.p, m1, m1, o.WS.ld, w, lin<TO>(o.ke), nullptr, skip, s);
                launch_gemv<TO, TRI_NONE>(o.Gt.p, m1, n, o.Gt.ld, o.kz1, lin<TO>(o.kz2, TO(-1), o.ke, TO(1)), nullptr, skip, s);
            } else {
                launch_gemv<TO, TRI_NONE>(o.Gt.p, m1, n, o.Gt.ld, o.kz1, lin<TO>(o.kz2, TO(-1)), nullptr, skip, s);
            }
            launch_gemv<TO, TRI_NONE>(o.GtT.p, n, m1, o.GtT.ld, o.kz2, lin<TO>(o.kt, TO(1), o.kz1, TO(1)), nullptr, skip, s);
            launch_gemv<TO, TRI_UPPER>(o.WHT.p, n, n, o.WHT.ld, o.kt, lin<TO>(a), nullptr, skip, s);
            if (mb) launch_gemv<TO, TRI_UPPER>(o.WST.p, m1, m1, o.WST.ld, o.kz2, lin<TO>(mb), nullptr, skip, s);
        } else {
            launch_gemv<TO, TRI_UPPER>(o.WHT.p, n, n, o.WHT.ld, o.kz1, lin<TO>(a), nullptr, skip, s);
        }
    }

    // q = K_F p = D p + C y, y = top block of K0^{-1} [C'p; 0]  (Sec. 5.2: a product
    // with C', a solve with the factor of F, a product with C).  Returns the grid of
    // the last GEMV (number of p'q partials in part_pq).
    template <typename TO>
    int kf_apply_dev(const TO* p, TO* q, const TO* Dw, const int* skip) {
        Op<TO>& o = op<TO>();
        launch_gemv<TO, TRI_NONE>(o.CWT.p, n, m2, o.CWT.ld, p, lin<TO>(o.pu), nullptr, skip, s);          // a6
        launch_gemv<TO, TRI_LOWER>(o.WH.p, n, n, o.WH.ld, o.pu, lin<TO>(o.pz1), nullptr, skip, s);       // a7
        const TO* top = o.pz1;
        if (m1) {
            launch_gemv<TO, TRI_NONE>(o.Gt.p, m1, n, o.Gt.ld, o.pz1, lin<TO>(o.pz2, TO(-1)), nullptr, skip, s);
            launch_gemv<TO, TRI_NONE>(o.GtT.p, n, m1, o.GtT.ld, o.pz2, lin<TO>(o.pt, TO(1), o.pz1, TO(1)), nullptr, skip, s);
            top = o.pt;
        }
        launch_gemv<TO, TRI_UPPER>(o.WHT.p, n, n, o.WHT.ld, top, lin<TO>(o.py), nullptr, skip, s);
        return launch_gemv<TO, TRI_NONE>(o.CW.p, m2, n, o.CW.ld, o.py, EpiKF<TO>{q, Dw, p}, part_pq, skip, s); // a8
    }

    // ------------------------------------------------------------------- PCG
    // One PCG iteration (a6-a10): K_F p, alpha update, preconditioner, beta update.
    template <typename TO, typename TP>
    void pcg_body(int kind) {
        Op<TO>& o = op<TO>();
        Pc<TP>& P = pcd<TP>();
        const int* skip = &st->done;
        const int npq = kf_apply_dev<TO>(o.pp, o.pq, o.pD, skip);
        const int gv = vec_grid(m2);
        if (kind == PC_L_K)
            pcg_alpha_kernel<TO, TP, PC_L_K><<<gv, kVecThreads, 0, s>>>(m2, st, part_pq, npq, o.px, o.pr, o.pp, o.pq,
                                                                         o.pz, o.pDinv, P.rs, P.sg, part_rr, part_rz);
        else if (kind == PC_H_K)
            pcg_alpha_kernel<TO, TP, PC_H_K><<<gv, kVecThreads, 0, s>>>(m2, st, part_pq, npq, o.px, o.pr, o.pp, o.pq,
                                                                         o.pz, o.pDinv, P.rs, P.sg, part_rr, part_rz);
        else
            pcg_alpha_kernel<TO, TP, PC_NONE_K><<<gv, kVecThreads, 0, s>>>(m2, st, part_pq, npq, o.px, o.pr, o.pp, o.pq,
                                                                            o.pz, o.pDinv, P.rs, P.sg, part_rr, part_rz);
        int nrz = gv;
        if (kind == PC_H_K) {                                                                          // a9
            launch_gemv<TP, TRI_LOWER>(P.WPl.p, m2, m2, P.WPl.ld, P.rs, lin<TP>(P.pv), nullptr, skip, s);
            nrz = launch_gemv<TP, TRI_UPPER>(P.WPu.p, m2, m2, P.WPu.ld, P.pv, EpiScaleDot<TP, TO>{o.pz, P.sg, o.pr},
                                             part_rz, skip, s);
        }
        pcg_beta_kernel<TO><<<gv, kVecThreads, 0, s>>>(m2, st, o.pz, o.pp, part_rz, nrz, part_rr, gv);    // a10
    }

    template <typename TO, typename TP>
    void pcg_init(int kind, const TO* rhs, double tol, int maxit, int stall) {
        Op<TO>& o = op<TO>();
        Pc<TP>& P = pcd<TP>();
        cur_tol = tol;
        const int gv = vec_grid(m2);
        if (kind == PC_L_K)
            pcg_init1_kernel<TO, TP, PC_L_K><<<gv, kVecThreads, 0, s>>>(m2, rhs, o.px, o.pr, o.pz, o.pDinv, P.rs, P.sg,
                                                                         part_bb, part_rz);
        else if (kind == PC_H_K)
            pcg_init1_kernel<TO, TP, PC_H_K><<<gv, kVecThreads, 0, s>>>(m2, rhs, o.px, o.pr, o.pz, o.pDinv, P.rs, P.sg,
                                                                         part_bb, part_rz);
        else
            pcg_init1_kernel<TO, TP, PC_NONE_K><<<gv, kVecThreads, 0, s>>>(m2, rhs, o.px, o.pr, o.pz, o.pDinv, P.rs,
                                                                            P.sg, part_bb, part_rz);
        int nrz = gv;
        if (kind == PC_H_K) {
            launch_gemv<TP, TRI_LOWER>(P.WPl.p, m2, m2, P.WPl.ld, P.rs, lin<TP>(P.pv), nullptr, nullptr, s);
            nrz = launch_gemv<TP, TRI_UPPER>(P.WPu.p, m2, m2, P.WPu.ld, P.pv, EpiScaleDot<TP, TO>{o.pz, P.sg, o.pr},
                                             part_rz, nullptr, s);
        }
        pcg_init2_kernel<TO><<<gv, kVecThreads, 0, s>>>(m2, st, o.pz, o.pp, part_bb, gv, part_rz, nrz, tol, maxit,
                                                        stall);
    }

    int check_every() const { return opt.pcg_check_every < 0 ? -opt.pcg_check_every : 8; }

    // Iterations without a 4x residual decrease after which a Newton-direction
    // solve stops: three times the exact-arithmetic bound of Corollaries 1/2
    // (n-m1+1 for P_L, m1+1 for P_H; m2 without preconditioner) plus 100, so the
    // plateau-then-drop convergence of CG on a few distinct eigenvalues is never cut.
    int stall_window(int kind) const {
        const int bound = kind == PC_L_K ? (n - m1 + 1) : (kind == PC_H_K ? (m1 + 1) : m2);
        return 3 * bound + 100;
    }

    template <typename TO, typename TP>
    cudaGraphExec_t get_graph(int kind) {
        Op<TO>& o = op<TO>();
        const int K = check_every();
        if (o.graph[kind] && o.graph_k[kind] == K) return o.graph[kind];
        if (o.graph[kind]) cudaGraphExecDestroy(o.graph[kind]);
        cudaGraph_t g;
        PCG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < K; ++i) pcg_body<TO, TP>(kind);
        PCG_CK(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ge;
        PCG_CK(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        o.graph[kind] = ge;
        o.graph_k[kind] = K;
        return ge;
    }

    // ------------------------------------------------- persistent PCG kernel
    // Phases of the persistent kernel for the handle's pcg_form and preconditioner
    // kind, with every block's rows (whole rows, balanced by chunk count) in tbl.
    struct FusedPlan {
        Phase ph[kMaxPhases];
        int nop = 0, npc = 0;
        size_t xs_elems_o = 0, xs_elems_p = 0;   // staged-vector length in TO / TP elements
        size_t spart_bytes = 0;
        size_t xo_bytes = 0;                      // the block's slice of x
        std::vector<int2> tbl;
    };
    int2* d_tbl = nullptr;                 // device copy of the block tables (kMaxPhases x (1024 + 1))
    std::vector<int2> h_tbl_cur;           // what d_tbl holds
    static constexpr int kTblStride = 1025;

    static Part mk_part(const void* M, long long ld, int r0, int r1, int cols, int tri, int xoff) {
        Part p;
        p.M = M; p.ld = ld; p.r0 = r0; p.r1 = r1; p.cols = cols; p.tri = tri; p.xoff = xoff;
        p.rp = nullptr; p.ci = nullptr;
        return p;
    }
    static Part mk_csr(const void* val, const int* rp, const int* ci, int rows, int cols) {
        Part p = mk_part(val, pad_ld(cols), 0, rows, cols, TRI_NONE, 0);
        p.rp = rp; p.ci = ci;
        return p;
    }
    static int padc(int v, int ch) { return (v + ch - 1) / ch * ch; }

    static int slot_bytes_for(int grid) { return grid > kMaxClusterBlocks ? kBigSlotBytes : kSmallSlotBytes; }

    template <typename TO, typename TP>
    FusedPlan plan_fused(int kind, int grid) {
        Op<TO>& o = op<TO>();
        Pc<TP>& P = pcd<TP>();
        const int sb = slot_bytes_for(grid);
        const int CHO = sb / (int)sizeof(TO), CHP = sb / (int)sizeof(TP);
        auto p32 = [](int v) { return (v + 31) / 32 * 32; };   // staged vectors: the matrices' leading dimension
        FusedPlan F;
        auto phase = [&](std::initializer_list<Part> parts, int rows) {
            Phase ph{};
            ph.np = 0;
            for (const Part& q : parts) ph.p[ph.np++] = q;
            ph.rows = rows;
            ph.in_s2 = 1.0f;
            return ph;
        };
        auto input = [&](Phase& ph, int len1, int off2, int len2, float s2, int pad) {
            ph.in_len1 = len1; ph.in_off2 = off2; ph.in_len2 = len2; ph.in_s2 = s2; ph.in_pad = pad;
        };
        const int form = opt.pcg_form;
        if (form == 3) {
            const int r = o.lr;
            F.ph[0] = phase({mk_part(o.LVT.p, o.LVT.ld, 0, r, m2, TRI_NONE, 0)}, r);
            F.ph[1] = phase({mk_part(o.LV.p, o.LV.ld, 0, m2, r, TRI_NONE, 0)}, m2);
            input(F.ph[1], r, 0, 0, 1.0f, p32(r));
            F.nop = 2;
        } else if (form == 1) {
            F.ph[0] = phase({mk_part(o.BW.p, o.BW.ld, 0, n + m1, m2, TRI_NONE, 0)}, n + m1);
            F.ph[1] = phase({mk_part(o.BWT.p, o.BWT.ld, 0, m2, n + m1, TRI_NONE, 0)}, m2);
            input(F.ph[1], n, n, m1, -1.0f, p32(n + m1));
            F.nop = 2;
        } else if (form == 2) {
            F.ph[0] = phase({crp ? mk_csr(o.ctval, ctrp, ctci, n, m2) : mk_part(o.CWT.p, o.CWT.ld, 0, n, m2, TRI_NONE, 0)}, n);
            if (m1) {
                F.ph[1] = phase({mk_part(o.WH.p, o.WH.ld, 0, n, n, TRI_LOWER, 0),
                                 mk_part(o.Et.p, o.Et.ld, n, n + m1, n, TRI_NONE, 0)}, n + m1);
                F.ph[2] = phase({mk_part(o.WHT.p, o.WHT.ld, 0, n, n, TRI_UPPER, 0),
                                 mk_part(o.EtT.p, o.EtT.ld, 0, n, m1, TRI_NONE, p32(n))}, n);
                input(F.ph[2], n, p32(n), m1, -1.0f, p32(n) + p32(m1));
            } else {
                F.ph[1] = phase({mk_part(o.WH.p, o.WH.ld, 0, n, n, TRI_LOWER, 0)}, n);
                F.ph[2] = phase({mk_part(o.WHT.p, o.WHT.ld, 0, n, n, TRI_UPPER, 0)}, n);
                input(F.ph[2], n, 0, 0, 1.0f, p32(n));
            }
            input(F.ph[1], n, 0, 0, 1.0f, p32(n));
            F.ph[3] = phase({crp ? mk_csr(o.cval, crp, cci, m2, n) : mk_part(o.CW.p, o.CW.ld, 0, m2, n, TRI_NONE, 0)}, m2);
            input(F.ph[3], n, 0, 0, 1.0f, p32(n));
            F.nop = 4;
        } else {
            F.ph[0] = phase({crp ? mk_csr(o.ctval, ctrp, ctci, n, m2) : mk_part(o.CWT.p, o.CWT.ld, 0, n, m2, TRI_NONE, 0)}, n);
            F.ph[1] = phase({mk_part(o.M0.p, o.M0.ld, 0, n, n, TRI_NONE, 0)}, n);
            input(F.ph[1], n, 0, 0, 1.0f, p32(n));
            F.ph[2] = phase({crp ? mk_csr(o.cval, crp, cci, m2, n) : mk_part(o.CW.p, o.CW.ld, 0, m2, n, TRI_NONE, 0)}, m2);
            input(F.ph[2], n, 0, 0, 1.0f, p32(n));
            F.nop = 3;
        }
        if (kind == PC_H_K) {
            if (P.PI.p) {
                F.ph[F.nop] = phase({mk_part(P.PI.p, P.PI.ld, 0, m2, m2, TRI_NONE, 0)}, m2);
                F.npc = 1;
            } else {
                F.ph[F.nop] = phase({mk_part(P.WPl.p, P.WPl.ld, 0, m2, m2, TRI_LOWER, 0)}, m2);
                F.ph[F.nop + 1] = phase({mk_part(P.WPu.p, P.WPu.ld, 0, m2, m2, TRI_UPPER, 0)}, m2);
                input(F.ph[F.nop + 1], m2, 0, 0, 1.0f, p32(m2));
                F.npc = 2;
            }
        }
        // the first phase's input is p (m2, padded); the P_H phases' is Sg r
        F.xs_elems_o = p32(m2);
        F.xs_elems_p = p32(m2);
        {   // the block's slice of x: m2 / grid elements, or whole kSeg segments (sliced FP64 update)
            const size_t nseg = (size_t)(m2 + kSeg - 1) / kSeg;
            const size_t el = std::max<size_t>((size_t)(m2 + grid - 1) / grid, (nseg + grid - 1) / grid * kSeg);
            F.xo_bytes = (el * sizeof(TO) + 15) / 16 * 16;
        }
        F.tbl.assign((size_t)(F.nop + F.npc) * (grid + 1), int2{0, 0});
        for (int k = 0; k < F.nop + F.npc; ++k) {
            Phase& ph = F.ph[k];
            const bool isP = k >= F.nop;
            const int CH = isP ? CHP : CHO;
            const size_t es = isP ? sizeof(TP) : sizeof(TO);
            if (k > 0 && k != F.nop) {
                if (isP) F.xs_elems_p = std::max(F.xs_elems_p, (size_t)ph.in_pad);
                else F.xs_elems_o = std::max(F.xs_elems_o, (size_t)ph.in_pad);
            }
            // balance rows by weight: 64 per ring item, 1 per row (CSR rows, rows of a
            // phase without dense chunks); the table records the item prefix
            std::vector<int> pre(ph.rows + 1, 0);
            std::vector<long long> wpre(ph.rows + 1, 0);
            int ncmax = 1;
            for (int r = 0; r < ph.rows; ++r) {
                const int it = row_items(ph, CH, r);
                ncmax = std::max(ncmax, it);
                pre[r + 1] = pre[r] + it;
                wpre[r + 1] = wpre[r] + 64LL * it + 1;
            }
            ph.ncmax = ncmax;
            ph.tbl = k * (grid + 1);
            ph.flat = (ph.np == 1 && !ph.p[0].rp && ph.p[0].tri == TRI_NONE && ph.p[0].r0 == 0 &&
                       ph.p[0].r1 == ph.rows) ? 1 : 0;
            const long long total = wpre[ph.rows];
            int maxrows = 0;
            for (int b = 0; b <= grid; ++b) {
                const long long tgt = (total * b + grid / 2) / grid;
                const int r = (b == grid) ? ph.rows
                                          : (int)(std::lower_bound(wpre.begin(), wpre.end(), tgt) - wpre.begin());
                F.tbl[(size_t)ph.tbl + b] = int2{r, pre[r]};
                if (b > 0) maxrows = std::max(maxrows, r - F.tbl[(size_t)ph.tbl + b - 1].x);
            }
            if (ph.flat) {
                // full-slot chunks over each block's contiguous rows: item prefix per block
                const long long ld = ph.p[0].ld;
                int acc = 0;
                for (int b = 0; b <= grid; ++b) {
                    int2& t = F.tbl[(size_t)ph.tbl + b];
                    const int r = t.x;
                    t.y = acc;
                    if (b < grid) acc += flat_items(r, F.tbl[(size_t)ph.tbl + b + 1].x, ld, CH);
                }
                ph.ncmax = (int)((ld + CH - 1) / CH) + 1;
                ncmax = ph.ncmax;
            }
            F.spart_bytes = std::max(F.spart_bytes, (size_t)maxrows * ncmax * es);
            // every part's stored row (leading dimension) must lie inside the staged vector
            for (int q = 0; q < ph.np; ++q) {
                const size_t need = (size_t)ph.p[q].xoff + (size_t)ph.p[q].ld;
                if (isP) F.xs_elems_p = std::max(F.xs_elems_p, need);
                else F.xs_elems_o = std::max(F.xs_elems_o, need);
            }
        }
        return F;
    }

    template <typename TO, typename TP>
    size_t fused_xs_bytes(const FusedPlan& F) const {
        const size_t b = std::max(F.xs_elems_o * sizeof(TO), F.xs_elems_p * sizeof(TP));
        return (b + 15) / 16 * 16;
    }

    // Ring depth: as deep as the block's shared-memory limit allows after the staged
    // vector, the m2-vector caches and the per-row partials (at most kMaxSlots).
    template <typename TO, typename TP>
    int fused_slots(const FusedPlan& F, int slot_bytes, int qcache) const {
        const size_t sp = fused_spart_offset<TO>(fused_xs_bytes<TO, TP>(F), m2, qcache);
        const size_t off = fused_ring_offset((sp + F.spart_bytes + 15) / 16 * 16, F.xo_bytes);
        const size_t lim = fused_smem_limit();
        const size_t per = slot_bytes + 2 * sizeof(uint64_t) + sizeof(int);
        if (off + 16 + per > lim) return 0;
        return (int)std::min<size_t>(kMaxSlots, (lim - off - 16) / per);
    }

    // The persistent cooperative PCG kernel: one launch runs the whole solve from
    // the pcg_init state (x = 0, r = rhs, p = z0); the final state ends in hst[0].
    // Small QPs (a grid of at most kMaxClusterBlocks) run 256-thread blocks, two per
    // SM; larger ones 512-thread blocks, one per SM.  The choice depends only on
    // the QP's sizes, so a QP's results do not depend on what else runs.
    template <typename TO, typename TP, int PC>
    void launch_fused() {
        int dev = 0, sms = 0;
        PCG_CK(cudaGetDevice(&dev));
        PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = grid_for<TO>(sms, PC);
        stats.pcg_grid = grid;
        if (grid <= kMaxClusterBlocks) launch_fused_nt<TO, TP, PC, kSmallBlock>(grid, sms);
        else launch_fused_nt<TO, TP, PC, kBigBlock>(grid, sms);
    }

    template <typename TO, typename TP, int PC, int NT>
    void launch_fused_nt(int grid, int sms) {
        Op<TO>& o = op<TO>();
        Pc<TP>& P = pcd<TP>();
        FusedPlan F = plan_fused<TO, TP>(PC, grid);
        const bool same = F.tbl.size() == h_tbl_cur.size() &&
                          std::memcmp(F.tbl.data(), h_tbl_cur.data(), F.tbl.size() * sizeof(int2)) == 0;
        if (!same) {
            if (F.tbl.size() > (size_t)kMaxPhases * kTblStride) throw QpError{QP_EINVAL};
            h_tbl_cur = F.tbl;
            PCG_CK(cudaMemcpyAsync(d_tbl, h_tbl_cur.data(), h_tbl_cur.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        }
        FusedArgs<TO, TP> fa{};
        fa.n = n; fa.m1 = m1; fa.m2 = m2;
        for (int k = 0; k < F.nop + F.npc; ++k) fa.ph[k] = F.ph[k];
        fa.nop = F.nop; fa.npc = F.npc;
        fa.tbl = d_tbl;
        if (opt.pcg_form == 1 || opt.pcg_form == 3) {
            fa.out[0] = o.oZ; fa.out[1] = o.oW;
        } else if (opt.pcg_form == 2) {
            fa.out[0] = o.oU; fa.out[1] = o.oZ; fa.out[2] = o.oY; fa.out[3] = o.oW;
        } else {
            fa.out[0] = o.oU; fa.out[1] = o.oY; fa.out[2] = o.oW;
        }
        fa.outP[0] = P.oV[0]; fa.outP[1] = P.oV[1];
        fa.sg = P.sg;
        fa.D = o.pD; fa.Dinv = o.pDinv; fa.x = o.px;
        fa.r_in = o.pr; fa.p_in = o.pp;
        fa.st = st; fa.bar = bar;
        fa.segp = o.segp; fa.zbuf = o.zb; fa.nseg = (m2 + kSeg - 1) / kSeg;
        fa.tstamp = phase_times ? tstamp : nullptr;
        fa.leave_early = leave_early ? 1 : 0;
        {   // block 0's chunks of iteration 2 (its items per iteration from the table)
            int per_it = 0;
            for (int k = 0; k < F.nop + F.npc; ++k) per_it += F.tbl[(size_t)F.ph[k].tbl + 1].y - F.tbl[(size_t)F.ph[k].tbl].y;
            fa.trace0 = 2 * per_it;
            trace_per_it = per_it;
        }
        auto kern = pcg_fused_kernel<TO, TP, PC, NT>;
        fa.xs_bytes = fused_xs_bytes<TO, TP>(F);
        // A QP whose grid covers most of the GPU takes the deepest ring that fits; a
        // small one (batched with others) a shallow ring, so that the blocks of several
        // QPs share an SM.  Without room for min_slots(grid) slots beside the q cache
        // (FP64 with a large m2), the cache gives way to the ring.
        fa.slot_bytes = slot_bytes_for(grid);
        fa.qcache = fused_qcache<TO, TP>(F, grid);
        fa.spart_off = fused_spart_offset<TO>(fa.xs_bytes, m2, fa.qcache);
        fa.xo_off = (fa.spart_off + F.spart_bytes + 15) / 16 * 16;
        fa.ring_off = fused_ring_offset(fa.xo_off, F.xo_bytes);
        int per_sm = 0;
        fa.slots = fused_slots<TO, TP>(F, fa.slot_bytes, fa.qcache);
        if (2 * grid < sms) fa.slots = std::min(fa.slots, kSmallRingSlots);
        if (fa.slots < (fa.qcache == 1 ? min_slots(grid) : kMinSlotsNoCache)) {
            if (verbose) std::fprintf(stderr, "  persistent PCG: %d ring slots of %d bytes do not fit\n", fa.slots, fa.slot_bytes);
            throw QpError{QP_ENOMEM};
        }
        const size_t smem = fused_smem_bytes(fa.ring_off, fa.slots, fa.slot_bytes);
        // Kernel attributes are shared by every thread of the process: set them once
        // (the dynamic shared-memory limit to the block's maximum; the launch itself
        // uses only `smem`), never per call.
        static const cudaError_t attr_ok = [&]() {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)fused_smem_limit());
            if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            return e;
        }();
        PCG_CK(attr_ok);
        PCG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
        if (per_sm < 1) {
            if (verbose) std::fprintf(stderr, "  persistent PCG: no block fits with %zu bytes of shared memory\n", smem);
            throw QpError{QP_ENOMEM};
        }
        PCG_CK(cudaMemsetAsync(bar, 0, sizeof(GridBar), s));
        // A grid of at most kMaxClusterBlocks blocks is launched as one thread-block
        // cluster: the hardware schedules the blocks of a cluster together, which is all
        // the grid barrier needs, and the cluster launches of QPs solved at the same
        // time run side by side.  Larger grids use a cooperative launch.
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = grid;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        bool cluster = false;
        if (grid <= kMaxClusterBlocks) {
            const void* key = (const void*)kern;
            if (cl_key != key || cl_grid != grid || cl_smem != smem) {
                int nclusters = 0;
                cl_ok = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0;
                cudaGetLastError();
                cl_key = key; cl_grid = grid; cl_smem = smem;
            }
            cluster = cl_ok;
        }
        if (cluster) {
            PCG_CK(cudaLaunchKernelEx(&cfg, kern, fa));
        } else {
            void* args[] = {(void*)&fa};
            PCG_CK(cudaLaunchCooperativeKernel((const void*)kern, grid, NT, args, smem, s));
        }
        last_fused_grid = grid;
    }
    int last_fused_grid = 0;
    int trace_per_it = 0;

    template <typename TO, typename TP>
    void pcg_run_fused(int kind) {
        if (kind == PC_L_K) launch_fused<TO, TP, PC_L_K>();
        else if (kind == PC_H_K) launch_fused<TO, TP, PC_H_K>();
        else launch_fused<TO, TP, PC_NONE_K>();
        PCG_CK(cudaMemcpyAsync(&hst[0], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaMemcpyAsync(h_info + 6, &bar->count, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        sync_check();
        if ((unsigned)h_info[6] & kBarErr) throw QpError{QP_ETIMEOUT};
        if (phase_times && hst[0].iter >= 4) {
            const int G = last_fused_grid;
            std::vector<unsigned long long> t(128 + 8 * (size_t)G);
            PCG_CK(cudaMemcpyAsync(t.data(), tstamp, t.size() * 8, cudaMemcpyDeviceToHost, s));
            wait_stream();
            std::fprintf(stderr, "phase marks (us from iteration start):");
            for (int i = 1; i < 4; ++i) {
                std::fprintf(stderr, "\n  it %d:", i);
                for (int ph = 1; ph < 32; ++ph)
                    if (t[i * 32 + ph] > t[i * 32]) std::fprintf(stderr, " m%d=%.1f", ph, (t[i * 32 + ph] - t[i * 32]) * 1e-3);
            }
            std::fprintf(stderr, "\n  iteration 2, phase ends over blocks (us from iteration start): ");
            for (int ph = 0; ph < 8; ++ph) {
                unsigned long long lo = ~0ull, hi = 0;
                for (int b = 0; b < G; ++b) {
                    const unsigned long long v = t[128 + (size_t)ph * G + b];
                    if (!v) continue;
                    lo = std::min(lo, v); hi = std::max(hi, v);
                }
                if (hi) std::fprintf(stderr, " ph%d [%.1f, %.1f]", ph, (lo - t[2 * 32]) * 1e-3, (hi - t[2 * 32]) * 1e-3);
            }
            std::fprintf(stderr, "\n");
            // block 0's chunk trace over iteration 2: copy latency, consumption, issue gaps
            std::vector<unsigned long long> tr(3 * kTrace);
            PCG_CK(cudaMemcpyAsync(tr.data(), tstamp + 128 + 8 * 1024, tr.size() * 8, cudaMemcpyDeviceToHost, s));
            wait_stream();
            std::vector<double> lat, use, wait_slot;
            const int nn = std::min(trace_per_it, kTrace);
            for (int q = 0; q < nn; ++q) {
                if (!tr[q] || !tr[kTrace + q] || !tr[2 * kTrace + q]) continue;
                lat.push_back((double)(tr[kTrace + q] - tr[q]) * 1e-3);
                use.push_back((double)(tr[2 * kTrace + q] - tr[kTrace + q]) * 1e-3);
            }
            auto med = [](std::vector<double> v) {
                if (v.empty()) return 0.0;
                std::sort(v.begin(), v.end());
                return v[v.size() / 2];
            };
            auto mx = [](const std::vector<double>& v) { return v.empty() ? 0.0 : *std::max_element(v.begin(), v.end()); };
            std::fprintf(stderr, "  block 0 chunks of iteration 2: %d traced; issue->landed median %.2f max %.2f us; "
                                 "landed->released median %.2f max %.2f us\n", (int)lat.size(), med(lat), mx(lat), med(use), mx(use));
            std::fprintf(stderr, "  issue times (us from the first): ");
            for (int q = 0; q < nn && q < 96; ++q) std::fprintf(stderr, "%.1f ", tr[q] ? (tr[q] - tr[0]) * 1e-3 : -1.0);
            std::fprintf(stderr, "\n  landed: ");
            for (int q = 0; q < nn && q < 96; ++q) std::fprintf(stderr, "%.1f ", tr[kTrace + q] ? (tr[kTrace + q] - tr[0]) * 1e-3 : -1.0);
            std::fprintf(stderr, "\n  released: ");
            for (int q = 0; q < nn && q < 96; ++q) std::fprintf(stderr, "%.1f ", tr[2 * kTrace + q] ? (tr[2 * kTrace + q] - tr[0]) * 1e-3 : -1.0);
            std::fprintf(stderr, "\n");
            PCG_CK(cudaMemsetAsync(tstamp, 0, (128 + 8 * 1024 + 3 * kTrace) * 8, s));
        }
    }

    // Shared memory of the persistent kernel: the opt-in limit of a block, less the
    // kernel's static shared memory (scalars, below 1 KB).
    static size_t fused_smem_limit() {
        static const size_t lim = []() {
            int d = 0, optin = 0;
            cudaGetDevice(&d);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
            if (optin <= 0) optin = 227 * 1024;
            return (size_t)optin - 2048;   // static shared memory of the kernel (scalars), below 2 KB
        }();
        return lim;
    }
    template <typename TO, typename TP>
    bool fused_fits(int kind) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = grid_for<TO>(sms, kind);
        const FusedPlan F = plan_fused<TO, TP>(kind, grid);
        return fused_qcache<TO, TP>(F, grid) >= 0;
    }
    // Fewest ring slots the persistent kernel runs with: 16 KB slots stream at the copy
    // rate with a handful in flight; 4 KB slots need one per consumer warp.
    static int min_slots(int grid) { return grid > kMaxClusterBlocks ? 6 : Blk<kSmallBlock>::warps; }
    // Fewest slots without the q cache (a large-grid ring of three 16 KB slots still
    // beats the per-phase kernels, whose launches cost more than the shallow ring).
    static constexpr int kMinSlotsNoCache = 3;
    // 1: the q cache and min_slots(grid) slots fit; 0: only without the cache (large
    // grids); -1: neither (the per-phase kernels run instead).
    template <typename TO, typename TP>
    int fused_qcache(const FusedPlan& F, int grid) const {
        const int sb = slot_bytes_for(grid);
        if (fused_slots<TO, TP>(F, sb, 1) >= min_slots(grid)) return 1;
        if (grid > kMaxClusterBlocks && fused_slots<TO, TP>(F, sb, 0) >= kMinSlotsNoCache) return 0;
        return -1;
    }

    bool use_fused() const { return opt.pcg_check_every >= 0; }

    // ---------------------------------------------------------------- autotuner
    // Grid of the persistent kernel per operator precision and preconditioner kind:
    // the tuned value once autotune_grid has run, else the rule (fused_grid).
    int tuned_grid[2][3] = {{0, 0, 0}, {0, 0, 0}};
    int force_grid = 0;   // set while the autotuner times a candidate
    template <typename TO>
    int grid_for(int sms, int kind) const {
        if (force_grid > 0) return force_grid;
        const int t = tuned_grid[std::is_same<TO, double>::value ? 1 : 0][kind];
        return t > 0 ? t : fused_grid(sms);
    }
    // Times a dozen PCG iterations (tolerance 0, the current right-hand side) for each
    // candidate grid -- the rule's G, 3G/4, G/2 and one block per SM, every one larger
    // than a cluster and with a ring that fits -- and keeps the fastest.  Only QPs whose
    // rule grid exceeds a cluster are tuned (small QPs share the GPU by design); the grid
    // never changes results, since every reduction has a grid-independent order.
    template <typename TO, typename TP>
    void autotune_grid(int kind) {
        const int pk = std::is_same<TO, double>::value ? 1 : 0;
        if (!opt.autotune || opt.pcg_blocks > 0 || !use_fused() || tuned_grid[pk][kind] != 0) return;
        int dev = 0, sms = 0;
        PCG_CK(cudaGetDevice(&dev));
        PCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int g0 = fused_grid(sms);
        tuned_grid[pk][kind] = g0;
        if (g0 <= kMaxClusterBlocks) return;
        std::vector<int> cand = {g0, std::max(kMaxClusterBlocks + 1, 3 * g0 / 4),
                                 std::max(kMaxClusterBlocks + 1, g0 / 2), sms};
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        Op<TO>& o = op<TO>();
        double best = 1e30;
        int best_g = g0;
        for (int g : cand) {
            if (g > sms) continue;
            force_grid = g;
            const bool fits = fused_qcache<TO, TP>(plan_fused<TO, TP>(kind, g), g) >= 0;
            if (!fits) continue;
            double ms_best = 1e30;
            for (int rep = 0; rep < 2; ++rep) {    // the first launch also uploads the tables
                pcg_init<TO, TP>(kind, o.prhs, 0.0, 12, 0);
                PCG_CK(cudaEventRecord(evA, s));
                pcg_run_fused<TO, TP>(kind);
                PCG_CK(cudaEventRecord(evB, s));
                sync_check();
                float ms = 0.f;
                PCG_CK(cudaEventElapsedTime(&ms, evA, evB));
                if (hst[0].iter > 0) ms_best = std::min(ms_best, (double)ms / hst[0].iter);
            }
            if (verbose) std::fprintf(stderr, "  autotune: grid %d, %.2f us per PCG iteration\n", g, ms_best * 1e3);
            if (ms_best < best) { best = ms_best; best_g = g; }
        }
        force_grid = 0;
        tuned_grid[pk][kind] = best_g;
    }

    // CTAs of the persistent kernel.  A QP streaming at most 32 x 512 KB per iteration
    // gets between 8 and kMaxClusterBlocks (one cluster, about one per 512 KB), so
    // that the kernels of several QPs solved concurrently share the GPU; a larger
    // one about one CTA per 128 KB, up to one per SM (a block's chunks of one
    // iteration then fit its ring, and an operator that stays in L2 -- the
    // low-rank form of the n=3000 few-dof workload, 19.6 MB -- is read by every SM).
    int fused_grid(int sms) const {
        const double by = bytes_per_iter(resolve_pc(opt.precond, n, m1));
        const int want = (int)std::ceil(by / (512.0 * 1024.0));
        int g = (want <= 2 * kMaxClusterBlocks) ? std::min(sms, std::max(8, std::min(want, kMaxClusterBlocks)))
                                                : std::min(sms, (int)std::ceil(by / (128.0 * 1024.0)));
        if (opt.pcg_blocks > 0) g = std::min(g, opt.pcg_blocks);
        return g;
    }

    // Runs PCG from the current pcg_init state until done; the final state ends in
    // hst[0].  Default: the persistent kernel.  pcg_check_every < 0: per-phase
    // kernels in a CUDA graph of |pcg_check_every| iterations, with status checks
    // pipelined one graph launch behind.
    template <typename TO, typename TP>
    void pcg_run(int kind, int maxit) {
        if (use_fused() && fused_fits<TO, TP>(kind)) {
            pcg_run_fused<TO, TP>(kind);
            return;
        }
        cudaGraphExec_t ge = get_graph<TO, TP>(kind);
        const int K = check_every();
        const int max_launch = maxit / K + 2;
        PCG_CK(cudaGraphLaunch(ge, s));
        PCG_CK(cudaMemcpyAsync(&hst[0], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaEventRecord(ev0, s));
        int launched = 1;
        int cur = 0;
        while (true) {
            const bool second = launched < max_launch;
            if (second) {
                PCG_CK(cudaGraphLaunch(ge, s));
                PCG_CK(cudaMemcpyAsync(&hst[1 - cur], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
                PCG_CK(cudaEventRecord(cur == 0 ? ev1 : ev0, s));
                ++launched;
            }
            PCG_CK(cudaEventSynchronize(cur == 0 ? ev0 : ev1));
            if (hst[cur].done || !second) {
                wait_stream();
                PCG_CK(cudaMemcpyAsync(&hst[0], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
                wait_stream();
                break;
            }
            cur = 1 - cur;
        }
        PCG_CK(cudaGetLastError());
    }

    // D-dependent data of the operator precision TO (D and 1/D for P_L).
    template <typename TO>
    void set_D_op(const double* Dd) {
        Op<TO>& o = op<TO>();
        convert1d<double, TO>(m2, Dd, 1.0, o.pD, s);
        recip_kernel<TO><<<vec_grid(m2), kVecThreads, 0, s>>>(m2, Dd, o.pDinv);
    }

    template <typename TP>
    double set_D_pc(const double* Dd, int pc) {
        if (pc_kind(pc) != PC_H_K) return 0.0;
        ensure_T<TP>(pc);
        PCG_CK(cudaEventRecord(evA, s));
        const double shift = build_ph<TP>(Dd);
        PCG_CK(cudaEventRecord(evB, s));
        PCG_CK(cudaEventSynchronize(evB));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, evA, evB);
        stats.t_precond_ms += ms;
        return shift;
    }

    // Mixed precision: once the FP32 Cholesky of P~ needs a diagonal shift (P~ has
    // eigenvalues below FP32 resolution: with m2 > n, the directions in null(C')
    // where D_i << T_ii), the QP moves its preconditioner and its operator to FP64
    // for the remaining IPM iterations.  (Applying the FP64 factor rounded to FP32
    // instead keeps the preconditioner SPD, but after the switch the inner solves
    // go to 1e-10 and a preconditioner applied at FP32 accuracy slows CG there:
    // 53% more PCG iterations on the n=2000 workload.)
    void set_D(const double* Dd, int pc) {
        if (!pc64) {
            const double shift = set_D_pc<float>(Dd, pc);
            if (shift > 0.0 && opt.precision == QP_PREC_FP32 && allow_pc64) {
                pc64 = true;
                if (verbose) std::fprintf(stderr, "  preconditioner -> FP64 at IPM iteration %d\n", ipm_k);
                if (stats.pc64_switch_iter < 0) stats.pc64_switch_iter = ipm_k;
                if (!use64) switch_to_op64();
            }
        }
        if (pc64) set_D_pc<double>(Dd, pc);
        if (use64) set_D_op<double>(Dd); else set_D_op<float>(Dd);
    }

    // PCG on K_F dnu = rhs with the operator of precision TO.
    template <typename TO, typename TP>
    int pcg_solve_t(const double* rhs, double* dnu, int kind, double tol, int maxit, int* iters, double* relres) {
        Op<TO>& o = op<TO>();
        convert1d<double, TO>(m2, rhs, 1.0, o.prhs, s);
        autotune_grid<TO, TP>(kind);
        pcg_init<TO, TP>(kind, o.prhs, tol, maxit, 0);
        pcg_run<TO, TP>(kind, maxit);
        convert1d<TO, double>(m2, o.px, 1.0, dnu, s);
        sync_check();
        if (iters) *iters = hst[0].iter;
        if (relres) *relres = hst[0].bb > 0 ? std::sqrt(hst[0].rr / hst[0].bb) : 0.0;
        if (hst[0].done == 3) return QP_ENUMERIC;
        if (hst[0].done == 2) return QP_EMAXIT;
        return QP_OK;
    }

    int pcg_solve(const double* Dd, const double* rhs, double* dnu, int pc, double tol, int maxit, int* iters,
                  double* relres) {
        pc = resolve_pc(pc, n, m1);
        set_D(Dd, pc);
        const int kind = pc_kind(pc);
        if (pc64) return pcg_solve_t<double, double>(rhs, dnu, kind, tol, maxit, iters, relres);
        if (use64) return pcg_solve_t<double, float>(rhs, dnu, kind, tol, maxit, iters, relres);
        return pcg_solve_t<float, float>(rhs, dnu, kind, tol, maxit, iters, relres);
    }

    template <typename TO, typename TP>
    void time_pcg_t(int kind, int warmup, int iters, double* ms_out) {
        Op<TO>& o = op<TO>();
        autotune_grid<TO, TP>(kind);
        if (use_fused() && fused_fits<TO, TP>(kind)) {
            // warm-up solve, then a timed solve of `iters` iterations (tolerance 0:
            // no early stop); the timed region includes the start kernels.
            pcg_init<TO, TP>(kind, o.prhs, 0.0, std::max(1, warmup), 0);
            pcg_run_fused<TO, TP>(kind);
            PCG_CK(cudaEventRecord(evA, s));
            pcg_init<TO, TP>(kind, o.prhs, 0.0, iters, 0);
            pcg_run_fused<TO, TP>(kind);
            PCG_CK(cudaEventRecord(evB, s));
            sync_check();
            float ms = 0.f;
            PCG_CK(cudaEventElapsedTime(&ms, evA, evB));
            *ms_out = hst[0].iter > 0 ? ms / hst[0].iter : -1.0;
            return;
        }
        const int K = check_every();
        cudaGraphExec_t ge = get_graph<TO, TP>(kind);
        const int nw = (warmup + K - 1) / K, nt = std::max(1, (iters + K - 1) / K);
        pcg_init<TO, TP>(kind, o.prhs, 0.0, (nw + nt) * K + 1, 0);
        for (int i = 0; i < nw; ++i) PCG_CK(cudaGraphLaunch(ge, s));
        PCG_CK(cudaMemcpyAsync(&hst[1], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        PCG_CK(cudaEventRecord(evA, s));
        for (int i = 0; i < nt; ++i) PCG_CK(cudaGraphLaunch(ge, s));
        PCG_CK(cudaEventRecord(evB, s));
        PCG_CK(cudaMemcpyAsync(&hst[0], st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        sync_check();
        float ms = 0.f;
        PCG_CK(cudaEventElapsedTime(&ms, evA, evB));
        const int done_iters = hst[0].iter - hst[1].iter;
        *ms_out = done_iters > 0 ? ms / done_iters : -1.0;
    }

    // Mean device time of one PCG iteration (rhs = D, tolerance 0: no early stop).
    void time_pcg(const double* Dd, int pc, int warmup, int iters, double* ms_out) {
        pc = resolve_pc(pc, n, m1);
        set_D(Dd, pc);
        const int kind = pc_kind(pc);
        if (use64) {
            convert1d<double, double>(m2, Dd, 1.0, o64.prhs, s);
            if (pc64) time_pcg_t<double, double>(kind, warmup, iters, ms_out);
            else time_pcg_t<double, float>(kind, warmup, iters, ms_out);
        } else {
            convert1d<double, float>(m2, Dd, 1.0, o32.prhs, s);
            time_pcg_t<float, float>(kind, warmup, iters, ms_out);
        }
    }

    // Algorithmic bytes of one PCG iteration (the per-iteration traffic of
    // Table tab:costs with dense operands): C' p and C y stream C twice; the K0
    // solve streams M0 (pcg_form 0), or the two triangles of R^{-1} and Et twice
    // (pcg_form 2 and the per-phase kernels), or B and B' replace all three
    // (pcg_form 1); P_H streams P~^{-1} (FP32) or the two triangles of its inverse
    // factor (FP64); plus the vector traffic.
    double bytes_per_iter(int pc) const {
        pc = resolve_pc(pc, n, m1);
        const double eo = use64 ? 8.0 : 4.0, ep = pc64 ? 8.0 : 4.0;
        const bool fused = use_fused();
        double bo = 2.0 * m2 * n + (double)n * (n + 1) + 2.0 * m1 * n;   // C', the factor's triangles, C
        if (fused && opt.pcg_form == 1) bo = 2.0 * (n + m1) * m2;         // B and B'
        if (fused && opt.pcg_form == 0) bo = 2.0 * m2 * n + (double)n * n;   // C', M0, C
        if (fused && opt.pcg_form == 3) bo = 2.0 * m2 * (n - m1);             // V' and V
        if (fused && crp && (opt.pcg_form == 0 || opt.pcg_form == 2))   // C and C' in CSR: values, plus 4-byte indices and row pointers
            bo += -2.0 * m2 * n + 2.0 * nnz * (1.0 + 4.0 / eo) + (m2 + n + 2) * 4.0 / eo;
        double bp = 0.0;
        if (pc_kind(pc) == PC_H_K) bp = (fused && !pc64) ? (double)m2 * m2 : (double)m2 * (m2 + 1);
        const double vec_el = 12.0 * m2 + 8.0 * n + 4.0 * m1;
        return bo * eo + bp * ep + vec_el * eo;
    }

    void kf_apply(const double* Dd, const double* p, double* q) {
        if (use64) kf_apply_t<double>(Dd, p, q); else kf_apply_t<float>(Dd, p, q);
    }
    template <typename TO>
    void kf_apply_t(const double* Dd, const double* p, double* q) {
        Op<TO>& o = op<TO>();
        convert1d<double, TO>(m2, Dd, 1.0, o.pD, s);
        convert1d<double, TO>(m2, p, 1.0, o.pp, s);
        kf_apply_dev<TO>(o.pp, o.pq, o.pD, nullptr);
        convert1d<TO, double>(m2, o.pq, 1.0, q, s);
        sync_check();
    }

    void k0_solve(const double* u, const double* w, double* a, double* bout) {
        if (use64) k0_solve_t<double>(u, w, a, bout); else k0_solve_t<float>(u, w, a, bout);
    }
    template <typename TO>
    void k0_solve_t(const double* u, const double* w, double* a, double* bout) {
        Op<TO>& o = op<TO>();
        convert1d<double, TO>(n, u, 1.0, o.ku, s);
        if (w && m1) convert1d<double, TO>(m1, w, 1.0, o.kw, s);
        k0_solve_dev<TO>(o.ku, (w && m1) ? o.kw : nullptr, o.ka, m1 ? o.kmb : nullptr);
        convert1d<TO, double>(n, o.ka, 1.0, a, s);
        if (bout && m1) convert1d<TO, double>(m1, o.kmb, -1.0, bout, s);
        sync_check();
    }

    // ------------------------------------------------- reduced Newton solve
    // Solve K^{(k)} [dx; dlam; dnu] = [f_g; f_e; f_a] (eq. [augmented]) through the
    // reduced system with the operator of precision TO:
    //   K_F dnu = f_a - [C 0] K0^{-1} [-f_g; f_e]      (eq. [ineq-const-reduced], K0 form)
    //   K0 [dx; -dlam] = [C' dnu - f_g; f_e]           (eq. [schur-delta-x], K0 form)
    // Inputs and outputs FP64; the right-hand side is scaled to unit norm inside
    // (the system is linear) so the working precision never under- or overflows.
    template <typename TO, typename TP>
    int reduced_solve_t(const double* gg, const double* ge_, const double* ga, double* ox, double* ol, double* on,
                        int kind, double tol, int maxit, double rhs_norm) {
        Op<TO>& o = op<TO>();
        const double inv = 1.0 / rhs_norm;
        convert1d<double, TO>(n, gg, -inv, o.ku, s);
        if (m1) convert1d<double, TO>(m1, ge_, inv, o.kw, s);
        k0_solve_dev<TO>(o.ku, m1 ? o.kw : nullptr, o.ka, nullptr);
        convert1d<double, TO>(m2, ga, inv, o.wa, s);
        launch_gemv<TO, TRI_NONE>(o.CW.p, m2, n, o.CW.ld, o.ka, EpiRnu<TO>{o.prhs, o.wa}, nullptr, nullptr, s);  // a5
        PCG_CK(cudaEventRecord(evA, s));
        pcg_init<TO, TP>(kind, o.prhs, tol, maxit, stall_window(kind));
        pcg_run<TO, TP>(kind, maxit);
        if (hst[0].done == 3 && kind != PC_L_K) {
            // non-finite PCG with the factored preconditioner: redo this solve with P_L
            if (verbose) std::fprintf(stderr, "    PCG non-finite with kind %d: retry with P_L\n", kind);
            pcg_init<TO, TP>(PC_L_K, o.prhs, tol, maxit, stall_window(PC_L_K));
            pcg_run<TO, TP>(PC_L_K, maxit);
        }
        PCG_CK(cudaEventRecord(evB, s));
        // recovery (a11)
        convert1d<double, TO>(n, gg, inv, o.wg, s);
        launch_gemv<TO, TRI_NONE>(o.CWT.p, n, m2, o.CWT.ld, o.px, lin<TO>(o.ku, TO(1), o.wg, TO(-1)), nullptr, nullptr, s);
        k0_solve_dev<TO>(o.ku, m1 ? o.kw : nullptr, o.ka, m1 ? o.kmb : nullptr);
        convert1d<TO, double>(n, o.ka, rhs_norm, ox, s);
        if (m1) convert1d<TO, double>(m1, o.kmb, rhs_norm, ol, s);
        convert1d<TO, double>(m2, o.px, rhs_norm, on, s);
        PCG_CK(cudaEventSynchronize(evB));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, evA, evB);
        stats.t_pcg_ms += ms;
        stats.newton_solves += 1;
        if (std::is_same<TO, double>::value && !f64) stats.op64_solves += 1;
        stats.pcg_iters_total += hst[0].iter;
        last_pcg_done = hst[0].done;
        last_pcg_rel = hst[0].bb > 0 ? std::sqrt(hst[0].rr / hst[0].bb) : 0.0;
        // a breakdown (done == 3) leaves the last finite iterate in place: it is returned
        // like a stagnated solve; the FP64 residual of the caller decides what it is worth
        return hst[0].iter;
    }

    int reduced_solve(const double* gg, const double* ge_, const double* ga, double* ox, double* ol, double* on,
                      int kind, double tol, int maxit, double rhs_norm) {
        if (!(rhs_norm > 0.0)) {   // zero right-hand side: zero direction
            axpby<double, double>(n, 0.0, gg, 0.0, ox, s);
            if (m1) axpby<double, double>(m1, 0.0, ge_, 0.0, ol, s);
            axpby<double, double>(m2, 0.0, ga, 0.0, on, s);
            return 0;
        }
        if (use64) {
            if (pc64) return reduced_solve_t<double, double>(gg, ge_, ga, ox, ol, on, kind, tol, maxit, rhs_norm);
            return reduced_solve_t<double, float>(gg, ge_, ga, ox, ol, on, kind, tol, maxit, rhs_norm);
        }
        return reduced_solve_t<float, float>(gg, ge_, ga, ox, ol, on, kind, tol, maxit, rhs_norm);
    }

    // rho = f - K^{(k)} z in FP64; returns |rho|_2^2 (eq. [augmented], D = s / nu).
    double kkt3_residual(const double* zx, const double* zl, const double* zn) {
        launch_gemv<double, TRI_NONE>(H.p, n, n, H.ld, zx, lin<double>(rho_g, 1.0, fg, 1.0), nullptr, nullptr, s);
        if (m1) launch_gemv<double, TRI_NONE>(AT.p, n, m1, AT.ld, zl, lin<double>(rho_g, -1.0, rho_g, 1.0), nullptr, nullptr, s);
        launch_gemv<double, TRI_NONE>(CT.p, n, m2, CT.ld, zn, lin<double>(rho_g, -1.0, rho_g, 1.0), nullptr, nullptr, s);
        if (m1) launch_gemv<double, TRI_NONE>(A.p, m1, n, A.ld, zx, lin<double>(rho_e, -1.0, fe, 1.0), nullptr, nullptr, s);
        launch_gemv<double, TRI_NONE>(C.p, m2, n, C.ld, zx,
                                      lin<double>(rho_a, -1.0, fa, 1.0, nullptr, 0.0, D64, zn, -1.0), nullptr, nullptr, s);
        return sumsq3(rho_g, rho_e, rho_a);
    }

    double sumsq3(const double* a, const double* bb, const double* cc) {
        norms_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, a, part_a, part_b);
        if (m1) norms_kernel<<<vec_grid(m1), kVecThreads, 0, s>>>(m1, bb, part_c, part_b);
        norms_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, cc, part_d, part_b);
        ReduceJob job{};
        job.part[0] = part_a; job.cnt[0] = vec_grid(n); job.op[0] = 0;
        job.part[1] = part_c; job.cnt[1] = m1 ? vec_grid(m1) : 0; job.op[1] = 0;
        job.part[2] = part_d; job.cnt[2] = vec_grid(m2); job.op[2] = 0;
        job.njobs = 3;
        reduce_jobs_kernel<<<1, kVecThreads, 0, s>>>(job, d_scal);
        PCG_CK(cudaMemcpyAsync(h_scal, d_scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        wait_stream();
        return h_scal[0] + (m1 ? h_scal[1] : 0.0) + h_scal[2];
    }

    // QP_PC_AUTO: move a QP from P_L to the exact P_H for the rest of its IPM
    // iterations.  Late in the IPM the non-unit eigenvalues 1 + lambda(X) of
    // P_L^{-1} K_F grow without bound as entries of D = V^{-1}S go to zero (Sec. 4.3,
    // Theorem 1) and PCG stops converging; P_H^{-1} K_F keeps its spectrum in (0, 1]
    // (Theorem 2).
    void switch_to_ph() {
        ipm_pc = QP_PC_PH_EXACT;
        stats.precond_used = ipm_pc;
        stats.pc_switch_iter = ipm_k;
        if (verbose) std::fprintf(stderr, "  preconditioner P_L -> P_H at IPM iteration %d\n", ipm_k);
        set_D(D64, ipm_pc);
    }

    // Move the operator to FP64 for the rest of the QP (mixed precision mode).
    void switch_to_op64() {
        if (use64) return;
        factor_op<double>();
        use64 = true;
        set_D_op<double>(D64);
        stats.op64_switch_iter = ipm_k;
        if (verbose) std::fprintf(stderr, "  operator -> FP64 at IPM iteration %d\n", ipm_k);
    }

    // Newton direction for the rhs (fg, fe, fa) already in place; result in (ox, ol, on).
    // PARITY mode refines against the FP64 residual of the 3x3 system.  With the FP32
    // operator a sweep contracts by about max(PCG tolerance, operator error); the next
    // corrections are then solved only to half that contraction (and never tighter than
    // a tenth of the reduction still needed), and a contraction worse than 1/4 (or a
    // correction that increases the residual) moves the QP to the FP64 operator.
    int newton_solve(double* ox, double* ol, double* on) {
        const int kind = pc_kind(ipm_pc);
        const bool paper = (opt.pcg_mode == QP_MODE_PAPER);
        const int maxit = opt.max_pcg > 0 ? opt.max_pcg : 4 * m2 + 50;
        auto base_tol = [&]() {
            double t = opt.pcg_tol;
            if (t <= 0) t = paper ? 1e-3 : (use64 ? 1e-10 : 1e-6);
            return t;
        };
        const double fnorm2 = sumsq3(fg, fe, fa);
        int it = reduced_solve(fg, fe, fa, ox, ol, on, kind, base_tol(), maxit, std::sqrt(fnorm2));
        if (verbose) std::fprintf(stderr, "    solve: |f|=%.3e pcg=%d done=%d rel=%.2e op64=%d\n", std::sqrt(fnorm2),
                                  it, last_pcg_done, last_pcg_rel, (int)use64);
        if (it < 0) return QP_ENUMERIC;
        if (opt.precond == QP_PC_AUTO && kind == PC_L_K && last_pcg_done >= 2 && last_pcg_rel > base_tol()) {
            // P_L ran out of iterations, broke down or stagnated: redo with P_H
            switch_to_ph();
            return newton_solve(ox, ol, on);
        }
        if (paper) return QP_OK;
        long long iters32 = use64 ? 0 : it;   // this direction's PCG iterations with the FP32 operator
        double prev = kkt3_residual(ox, ol, on);
        const double rtol2 = opt.refine_tol * opt.refine_tol * fnorm2;
        if (verbose) std::fprintf(stderr, "      refine 0: |rho|/|f|=%.3e\n", std::sqrt(prev / fnorm2));
        double last = fnorm2;
        int budget = opt.refine_max;
        for (int sweep = 0; sweep < budget && prev > rtol2; ++sweep) {
            const double contraction = std::sqrt(prev / last);
            if (!use64 && allow_pc64 && sweep > 0 && contraction > 0.25) {
                switch_to_op64();
                budget = sweep + opt.refine_max;   // fresh sweeps with the FP64 operator
            }
            double ctol = base_tol();
            if (!use64 && opt.pcg_tol <= 0) ctol = std::min(1e-1, std::max(ctol, 0.5 * contraction));
            // A correction only has to take the residual to the refinement target: solve it
            // to a tenth of the reduction still needed (the last sweep of an FP64 direction
            // then runs at about 1e-4 instead of 1e-10).
            if (opt.pcg_tol <= 0) ctol = std::min(1e-1, std::max(ctol, 0.1 * std::sqrt(rtol2 / prev)));
            last = prev;
            it = reduced_solve(rho_g, rho_e, rho_a, tx, tl, tn, kind, ctol, maxit, std::sqrt(prev));
            if (it < 0) return QP_ENUMERIC;
            if (!use64) iters32 += it;
            axpby<double, double>(n, 1.0, tx, 1.0, ox, s);
            if (m1) axpby<double, double>(m1, 1.0, tl, 1.0, ol, s);
            axpby<double, double>(m2, 1.0, tn, 1.0, on, s);
            stats.refine_sweeps += 1;
            const double r2 = kkt3_residual(ox, ol, on);
            if (verbose) std::fprintf(stderr, "      refine %d: pcg=%d done=%d rel=%.2e |rho|/|f|=%.3e op64=%d\n",
                                      sweep + 1, it, last_pcg_done, last_pcg_rel, std::sqrt(r2 / fnorm2), (int)use64);
            if (r2 > prev) {
                // the correction made it worse: undo it; with the FP32 operator move to FP64
                axpby<double, double>(n, -1.0, tx, 1.0, ox, s);
                if (m1) axpby<double, double>(m1, -1.0, tl, 1.0, ol, s);
                axpby<double, double>(m2, -1.0, tn, 1.0, on, s);
                if (use64 || !allow_pc64) break;
                kkt3_residual(ox, ol, on);     // restore rho for the next correction
                switch_to_op64();
                budget = sweep + 1 + opt.refine_max;
                last = prev;
                continue;
            }
            prev = r2;
        }
        // Corollaries 1 and 2 bound CG by n - m1 + 1 (P_L) or m1 + 1 (P_H) iterations in
        // exact arithmetic.  Far beyond that, rounding drives the count (late in the IPM
        // P_L's spectrum grows without bound, Theorem 1), and FP32 CG needs several times
        // the FP64 iterations per direction -- more than its cheaper iterations repay:
        // the QP's later directions use the FP64 operator.
        const long long bound = (kind == PC_L_K) ? (long long)(n - m1 + 1) : (kind == PC_H_K) ? (long long)(m1 + 1) : m2;
        if (!use64 && allow_pc64 && opt.pcg_tol <= 0 && iters32 > kCgExcess * bound) {
            if (verbose) std::fprintf(stderr, "  %lld FP32 PCG iterations for one direction (bound %lld)\n", iters32, bound);
            switch_to_op64();
        }
        return QP_OK;
    }
    // FP32 CG iterations per direction, in units of the exact-arithmetic bound, beyond
    // which the mixed path moves to the FP64 operator (n=3000 few-dof workload: from
    // IPM iteration 14 on, where an FP32 direction took about 20,000 iterations against
    // 7,000 in FP64 at three times the cost per iteration).
    static constexpr long long kCgExcess = 32;

    // -------------------------------------------------------------------- IPM
    // |r_g|_inf, |r_e|_inf, |r_i|_inf, s'nu, x'Hx, c'x at the current iterate.
    void residuals(double* out6) {
        launch_gemv<double, TRI_NONE>(H.p, n, n, H.ld, x, lin<double>(hx), nullptr, nullptr, s);
        // r_g = -Hx - c + A'lam + C'nu ; r_e = Ax - b ; r_i = Cx - d - s  (eq. [rhs-KKT4])
        launch_gemv<double, TRI_NONE>(CT.p, n, m2, CT.ld, nu, lin<double>(rg, 1.0, hx, -1.0, c, -1.0), nullptr, nullptr, s);
        if (m1) launch_gemv<double, TRI_NONE>(AT.p, n, m1, AT.ld, lam, lin<double>(rg, 1.0, rg, 1.0), nullptr, nullptr, s);
        if (m1) launch_gemv<double, TRI_NONE>(A.p, m1, n, A.ld, x, lin<double>(re, 1.0, b, -1.0), nullptr, nullptr, s);
        launch_gemv<double, TRI_NONE>(C.p, m2, n, C.ld, x, lin<double>(ri, 1.0, d, -1.0, sl, -1.0), nullptr, nullptr, s);
        norms_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, rg, part_a, part_b);
        if (m1) norms_kernel<<<vec_grid(m1), kVecThreads, 0, s>>>(m1, re, part_a, part_c);
        norms_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, ri, part_a, part_d);
        dot_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, sl, nu, part_e);
        dot_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, x, hx, part_f);
        dot_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(n, x, c, part_bb);
        ReduceJob job{};
        job.part[0] = part_b; job.cnt[0] = vec_grid(n); job.op[0] = 1;
        job.part[1] = part_c; job.cnt[1] = m1 ? vec_grid(m1) : 0; job.op[1] = 1;
        job.part[2] = part_d; job.cnt[2] = vec_grid(m2); job.op[2] = 1;
        job.part[3] = part_e; job.cnt[3] = vec_grid(m2); job.op[3] = 0;
        job.part[4] = part_f; job.cnt[4] = vec_grid(n); job.op[4] = 0;
        job.part[5] = part_bb; job.cnt[5] = vec_grid(n); job.op[5] = 0;
        job.njobs = 6;
        reduce_jobs_kernel<<<1, kVecThreads, 0, s>>>(job, d_scal);
        PCG_CK(cudaMemcpyAsync(h_scal, d_scal, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
        sync_check();
        for (int k = 0; k < 6; ++k) out6[k] = h_scal[k];
        if (!m1) out6[1] = 0.0;
    }

    double reduce1(const double* part, int cnt, int opk) {
        ReduceJob job{};
        job.part[0] = part; job.cnt[0] = cnt; job.op[0] = opk; job.njobs = 1;
        reduce_jobs_kernel<<<1, kVecThreads, 0, s>>>(job, d_scal);
        PCG_CK(cudaMemcpyAsync(h_scal, d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        sync_check();
        return h_scal[0];
    }

    double max_step(const double* s_, const double* ds_, const double* nu_, const double* dnu_) {
        ipm_maxstep_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, s_, ds_, nu_, dnu_, part_a);
        return reduce1(part_a, vec_grid(m2), 2);
    }

    double mu_aff(double a) {
        ipm_muaff_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, sl, dsa, nu, dna, a, part_a);
        return reduce1(part_a, vec_grid(m2), 0) / m2;
    }

    // Start point: K0 [x; -lam] = [-c; b] refined in FP64, s = max(Cx - d, 1), nu = 1.
    template <typename TO>
    void start_point_t() {
        Op<TO>& o = op<TO>();
        constexpr bool is64 = std::is_same<TO, double>::value;
        convert1d<double, TO>(n, c, -1.0, o.ku, s);
        if (m1) convert1d<double, TO>(m1, b, 1.0, o.kw, s);
        k0_solve_dev<TO>(o.ku, m1 ? o.kw : nullptr, o.ka, m1 ? o.kmb : nullptr);
        convert1d<TO, double>(n, o.ka, 1.0, x, s);
        if (m1) convert1d<TO, double>(m1, o.kmb, 1.0, lam, s);
        for (int sweep = 0; sweep < (is64 ? 2 : 6); ++sweep) {
            // rho1 = -c - H x + A' lam ; rho2 = b - A x ; K0 [dx; -dlam] = [rho1; rho2]
            launch_gemv<double, TRI_NONE>(H.p, n, n, H.ld, x, lin<double>(rho_g, -1.0, c, -1.0), nullptr, nullptr, s);
            if (m1) {
                launch_gemv<double, TRI_NONE>(AT.p, n, m1, AT.ld, lam, lin<double>(rho_g, 1.0, rho_g, 1.0), nullptr, nullptr, s);
                launch_gemv<double, TRI_NONE>(A.p, m1, n, A.ld, x, lin<double>(rho_e, -1.0, b, 1.0), nullptr, nullptr, s);
                convert1d<double, TO>(m1, rho_e, 1.0, o.kw, s);
            }
            convert1d<double, TO>(n, rho_g, 1.0, o.ku, s);
            k0_solve_dev<TO>(o.ku, m1 ? o.kw : nullptr, o.ka, m1 ? o.kmb : nullptr);
            convert1d<TO, double>(n, o.ka, 1.0, tx, s);
            axpby<double, double>(n, 1.0, tx, 1.0, x, s);
            if (m1) {
                convert1d<TO, double>(m1, o.kmb, 1.0, tl, s);
                axpby<double, double>(m1, 1.0, tl, 1.0, lam, s);
            }
        }
        launch_gemv<double, TRI_NONE>(C.p, m2, n, C.ld, x, lin<double>(ri, 1.0, d, -1.0), nullptr, nullptr, s);
        ipm_start_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, ri, sl, nu);
    }

    int ipm_solve() {
        factor();
        const auto t0 = std::chrono::steady_clock::now();
        stats.ipm_iters = 0; stats.pcg_iters_total = 0; stats.newton_solves = 0; stats.refine_sweeps = 0;
        stats.t_pcg_ms = 0; stats.t_precond_ms = 0; stats.op64_solves = 0; stats.op64_switch_iter = -1;
        stats.pc64_switch_iter = -1; stats.pc_switch_iter = -1;
        use64 = f64 || all64;
        pc64 = f64 || all64;
        if (all64) { stats.op64_switch_iter = 0; stats.pc64_switch_iter = 0; }
        ipm_k = 0;
        ipm_pc = resolve_pc(opt.precond, n, m1);
        stats.precond_used = ipm_pc;
        if (use64) start_point_t<double>(); else start_point_t<float>();
        int status = QP_EMAXIT;
        int k = 0;
        const double tau = 0.995;
        while (true) {
            double r6[6];
            residuals(r6);
            const double res_p = std::max(r6[1] / (1.0 + b_inf), r6[2] / (1.0 + d_inf));
            const double res_d = r6[0] / (1.0 + c_inf + h_norm_inf);
            const double mu = r6[3] / m2;
            const double f = 0.5 * r6[4] + r6[5];
            stats.res_p = res_p; stats.res_d = res_d; stats.mu = mu; stats.obj = f;
            if (!std::isfinite(res_p) || !std::isfinite(res_d) || !std::isfinite(mu)) { status = QP_ENUMERIC; break; }
            if (res_p <= opt.tol_feas && res_d <= opt.tol_feas && mu <= opt.tol_mu * (1.0 + std::fabs(f))) {
                status = QP_OK;
                break;
            }
            if (k >= opt.max_ipm) break;
            ipm_k = k;
            // D = V^{-1}S, predictor r_c = S V e, r_a = r_i + V^{-1} r_c
            ipm_rc_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, sl, nu, ri, nullptr, nullptr, 0.0, rc, ra, D64);
            set_D(D64, ipm_pc);
            // right-hand side of eq. [augmented]: -(r_g, r_e, r_a)
            axpby<double, double>(n, -1.0, rg, 0.0, fg, s);
            if (m1) axpby<double, double>(m1, -1.0, re, 0.0, fe, s);
            axpby<double, double>(m2, -1.0, ra, 0.0, fa, s);
            int st_ = newton_solve(dxa, dla, dna);
            if (st_ != QP_OK) { status = st_; break; }
            ipm_ds_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, rc, nu, D64, dna, dsa);
            const double a_aff = std::min(1.0, max_step(sl, dsa, nu, dna));
            const double mua = mu_aff(a_aff);
            const double sigma = std::pow(mua / mu, 3.0);
            // corrector: r_c = S V e + dS_aff dV_aff e - sigma mu e
            ipm_rc_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, sl, nu, ri, dsa, dna, sigma * mu, rc, ra, nullptr);
            axpby<double, double>(m2, -1.0, ra, 0.0, fa, s);
            st_ = newton_solve(dx, dl, dn);
            if (st_ != QP_OK) { status = st_; break; }
            ipm_ds_kernel<<<vec_grid(m2), kVecThreads, 0, s>>>(m2, rc, nu, D64, dn, ds);
            const double alpha = std::min(1.0, tau * max_step(sl, ds, nu, dn));
            if (verbose)
                std::fprintf(stderr, "ipm %d: mu=%.3e res_p=%.3e res_d=%.3e f=%.10g a_aff=%.3e sigma=%.3e alpha=%.3e\n",
                             k, mu, res_p, res_d, f, a_aff, sigma, alpha);
            axpby<double, double>(n, alpha, dx, 1.0, x, s);
            if (m1) axpby<double, double>(m1, alpha, dl, 1.0, lam, s);
            axpby<double, double>(m2, alpha, dn, 1.0, nu, s);
            axpby<double, double>(m2, alpha, ds, 1.0, sl, s);
            ++k;
        }
        sync_check();
        stats.ipm_iters = k;
        stats.status = status;
        stats.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return status;
    }

    void copy_solution(double* xo, double* lo, double* no, double* so, bool to_host) {
        const cudaMemcpyKind kd = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (xo) PCG_CK(cudaMemcpyAsync(xo, x, (size_t)n * 8, kd, s));
        if (lo && m1) PCG_CK(cudaMemcpyAsync(lo, lam, (size_t)m1 * 8, kd, s));
        if (no) PCG_CK(cudaMemcpyAsync(no, nu, (size_t)m2 * 8, kd, s));
        if (so) PCG_CK(cudaMemcpyAsync(so, sl, (size_t)m2 * 8, kd, s));
        wait_stream();
    }
};

}  // namespace pcgipm
