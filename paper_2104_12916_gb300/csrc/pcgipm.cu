// pcgipm.cu -- C ABI of the GB300 preconditioned inexact IPM (declared in include/pcgipm.h).
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <cstdio>
#include <memory>
#include <thread>
#include <vector>

#include "engine.cuh"

using namespace pcgipm;

struct qp_s {
    std::unique_ptr<Engine> eng;
};

namespace {

int translate(const CudaError& e) {
    const char* v = std::getenv("PCGIPM_VERBOSE");
    if (v && v[0] == '1')
        std::fprintf(stderr, "pcgipm: CUDA error %d (%s) at engine.cuh:%d\n", (int)e.e, cudaGetErrorString(e.e), e.line);
    return QP_ECUDA;
}

template <class F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const QpError& e) {
        return e.code;
    } catch (const NoMem&) {
        return QP_ENOMEM;
    } catch (const CudaError& e) {
        return translate(e);
    } catch (const std::bad_alloc&) {
        return QP_ENOMEM;
    } catch (...) {
        return QP_ECUDA;
    }
}

// Copy `count` doubles from a caller buffer into a staging device vector (or
// return the caller's device pointer unchanged).
const double* stage_in(Engine* e, int slot, const double* p, int count, int ptr_kind) {
    if (!p) return nullptr;
    if (ptr_kind == QP_PTR_DEVICE) return p;
    PCG_CK(cudaMemcpyAsync(e->stage[slot], p, (size_t)count * 8, cudaMemcpyHostToDevice, e->s));
    return e->stage[slot];
}

double* stage_out(Engine* e, int slot, double* p, int ptr_kind) {
    if (!p) return nullptr;
    return ptr_kind == QP_PTR_DEVICE ? p : e->stage[slot];
}

void finish_out(Engine* e, int slot, double* p, int count, int ptr_kind) {
    if (!p || ptr_kind == QP_PTR_DEVICE) return;
    PCG_CK(cudaMemcpyAsync(p, e->stage[slot], (size_t)count * 8, cudaMemcpyDeviceToHost, e->s));
}

}  // namespace

extern "C" {

void qp_opts_default(qp_opts* o) {
    if (!o) return;
    o->precision = QP_PREC_FP32;
    o->precond = QP_PC_AUTO;
    o->pcg_mode = QP_MODE_PARITY;
    o->max_ipm = 100;
    o->max_pcg = 0;
    o->refine_max = 5;
    o->pcg_tol = 0.0;
    o->refine_tol = 1e-11;
    o->tol_feas = 1e-10;
    o->tol_mu = 1e-11;
    o->pcg_check_every = 8;
    o->mixed_fallback = 1;
    o->pcg_blocks = 0;
    o->blocking_wait = 0;
    o->pcg_form = QP_FORM_AUTO;
    o->factor_tc = 0;
    o->autotune = 1;
    o->factor_bk = 0;
    o->stream = nullptr;
}

static int create_common(qp_t* out, int n, int m1, int m2, const double* H, const double* c, const double* A,
                         const double* b, const double* C, const Engine::CsrIn* csr, const double* d,
                         const qp_opts* opts, int ptr_kind) {
    if (!out) return QP_EINVAL;
    *out = nullptr;
    if (n < 1 || m1 < 0 || m1 > n || m2 < 1) return QP_EINVAL;
    if (!H || !c || (!C && !csr) || !d || (m1 > 0 && (!A || !b))) return QP_EINVAL;
    if (ptr_kind != QP_PTR_HOST && ptr_kind != QP_PTR_DEVICE) return QP_EINVAL;
    qp_opts o;
    qp_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != QP_PREC_FP32 && o.precision != QP_PREC_FP64) return QP_EINVAL;
    if (o.precond < QP_PC_AUTO || o.precond > QP_PC_NONE) return QP_EINVAL;
    if (o.pcg_form < QP_FORM_AUTO || o.pcg_form > 3) return QP_EINVAL;
    return guarded([&]() {
        std::unique_ptr<qp_s> h(new qp_s);
        h->eng.reset(new Engine(n, m1, m2, o, csr != nullptr));
        h->eng->load(H, c, A, b, C, d, ptr_kind, csr);
        *out = h.release();
        return QP_OK;
    });
}

int qp_create(qp_t* out, int n, int m1, int m2, const double* H, const double* c, const double* A,
              const double* b, const double* C, const double* d, const qp_opts* opts, int ptr_kind) {
    if (!C) return QP_EINVAL;
    return create_common(out, n, m1, m2, H, c, A, b, C, nullptr, d, opts, ptr_kind);
}

int qp_create_csr(qp_t* out, int n, int m1, int m2, const double* H, const double* c, const double* A,
                  const double* b, const int* C_rowptr, const int* C_colidx, const double* C_val,
                  const double* d, const qp_opts* opts, int ptr_kind) {
    if (!C_rowptr || !C_colidx || !C_val) {
        if (out) *out = nullptr;
        return QP_EINVAL;
    }
    const Engine::CsrIn csr{C_rowptr, C_colidx, C_val};
    return create_common(out, n, m1, m2, H, c, A, b, nullptr, &csr, d, opts, ptr_kind);
}

size_t qp_device_bytes_bound(int n, int m1, int m2, const qp_opts* opts) {
    if (n < 1 || m1 < 0 || m1 > n || m2 < 1) return 0;
    qp_opts o;
    qp_opts_default(&o);
    if (opts) o = *opts;
    return Engine::bytes_bound(n, m1, m2, o);
}

int qp_factor_K0(qp_t qp) {
    if (!qp) return QP_EINVAL;
    return guarded([&]() {
        qp->eng->factor();
        return QP_OK;
    });
}

int qp_kf_apply(qp_t qp, const double* D, const double* p, double* q, int ptr_kind) {
    if (!qp || !D || !p || !q) return QP_EINVAL;
    if (!qp->eng->factored) return QP_ESTATE;
    return guarded([&]() {
        Engine* e = qp->eng.get();
        const double* Dd = stage_in(e, 0, D, e->m2, ptr_kind);
        const double* pd = stage_in(e, 1, p, e->m2, ptr_kind);
        double* qd = stage_out(e, 2, q, ptr_kind);
        e->kf_apply(Dd, pd, qd);
        finish_out(e, 2, q, e->m2, ptr_kind);
        PCG_CK(cudaStreamSynchronize(e->s));
        return QP_OK;
    });
}

int qp_k0_solve(qp_t qp, const double* u, const double* w, double* a, double* bo, int ptr_kind) {
    if (!qp || !u || !a) return QP_EINVAL;
    if (!qp->eng->factored) return QP_ESTATE;
    return guarded([&]() {
        Engine* e = qp->eng.get();
        const double* ud = stage_in(e, 0, u, e->n, ptr_kind);
        const double* wd = e->m1 ? stage_in(e, 1, w, e->m1, ptr_kind) : nullptr;
        double* ad = stage_out(e, 2, a, ptr_kind);
        double* bd = e->m1 ? stage_out(e, 3, bo, ptr_kind) : nullptr;
        e->k0_solve(ud, wd, ad, bd);
        finish_out(e, 2, a, e->n, ptr_kind);
        if (e->m1) finish_out(e, 3, bo, e->m1, ptr_kind);
        PCG_CK(cudaStreamSynchronize(e->s));
        return QP_OK;
    });
}

int qp_pcg_reduced_solve(qp_t qp, const double* D, const double* rhs, double* dnu, int precond, double tol,
                         int maxit, int* iters, double* relres, int ptr_kind) {
    if (!qp || !D || !rhs || !dnu) return QP_EINVAL;
    if (precond < QP_PC_AUTO || precond > QP_PC_NONE || maxit < 0) return QP_EINVAL;
    if (!qp->eng->factored) return QP_ESTATE;
    return guarded([&]() {
        Engine* e = qp->eng.get();
        const double* Dd = stage_in(e, 0, D, e->m2, ptr_kind);
        const double* rd = stage_in(e, 1, rhs, e->m2, ptr_kind);
        double* od = stage_out(e, 2, dnu, ptr_kind);
        const int st = e->pcg_solve(Dd, rd, od, precond, tol, maxit, iters, relres);
        finish_out(e, 2, dnu, e->m2, ptr_kind);
        PCG_CK(cudaStreamSynchronize(e->s));
        return st;
    });
}

int qp_ipm_solve(qp_t qp, double* x, double* lam, double* nu, double* s, double* obj, int* ipm_iters,
                 long long* pcg_iters_total, int ptr_kind) {
    if (!qp) return QP_EINVAL;
    return guarded([&]() {
        Engine* e = qp->eng.get();
        const int st = e->ipm_solve();
        e->copy_solution(x, lam, nu, s, ptr_kind == QP_PTR_HOST);
        if (obj) *obj = e->stats.obj;
        if (ipm_iters) *ipm_iters = e->stats.ipm_iters;
        if (pcg_iters_total) *pcg_iters_total = e->stats.pcg_iters_total;
        return st;
    });
}

int qp_batch_solve(qp_t* qps, int count, int max_concurrent, qp_result* results) {
    if (!qps || count < 0 || !results) return QP_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!qps[i] || !qps[i]->eng->own_stream) return QP_EINVAL;
    if (count == 0) return QP_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QP_ECUDA;
    const int workers = std::max(1, std::min(count, max_concurrent > 0 ? max_concurrent : 16));
    std::atomic<int> next(0);
    auto work = [&]() {
        cudaSetDevice(dev);
        while (true) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            Engine* e = qps[i]->eng.get();
            qp_result r{};
            const auto t0 = std::chrono::steady_clock::now();
            r.status = guarded([&]() { return e->ipm_solve(); });
            r.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            r.ipm_iters = e->stats.ipm_iters;
            r.pcg_iters = e->stats.pcg_iters_total;
            r.obj = e->stats.obj;
            r.res_p = e->stats.res_p;
            r.res_d = e->stats.res_d;
            r.mu = e->stats.mu;
            r.wait_ms = 0.0;
            r.latency_ms = r.solve_ms;
            results[i] = r;
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < count; ++i)
        if (results[i].status != QP_OK) return results[i].status;
    return QP_OK;
}

int qp_get_solution(qp_t qp, double* x, double* lam, double* nu, double* s, int ptr_kind) {
    if (!qp) return QP_EINVAL;
    return guarded([&]() {
        qp->eng->copy_solution(x, lam, nu, s, ptr_kind == QP_PTR_HOST);
        return QP_OK;
    });
}

int qp_get_stats(qp_t qp, qp_stats* st) {
    if (!qp || !st) return QP_EINVAL;
    *st = qp->eng->stats;
    return QP_OK;
}

size_t qp_device_bytes(qp_t qp) { return qp ? qp->eng->arena.bytes() : 0; }

double qp_pcg_bytes_per_iter(qp_t qp, int precond) { return qp ? qp->eng->bytes_per_iter(precond) : 0.0; }

int qp_time_pcg_iteration(qp_t qp, const double* D, int precond, int warmup, int iters, double* ms_per_iter,
                          int ptr_kind) {
    if (!qp || !D || !ms_per_iter || iters < 1 || warmup < 0) return QP_EINVAL;
    if (!qp->eng->factored) return QP_ESTATE;
    return guarded([&]() {
        Engine* e = qp->eng.get();
        const double* Dd = stage_in(e, 0, D, e->m2, ptr_kind);
        e->time_pcg(Dd, precond, warmup, iters, ms_per_iter);
        return QP_OK;
    });
}

unsigned long long qp_kernel_launches(void) {
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return 0;
    if (cudaMemcpyFromSymbol(&v, pcgipm::g_kernel_launches, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

void qp_destroy(qp_t qp) {
    if (!qp) return;
    try {
        cudaStreamSynchronize(qp->eng->s);
        delete qp;
    } catch (...) {
    }
}

const char* qp_strerror(int st) {
    switch (st) {
        case QP_OK: return "ok";
        case QP_EINVAL: return "invalid argument (dimension, NULL pointer, non-finite or asymmetric input)";
        case QP_ENOMEM: return "device allocation failed";
        case QP_ESINGULAR: return "A H^-1 A' has a non-positive pivot (A rank-deficient)";
        case QP_ENOTCONVEX: return "H has a non-positive pivot (not positive definite)";
        case QP_EMAXIT: return "iteration limit reached";
        case QP_ENUMERIC: return "non-finite value during the iteration";
        case QP_ETIMEOUT: return "bounded device wait expired";
        case QP_EAGAIN: return "result not ready";
        case QP_ECUDA: return "CUDA runtime error";
        case QP_ESTATE: return "call out of order (factor first)";
        default: return "unknown status";
    }
}

}  // extern "C"
