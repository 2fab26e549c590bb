// server.cpp -- the serving layer (continuous batching) declared in include/pcgipm.h.
//
// Host code over the library's own C ABI: a FIFO of submitted QPs, a device-
// memory budget, and one worker thread per slot.  A worker admits the head of
// the queue once its qp_device_bytes_bound fits in what the budget has left,
// then creates, factors and solves that QP on the QP's own stream (its K0 factor
// and IPM state stay on the device for the whole solve), copies the solution to
// the request, destroys the handle and returns the bytes to the budget.  Several
// workers run at once, so the QPs in flight overlap on the GPU: their persistent
// PCG kernels, each sized by its QP's per-iteration bytes, share the SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "pcgipm.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    unsigned long long ticket = 0;
    int n = 0, m1 = 0, m2 = 0;
    bool csr = false;
    std::vector<double> H, c, A, b, C, Cval, d;
    std::vector<int> rowptr, colidx;
    size_t bound = 0;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    qp_result res{};
    std::vector<double> x, lam, nu, s;
};

}  // namespace

struct qp_server_s {
    std::mutex mu;
    std::condition_variable cv_work;   // queue changed, budget returned, or stopping
    std::condition_variable cv_done;   // a request finished
    std::deque<Request*> queue;
    std::map<unsigned long long, std::unique_ptr<Request>> tickets;
    size_t budget = 0, reserved = 0, peak_reserved = 0, peak_dev = 0;
    int active = 0;
    long long submitted = 0, completed = 0, failed = 0;
    unsigned long long next_ticket = 1;
    bool stopping = false;
    qp_opts opts{};
    int device = 0;
    std::vector<std::thread> workers;
};

namespace {

// Create, solve and release one admitted QP; the result lands in *r.
void run_one(qp_server_s* S, Request* r) {
    qp_t h = nullptr;
    const double* A = r->m1 ? r->A.data() : nullptr;
    const double* b = r->m1 ? r->b.data() : nullptr;
    int st;
    if (r->csr)
        st = qp_create_csr(&h, r->n, r->m1, r->m2, r->H.data(), r->c.data(), A, b, r->rowptr.data(),
                           r->colidx.data(), r->Cval.data(), r->d.data(), &S->opts, QP_PTR_HOST);
    else
        st = qp_create(&h, r->n, r->m1, r->m2, r->H.data(), r->c.data(), A, b, r->C.data(), r->d.data(),
                       &S->opts, QP_PTR_HOST);
    qp_result res{};
    res.status = st;
    if (st == QP_OK) {
        r->x.assign(r->n, 0.0);
        r->lam.assign(r->m1, 0.0);
        r->nu.assign(r->m2, 0.0);
        r->s.assign(r->m2, 0.0);
        double obj = 0.0;
        int it = 0;
        long long pit = 0;
        st = qp_ipm_solve(h, r->x.data(), r->m1 ? r->lam.data() : nullptr, r->nu.data(), r->s.data(), &obj, &it,
                          &pit, QP_PTR_HOST);
        qp_stats stt{};
        qp_get_stats(h, &stt);
        res.status = st;
        res.ipm_iters = stt.ipm_iters;
        res.pcg_iters = stt.pcg_iters_total;
        res.obj = stt.obj;
        res.res_p = stt.res_p;
        res.res_d = stt.res_d;
        res.mu = stt.mu;
        const size_t dev = qp_device_bytes(h);
        std::lock_guard<std::mutex> lk(S->mu);
        S->peak_dev = std::max(S->peak_dev, dev);
    }
    if (h) qp_destroy(h);
    // the problem data is no longer needed
    std::vector<double>().swap(r->H);
    std::vector<double>().swap(r->A);
    std::vector<double>().swap(r->C);
    std::vector<double>().swap(r->Cval);
    std::vector<int>().swap(r->rowptr);
    std::vector<int>().swap(r->colidx);
    r->res = res;
}

void worker(qp_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_work.wait(lk, [&]() {
            if (!S->queue.empty()) return S->reserved + S->queue.front()->bound <= S->budget;
            return S->stopping;
        });
        if (S->queue.empty()) break;   // stopping, nothing left
        Request* r = S->queue.front();
        S->queue.pop_front();
        S->reserved += r->bound;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        S->active += 1;
        r->t_admit = Clock::now();
        lk.unlock();
        run_one(S, r);
        const Clock::time_point t_done = Clock::now();
        lk.lock();
        r->t_done = t_done;
        r->res.wait_ms = ms_between(r->t_submit, r->t_admit);
        r->res.solve_ms = ms_between(r->t_admit, t_done);
        r->res.latency_ms = ms_between(r->t_submit, t_done);
        r->done = true;
        S->reserved -= r->bound;
        S->active -= 1;
        S->completed += 1;
        if (r->res.status != QP_OK) S->failed += 1;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

template <typename T>
void copy_in(std::vector<T>& dst, const T* src, size_t count) {
    dst.resize(count);
    if (count) std::memcpy(dst.data(), src, count * sizeof(T));
}

}  // namespace

extern "C" {

int qp_server_create(qp_server_t* out, size_t hbm_budget_bytes, int max_slots, const qp_opts* opts) {
    if (!out) return QP_EINVAL;
    *out = nullptr;
    if (max_slots < 0) return QP_EINVAL;
    qp_opts o;
    qp_opts_default(&o);
    if (opts) o = *opts;
    if (o.stream) return QP_EINVAL;
    if (o.precision != QP_PREC_FP32 && o.precision != QP_PREC_FP64) return QP_EINVAL;
    if (o.precond < QP_PC_AUTO || o.precond > QP_PC_NONE) return QP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QP_ECUDA;
    if (hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return QP_ECUDA;
        hbm_budget_bytes = free_b / 10 * 9;
    }
    std::unique_ptr<qp_server_s> S(new qp_server_s);
    S->budget = hbm_budget_bytes;
    S->opts = o;
    S->device = dev;
    const int slots = max_slots > 0 ? max_slots : 16;
    try {
        for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker, S.get());
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stopping = true;
        }
        S->cv_work.notify_all();
        for (auto& t : S->workers) t.join();
        return QP_ENOMEM;
    }
    *out = S.release();
    return QP_OK;
}

int qp_server_submit(qp_server_t S, const qp_problem* p, unsigned long long* ticket) {
    if (!S || !p || !ticket) return QP_EINVAL;
    const int n = p->n, m1 = p->m1, m2 = p->m2;
    if (n < 1 || m1 < 0 || m1 > n || m2 < 1) return QP_EINVAL;
    if (!p->H || !p->c || !p->d || (m1 > 0 && (!p->A || !p->b))) return QP_EINVAL;
    const bool csr = p->C_rowptr != nullptr;
    if (csr == (p->C != nullptr)) return QP_EINVAL;
    if (csr && (!p->C_colidx || !p->C_val)) return QP_EINVAL;
    std::unique_ptr<Request> r(new Request);
    try {
        r->n = n; r->m1 = m1; r->m2 = m2; r->csr = csr;
        copy_in(r->H, p->H, (size_t)n * n);
        copy_in(r->c, p->c, (size_t)n);
        copy_in(r->A, p->A, (size_t)m1 * n);
        copy_in(r->b, p->b, (size_t)m1);
        copy_in(r->d, p->d, (size_t)m2);
        if (csr) {
            const int nnz = p->C_rowptr[m2];
            if (nnz < 0) return QP_EINVAL;
            copy_in(r->rowptr, p->C_rowptr, (size_t)m2 + 1);
            copy_in(r->colidx, p->C_colidx, (size_t)nnz);
            copy_in(r->Cval, p->C_val, (size_t)nnz);
        } else {
            copy_in(r->C, p->C, (size_t)m2 * n);
        }
    } catch (const std::bad_alloc&) {
        return QP_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return QP_ESTATE;
    r->bound = qp_device_bytes_bound(n, m1, m2, &S->opts);
    if (r->bound > S->budget) return QP_ENOMEM;
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    *ticket = r->ticket;
    S->queue.push_back(r.get());
    S->tickets[r->ticket] = std::move(r);
    S->submitted += 1;
    S->cv_work.notify_all();
    return QP_OK;
}

int qp_server_poll(qp_server_t S, unsigned long long ticket, qp_result* res, double* x, double* lam, double* nu,
                   double* s) {
    if (!S) return QP_EINVAL;
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return QP_EINVAL;
        if (!it->second->done) return QP_EAGAIN;
        r = std::move(it->second);
        S->tickets.erase(it);
    }
    if (res) *res = r->res;
    auto out = [](double* dst, const std::vector<double>& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(double));
    };
    out(x, r->x);
    out(lam, r->lam);
    out(nu, r->nu);
    out(s, r->s);
    return QP_OK;
}

int qp_server_drain(qp_server_t S, double timeout_ms) {
    if (!S) return QP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto idle = [&]() { return S->queue.empty() && S->active == 0; };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, idle);
        return QP_OK;
    }
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), idle);
    return ok ? QP_OK : QP_ETIMEOUT;
}

int qp_server_get_stats(qp_server_t S, qp_server_stats* st) {
    if (!S || !st) return QP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->queued = (int)S->queue.size();
    st->active = S->active;
    st->reserved_bytes = S->reserved;
    st->peak_reserved_bytes = S->peak_reserved;
    st->peak_device_bytes = S->peak_dev;
    return QP_OK;
}

void qp_server_destroy(qp_server_t S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
}

}  // extern "C"
