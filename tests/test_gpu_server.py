"""The serving layer (qp_server_*), CSR input and the device-memory bound.

Requests of the served workload's recipe (sparse C with 8 nonzeros per row, m1
and m2 drawn as fractions of n) at sizes the CPU oracle finishes quickly.  The
server must give each QP the same solution as solving it alone (every reduction
runs in a fixed order within its QP and the PCG grid depends only on the QP's
size, so the two are bit-identical), match the FP64 oracle, and keep the bytes
it admits within its budget.
"""
import math
import time

import numpy as np
import pytest

import qpgen
from oracle import ipm

pytestmark = pytest.mark.gpu


def _requests(count, seed0=700):
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(math.exp(rng.uniform(math.log(24), math.log(140)))))
        m1 = max(1, int(n * rng.uniform(0.05, 0.9)))
        m2 = max(1, int(n * rng.uniform(1.0, 3.0)))
        out.append(qpgen.dense_qp(n, m1, m2, seed=seed0 + 1000 + i, lam_lo=1e-2, lam_hi=1e2, c_sparse_nnz=8,
                                  name=f"req{i}_n{n}_m1_{m1}_m2_{m2}"))
    return out


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _solve_alone(B, q, opts):
    rp, ci, val = q.C_csr
    h = B.qp_create_csr(np.ascontiguousarray(q.H), q.c, q.A if q.m1 else None, q.b if q.m1 else None,
                        rp, ci, val, q.d, opts)
    try:
        x = np.zeros(q.n)
        st, f, its, _ = B.qp_ipm_solve(h, x, allow=(B.QP_OK, B.QP_EMAXIT, B.QP_ENUMERIC))
        return st, f, its, x
    finally:
        B.qp_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_csr_create_matches_dense_create(B, prec):
    """A CSR C is applied in the persistent kernel as sparse row sums (C' p and
    C y over the 8 nonzeros of a row), a dense C as streamed rows: the same
    operator with different rounding, so both reach the oracle's optimum."""
    q = _requests(1, seed0=42)[0]
    ref = ipm.solve_qp(q, variant="kkt3")
    o = B.qp_opts_default()
    o.precision = prec
    hd = B.QP(np.ascontiguousarray(q.H), q.c, q.A, q.b, np.ascontiguousarray(q.C_dense()), q.d, o)
    st, f, its, x = _solve_alone(B, q, o)
    xd = np.zeros(q.n)
    std, fd, itsd, _ = B.qp_ipm_solve(hd.h, xd)
    assert st == std == B.QP_OK
    for ff, ii in ((f, its), (fd, itsd)):
        assert abs(ff - ref.f) / max(abs(ref.f), 1.0) <= 1e-6
        assert abs(ii - ref.iters) <= 2
    assert np.linalg.norm(x - xd) <= 1e-5 * max(1.0, np.linalg.norm(xd))
    hd.close()


def test_csr_rejects_bad_pattern(B):
    q = _requests(1, seed0=43)[0]
    rp, ci, val = q.C_csr
    bad = np.array(ci, dtype=np.int32).copy()
    bad[3] = q.n                          # column out of range
    with pytest.raises(B.QPError) as e:
        B.qp_create_csr(np.ascontiguousarray(q.H), q.c, q.A, q.b, rp, bad, val, q.d)
    assert e.value.status == B.QP_EINVAL
    rp2 = np.array(rp, dtype=np.int32).copy()
    rp2[1], rp2[2] = rp2[2], rp2[1]      # decreasing row pointer
    with pytest.raises(B.QPError) as e:
        B.qp_create_csr(np.ascontiguousarray(q.H), q.c, q.A, q.b, rp2, ci, val, q.d)
    assert e.value.status == B.QP_EINVAL


@pytest.mark.parametrize("prec,pc", [(1, 0), (0, 0), (1, 1), (0, 2)])
def test_device_bytes_within_bound(B, prec, pc):
    for q in _requests(3, seed0=60 + 7 * prec + pc):
        o = B.qp_opts_default()
        o.precision, o.precond = prec, pc
        bound = B.qp_device_bytes_bound(q.n, q.m1, q.m2, o)
        h = B.QP.from_qpgen(q, o)
        B.qp_ipm_solve(h.h, allow=(B.QP_OK, B.QP_EMAXIT, B.QP_ENUMERIC))
        used = B.qp_device_bytes(h.h)
        assert 0 < used <= bound, (q.name, used, bound)
        h.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_server_results_same_alone_and_in_mix(B, prec):
    qps = _requests(12)
    o = B.qp_opts_default()
    o.precision = prec
    bounds = [B.qp_device_bytes_bound(q.n, q.m1, q.m2, o) for q in qps]
    # a budget that holds about three of these QPs at once: requests wait for memory
    budget = 3 * max(bounds)
    srv = B.Server(budget_bytes=budget, max_slots=6, opts=o)
    tickets = []
    for k, q in enumerate(qps):
        tickets.append(srv.submit(q))
        if k % 4 == 3:
            time.sleep(0.01)                 # arrivals spread out: later ones join a running mix
    assert srv.drain(timeout_ms=600_000) == B.QP_OK
    st = srv.stats()
    assert st["completed"] == len(qps) and st["queued"] == 0 and st["active"] == 0
    assert st["peak_reserved_bytes"] <= budget
    assert 0 < st["peak_device_bytes"] <= max(bounds)
    got = {}
    for t, q in zip(tickets, qps):
        r = srv.poll(t)
        assert r is not None
        res, x = r
        assert res["latency_ms"] >= res["solve_ms"] > 0 and res["wait_ms"] >= 0
        got[q.name] = (res, x)
    with pytest.raises(B.QPError):
        srv.poll(tickets[0])                 # released
    srv.close()
    for q in qps:
        res, x = got[q.name]
        st_a, f_a, its_a, x_a = _solve_alone(B, q, o)
        assert res["status"] == st_a == B.QP_OK, (q.name, res)
        assert np.array_equal(x, x_a), q.name
        assert res["obj"] == f_a and res["ipm_iters"] == its_a
        ref = ipm.solve_qp(q, variant="kkt3")
        assert abs(res["obj"] - ref.f) / max(abs(ref.f), 1.0) <= 1e-6, (q.name, res["obj"], ref.f)
        assert abs(res["ipm_iters"] - ref.iters) <= 2


def test_server_rejects_what_can_never_fit(B):
    o = B.qp_opts_default()
    q = _requests(1, seed0=5)[0]
    bound = B.qp_device_bytes_bound(q.n, q.m1, q.m2, o)
    srv = B.Server(budget_bytes=bound - 1, max_slots=2, opts=o)
    with pytest.raises(B.QPError) as e:
        srv.submit(q)
    assert e.value.status == B.QP_ENOMEM
    with pytest.raises(B.QPError) as e:
        srv.poll(12345)
    srv.close()


@pytest.mark.parametrize("prec", [1, 0])
def test_server_large_requests_match_oracle(B, prec):
    """Requests of the served workload itself with n > 1024 (requests 54, 19 and 89
    of its stream: P_H with few and with more equalities, and P_L with few degrees
    of freedom), served among small ones: each result equals the same QP solved
    alone and the FP64 oracle's optimum."""
    big = [qpgen.serving_qp(i) for i in (54, 19, 89)]
    assert all(q.n > 1024 for q in big)
    qps = big + _requests(4, seed0=900)
    o = B.qp_opts_default()
    o.precision = prec
    srv = B.Server(budget_bytes=sum(B.qp_device_bytes_bound(q.n, q.m1, q.m2, o) for q in qps),
                   max_slots=4, opts=o)
    tickets = [srv.submit(q) for q in qps]
    assert srv.drain(timeout_ms=600_000) == B.QP_OK
    got = [srv.poll(t) for t in tickets]
    srv.close()
    for q, (res, x) in zip(big, got[:len(big)]):
        assert res["status"] == B.QP_OK, (q.name, res)
        st_a, f_a, its_a, x_a = _solve_alone(B, q, o)
        assert st_a == B.QP_OK and np.array_equal(x, x_a) and res["obj"] == f_a, q.name
        ref = ipm.solve_qp(q, variant="kkt3")
        assert abs(res["obj"] - ref.f) / max(abs(ref.f), 1.0) <= 1e-6, (q.name, res["obj"], ref.f)
        assert abs(res["ipm_iters"] - ref.iters) <= 2, (q.name, res["ipm_iters"], ref.iters)
