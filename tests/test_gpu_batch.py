"""qp_batch_solve: many QPs of uneven size solved concurrently.

Checks each result against the FP64 oracle (relative objective 1e-6, IPM
iterations within 2) and that a QP's solution does not depend on what it is
batched with: every reduction runs in a fixed order within its own QP and the
persistent kernel's grid depends only on the QP's size, so the solution alone
and in the batch must be bit-identical.
"""
import numpy as np
import pytest

import qpgen
from oracle import ipm

pytestmark = pytest.mark.gpu


def _mini_batch(count, seed0=300):
    """QPs of the batched workload's recipe (m1 in [0.1n, 0.5n], m2 in [n, 3n])
    at n in [32, 110] so the CPU oracle stays quick."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(32, 111))
        m1 = int(rng.integers(int(np.ceil(0.1 * n)), n // 2 + 1))
        m2 = int(rng.integers(n, 3 * n + 1))
        out.append(qpgen.dense_qp(n, m1, m2, seed=seed0 + 1000 + i))
    return out


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle_and_alone(B, prec):
    qps = _mini_batch(10)
    o = B.qp_opts_default()
    o.precision = prec
    handles = [B.QP.from_qpgen(q, o) for q in qps]
    st, res = B.qp_batch_solve([h.h for h in handles], max_concurrent=6)
    assert st == B.QP_OK, res
    xs_batch = []
    for q, h, r in zip(qps, handles, res):
        x = np.zeros(q.n)
        B.qp_get_solution(h.h, x)
        xs_batch.append(x)
        ref = ipm.solve_qp(q, variant="kkt3")
        assert abs(r["obj"] - ref.f) / max(abs(ref.f), 1.0) <= 1e-6, (q.name, r, ref.f)
        assert abs(r["ipm_iters"] - ref.iters) <= 2
    # the same QPs one at a time give bit-identical solutions
    for q, xb in zip(qps[:4], xs_batch[:4]):
        h = B.QP.from_qpgen(q, o)
        x = np.zeros(q.n)
        B.qp_ipm_solve(h.h, x)
        assert np.array_equal(x, xb), q.name


@pytest.mark.parametrize("prec", [0, 1])
def test_auto_moves_from_pl_to_ph_when_pl_stops_converging(B, prec):
    """A QP of the batched recipe at the tie 2 m1 = n (AUTO picks P_L) whose late
    IPM iterations take D over 18 decades: the P_L-preconditioned spectrum
    1 + lambda(X) grows without bound (Sec. 4.3, Theorem 1) and PCG stops
    converging, so AUTO moves the QP to P_H."""
    q = qpgen.batch_qp(201)
    assert 2 * q.m1 == q.n
    ref = ipm.solve_qp(q, variant="kkt3")
    o = B.qp_opts_default()
    o.precision = prec
    h = B.QP.from_qpgen(q, o)
    st, f, its, _ = B.qp_ipm_solve(h.h)
    assert st == B.QP_OK
    stats = B.qp_get_stats(h.h)
    assert stats["pc_switch_iter"] >= 0 and stats["precond_used"] == B.QP_PC_PH_EXACT, stats
    assert abs(f - ref.f) / max(abs(ref.f), 1.0) <= 1e-9
    assert abs(its - ref.iters) <= 2
    h.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_one_block_grid_gives_identical_results(B, prec):
    """pcg_blocks = 1 runs the persistent PCG kernel on a single block (block
    barriers only): every reduction keeps its order, so the solution is
    bit-identical to the default grid's; and a batch of such QPs with many in
    flight (blocking host waits) matches too."""
    qps = _mini_batch(6, seed0=900)
    for q in qps[:2]:
        xs = []
        for blocks in (0, 1):
            o = B.qp_opts_default()
            o.precision, o.pcg_blocks = prec, blocks
            h = B.QP.from_qpgen(q, o)
            x = np.zeros(q.n)
            B.qp_ipm_solve(h.h, x)
            xs.append(x)
            h.close()
        assert np.array_equal(xs[0], xs[1]), q.name
    o = B.qp_opts_default()
    o.precision, o.pcg_blocks, o.blocking_wait = prec, 1, 1
    handles = [B.QP.from_qpgen(q, o) for q in qps]
    st, res = B.qp_batch_solve([h.h for h in handles], max_concurrent=len(qps))
    assert st == B.QP_OK, res
    for q, h in zip(qps, handles):
        x = np.zeros(q.n)
        B.qp_get_solution(h.h, x)
        o2 = B.qp_opts_default()
        o2.precision = prec
        h2 = B.QP.from_qpgen(q, o2)
        x2 = np.zeros(q.n)
        B.qp_ipm_solve(h2.h, x2)
        assert np.array_equal(x, x2), q.name
