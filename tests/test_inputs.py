"""The seeded input recipes (qpgen) hold what the workloads promise: the
spectrum of H, a strictly feasible x0, the orthogonalised-and-scaled A of the
few-degrees-of-freedom workload, 8-nonzero rows of the served workload's C,
the size mixes of the batched and served workloads, Poisson arrivals, and
bit-for-bit determinism."""
import numpy as np
import pytest

import qpgen


@pytest.mark.parametrize("k,scale", [(0, 1.0), (1, 0.1), (2, 0.1)])
def test_single_qp_recipe(k, scale):
    q = qpgen.config_qp(k, scale)
    cfg = qpgen.CONFIGS[k]
    if scale == 1.0:
        assert (q.n, q.m1, q.m2) == (cfg["n"], cfg["m1"], cfg["m2"])
    assert np.array_equal(q.H, q.H.T)
    lam = np.linalg.eigvalsh(q.H)
    assert lam.min() >= cfg["lam_lo"] * (1 - 1e-9) and lam.max() <= cfg["lam_hi"] * (1 + 1e-9)
    # x0 strictly feasible: A x0 = b, C x0 - d = u in [0.1, 1]
    assert np.allclose(q.A @ q.x0, q.b, rtol=0, atol=1e-9 * (1 + np.abs(q.b).max()))
    u = q.C @ q.x0 - q.d
    assert u.min() >= 0.1 - 1e-9 and u.max() <= 1.0 + 1e-9
    if cfg.get("a_kind") == "orth_scaled":
        sv = np.linalg.svd(q.A, compute_uv=False)
        assert sv.min() >= 1e-2 * (1 - 1e-9) and sv.max() <= 1.0 + 1e-9


def test_determinism():
    a, b = qpgen.config_qp(0), qpgen.config_qp(0)
    for f in ("H", "c", "A", "b", "C", "d", "x0"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(qpgen.batch_qp(3).H[:4, :4], qpgen.batch_qp(4).H[:4, :4])


def test_batch_size_mix():
    for i in range(512):
        n, m1, m2 = qpgen.batch_dims(i)[:3]
        assert 64 <= n <= 512
        assert np.ceil(0.1 * n) <= m1 <= n // 2
        assert n <= m2 <= 3 * n


def test_serving_size_mix_and_sparse_C():
    ns = []
    for i in range(400):
        n, m1, m2 = qpgen.serving_dims(i)
        ns.append(n)
        assert 64 <= n <= 4096 and 1 <= m1 <= 0.9 * n + 1 and n <= m2 <= 3 * n
    # log-uniform: about half below the geometric midpoint sqrt(64 * 4096) = 512
    assert 0.4 < np.mean(np.array(ns) < 512) < 0.6
    small = [i for i in range(200) if qpgen.serving_dims(i)[0] <= 150][:3]
    for i in small:
        q = qpgen.serving_qp(i)
        rp, ci, val = q.C_csr
        assert rp[0] == 0 and len(rp) == q.m2 + 1
        for r in range(q.m2):
            cols = ci[rp[r]:rp[r + 1]]
            assert len(cols) == 8 and len(set(cols.tolist())) == 8 and cols.min() >= 0 and cols.max() < q.n
        u = q.C_dense() @ q.x0 - q.d
        assert u.min() >= 0.1 - 1e-9


def test_poisson_arrivals():
    t = qpgen.arrival_times(20000, rate_per_s=200.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0          # mean gap 1/rate (about 4 sigma)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05           # exponential: std = mean
