"""The paper's synthetic family SyQP^n_{m1} (Sec. 6, Test problems; C = I,
d = 0) and its CG-count experiment (Sec. 6, Conjugate gradient iteration
count), reproduced with the oracle: at every IPM iteration of the oracle's
solve, PCG on K_F (eq. [ineq-const-reduced], explicit) with P_L and P_H at the
inexact IPM's tolerance eps = 1e-3.  The paper states the medians over IPM
iterations stay within m1 + 1 (P_H, Corollary 2) and, for m1 > n/2, within
2(n - m1) + 1 (P_L, the figure's looser form of Corollary 1)."""
import numpy as np
import pytest

import qpgen
from oracle import ipm, reduced as R

N = 64


def _cg_medians(m1, tol=1e-3):
    q = qpgen.syqp(N, m1)
    counts = {"PL": [], "PH": []}

    class Probe(ipm._KKT3):
        def __init__(self, H, A, C, s, nu):
            super().__init__(H, A, C, s, nu)
            D = s / nu
            K = R.kf_explicit(H, A, C, D)
            rhs = K @ np.ones(len(D))
            for name, P in (("PL", R.P_L(D)), ("PH", R.P_H(H, C, D))):
                Pi = np.linalg.inv(P)
                _, it, _ = R.pcg(lambda p: K @ p, lambda r: Pi @ r, rhs, tol, 10 * len(D))
                counts[name].append(it)

    r = ipm.solve(q.H, q.c, q.A, q.b, q.C, q.d, variant="kkt3", newton=Probe)
    assert r.status == "optimal"
    return {k: float(np.median(v)) for k, v in counts.items()}


def test_syqp_generator_shape():
    for m1 in (1, 17, 64):
        q = qpgen.syqp(N, m1)
        assert np.array_equal(q.C, np.eye(N)) and not q.d.any()
        assert np.linalg.matrix_rank(q.A) == m1
        assert np.all(q.A >= 0) and np.all(q.x0 > 0)
        assert np.allclose(q.A @ q.x0, q.b)
        # block diagonal H (4 x 4 blocks), the same for every m1
        mask = np.kron(np.eye(N // 4), np.ones((4, 4))) == 0
        assert not q.H[mask].any()
        assert np.array_equal(q.H, qpgen.syqp(N, 5).H)


@pytest.mark.parametrize("m1", [1, 4, 16, 32, 40, 48, 56, 63, 64])
def test_syqp_cg_medians_within_the_paper_bounds(m1):
    med = _cg_medians(m1)
    assert med["PH"] <= m1 + 1, med
    if m1 > N // 2:
        assert med["PL"] <= 2 * (N - m1) + 1, med
