"""The paper's synthetic family SyQP^n_{m1} (simple bounds, C = I) solved by the
GPU path against the FP64 oracle: relative objective 1e-6, scaled residuals
1e-8, IPM iterations within 2, in both precisions and on both sides of the
AUTO preconditioner rule (2 m1 >= n picks P_L)."""
import numpy as np
import pytest

import qpgen
from oracle import ipm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("n,m1", [(64, 16), (64, 48), (256, 40), (256, 200)])
@pytest.mark.parametrize("prec", [0, 1])
def test_syqp_matches_oracle(B, n, m1, prec):
    q = qpgen.syqp(n, m1, seed=1)
    ref = ipm.solve_qp(q, variant="kkt3")
    assert ref.status == "optimal"
    o = B.qp_opts_default()
    o.precision = prec
    h = B.QP.from_qpgen(q, o)
    x = np.zeros(n)
    st, f, its, _ = B.qp_ipm_solve(h.h, x)
    s = B.qp_get_stats(h.h)
    assert st == B.QP_OK
    assert abs(f - ref.f) / max(abs(ref.f), 1.0) <= 1e-6, (f, ref.f)
    assert s["res_p"] <= 1e-8 and s["res_d"] <= 1e-8
    assert abs(its - ref.iters) <= 2, (its, ref.iters)
    assert np.all(x >= -1e-8)
    h.close()
