"""The grid autotuner of the persistent PCG kernel (qp_opts.autotune).  Every
reduction of the kernel has an order that does not depend on the grid, so a
tuned solve must give bit-identical results to the same solve on the rule's
grid; the tuned grid is reported in qp_stats.pcg_grid.  The QP streams about
45 MB per PCG iteration (M0 form), so its grid spans the GPU and is tuned."""
import numpy as np
import pytest

import qpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_solve_is_bit_identical(B, prec):
    q = qpgen.dense_qp(1500, 100, 3000, seed=77)
    out = {}
    for tune in (0, 1):
        o = B.qp_opts_default()
        o.precision, o.autotune, o.pcg_form = prec, tune, 0
        h = B.QP.from_qpgen(q, o)
        x = np.zeros(q.n)
        st, f, its, pits = B.qp_ipm_solve(h.h, x)
        assert st == B.QP_OK
        nu = np.zeros(q.m2)
        B.qp_get_solution(h.h, x=x, nu=nu)
        out[tune] = (x.copy(), nu, f, its, pits, B.qp_get_stats(h.h))
        h.close()
    (x0, nu0, f0, i0, p0, s0), (x1, nu1, f1, i1, p1, s1) = out[0], out[1]
    assert s0["pcg_grid"] > 16 and s1["pcg_grid"] > 16
    assert i0 == i1 and p0 == p1
    assert f0 == f1
    assert np.array_equal(x0, x1) and np.array_equal(nu0, nu1)
