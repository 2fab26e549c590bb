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


def test_paper_mode_objective_loss_and_iterations(B):
    """Sec. 6 setting on the paper's own SyQP family: one PCG solve per Newton
    direction at eps = 1e-3 with no refinement (QP_MODE_PAPER, P_H, FP64), against
    the same IPM with every direction refined to its FP64 residual (PARITY).
    The paper reports an objective loss below 6e-7 for the inexact IPM against a
    direct solve and a median of 22% more IPM iterations.  Both runs stop at the
    same tolerances (1e-8 feasibility, mu <= 1e-9 (1 + |f|)); the median loss over
    the family must stay below the paper's 6e-7, and the median iteration increase
    is reported (printed) beside its 22%."""
    losses, ratios = [], []
    for n, m1, seed in [(64, 4, 1), (64, 16, 2), (64, 32, 3), (128, 24, 4), (128, 64, 5), (256, 40, 6)]:
        q = qpgen.syqp(n, m1, seed=seed)
        ref = ipm.solve_qp(q, variant="kkt3")
        out = {}
        for mode in (B.QP_MODE_PARITY, B.QP_MODE_PAPER):
            o = B.qp_opts_default()
            o.precision, o.precond, o.pcg_mode = B.QP_PREC_FP64, B.QP_PC_PH_EXACT, mode
            o.tol_feas, o.tol_mu, o.max_ipm = 1e-8, 1e-9, 100
            h = B.QP.from_qpgen(q, o)
            st, f, its, _ = B.qp_ipm_solve(h.h, allow=(B.QP_OK, B.QP_EMAXIT))
            out[mode] = (st, f, its, B.qp_get_stats(h.h)["refine_sweeps"])
            h.close()
        assert out[B.QP_MODE_PAPER][3] == 0
        losses.append(abs(out[B.QP_MODE_PAPER][1] - ref.f) / max(abs(ref.f), 1.0))
        ratios.append(out[B.QP_MODE_PAPER][2] / max(1, out[B.QP_MODE_PARITY][2]))
    med_loss, med_ratio = float(np.median(losses)), float(np.median(ratios))
    print(f"PAPER mode on SyQP: median objective loss {med_loss:.2e} (paper: < 6e-7), "
          f"median IPM iterations x{med_ratio:.2f} (paper: x1.22); per QP {losses} {ratios}")
    assert med_loss <= 6e-7
