"""Failure detection on the GPU without a GPU fault: every wait in the
persistent PCG kernel is bounded (2 s on %globaltimer).  With
PCGIPM_TEST_LEAVE_EARLY=1, block 0 of the kernel stops before its first grid
barrier, as a block that died would; the other blocks' waits run out, the
kernel returns, and the host reports QP_ETIMEOUT.  Nothing traps or faults, so
the context stays usable: a new handle then solves normally."""
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


def test_bounded_wait_reports_timeout_and_context_survives(B, monkeypatch):
    q = qpgen.config_qp(0)                 # grid of 8 blocks: there are other blocks to wait
    D, rhs = qpgen.pcg_inputs(q.m2, 11)
    o = B.qp_opts_default()
    o.precision = B.QP_PREC_FP64
    monkeypatch.setenv("PCGIPM_TEST_LEAVE_EARLY", "1")
    h = B.QP.from_qpgen(q, o).factor()     # the engine reads the variable when it is created
    dnu = np.zeros(q.m2)
    with pytest.raises(B.QPError) as e:
        B.qp_pcg_reduced_solve(h.h, D, rhs, dnu, precond=B.QP_PC_PH_EXACT, tol=1e-10, maxit=200)
    assert e.value.status == B.QP_ETIMEOUT
    h.close()
    monkeypatch.delenv("PCGIPM_TEST_LEAVE_EARLY")
    h2 = B.QP.from_qpgen(q, o).factor()
    st, it, rel = B.qp_pcg_reduced_solve(h2.h, D, rhs, dnu, precond=B.QP_PC_PH_EXACT, tol=1e-10, maxit=200)
    assert st == B.QP_OK and rel <= 1e-10 and np.all(np.isfinite(dnu))
    h2.close()
