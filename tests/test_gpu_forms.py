"""The other forms of the same K_F product in the persistent kernel:
  pcg_form 1: through B = L^{-1}[C'; 0] formed once per QP (two matrix phases);
  pcg_form 2: the forward and the back solve with the stored inverse factor as
              two phases (four matrix phases);
  pcg_form 3: the low-rank form K_F = D + V V', V = C Z with M0 = Z Z' of rank
              n - m1 (Sec. 4.3, Lemma 2), Z from a pivoted Cholesky of M0.
The same operator, so the same bars as the default form: reduced solves against
the direct solve of the explicit K_F (FP64 1e-8, FP32 2e-3; in FP32 mode the
matrices are formed from the FP64 factor and rounded once), and whole IPM solves
against the FP64 oracle (objective 1e-6, iterations within 2, residuals 1e-8)."""
import json
import os

import numpy as np
import pytest

import qpgen
from oracle import ipm, reduced

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _opts(B, prec, pc=0, form=1):
    o = B.qp_opts_default()
    o.precision, o.precond, o.pcg_form = prec, pc, form
    return o


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("pc", [1, 2])
@pytest.mark.parametrize("shape", [(60, 20, 150), (130, 70, 150), (64, 0, 96), (300, 40, 1100)])
def test_form_reduced_solve(B, prec, pc, shape, form):
    n, m1, m2 = shape
    q = qpgen.dense_qp(n, m1, m2, seed=41)
    D, rhs = qpgen.pcg_inputs(m2, 6, 0.1, 10.0)
    h = B.QP.from_qpgen(q, _opts(B, prec, form=form)).factor()
    tol = 1e-12 if prec == 0 else 1e-5
    dnu = np.zeros(m2)
    st, it, rel = B.qp_pcg_reduced_solve(h.h, D, rhs, dnu, precond=pc, tol=tol, maxit=20000)
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    ref = np.linalg.solve(K, rhs)
    assert rel <= tol
    err = np.linalg.norm(dnu - ref) / np.linalg.norm(ref)
    assert err <= (1e-8 if prec == 0 else 2e-3), (it, err)
    h.close()


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_form_ipm_config0(B, prec, form):
    q = qpgen.config_qp(0)
    with open(os.path.join(HERE, "golden", "oracle_config0.json")) as fh:
        gold = json.load(fh)
    h = B.QP.from_qpgen(q, _opts(B, prec, form=form))
    x = np.zeros(q.n)
    st, f, its, _ = B.qp_ipm_solve(h.h, x)
    s = B.qp_get_stats(h.h)
    assert st == B.QP_OK
    assert abs(f - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6
    assert abs(its - gold["ipm_iters"]) <= 2
    assert s["res_p"] <= 1e-8 and s["res_d"] <= 1e-8
    h.close()


@pytest.mark.parametrize("form", [1, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_form_ipm_syqp_and_batch_member(B, prec, form):
    for q in (qpgen.syqp(128, 96, seed=2), qpgen.batch_qp(7)):
        ref = ipm.solve_qp(q, variant="kkt3")
        h = B.QP.from_qpgen(q, _opts(B, prec, form=form))
        st, f, its, _ = B.qp_ipm_solve(h.h)
        assert st == B.QP_OK, q.name
        assert abs(f - ref.f) / max(abs(ref.f), 1.0) <= 1e-6, q.name
        assert abs(its - ref.iters) <= 2, q.name
        h.close()


@pytest.mark.parametrize("form", [0, 2])
def test_factor_tc_reduced_solve_and_ipm(B, form):
    """qp_opts.factor_tc: the FP32 K0 factor (and M0) formed on the tcgen05 tensor
    cores with FP64 pivots on the diagonal blocks.  The reduced solve meets the
    FP32 bar against the explicit K_F, and a whole IPM solve meets the oracle's
    (objective 1e-6, iterations within 2, residuals 1e-8) through the FP64
    refinement; the handle reports that the tensor-core factor was used."""
    q = qpgen.dense_qp(300, 40, 1100, seed=41)
    D, rhs = qpgen.pcg_inputs(q.m2, 6, 0.1, 10.0)
    o = _opts(B, 1, 2, form=form)
    o.factor_tc = 1
    h = B.QP.from_qpgen(q, o).factor()
    assert B.qp_get_stats(h.h)["factor_tc"] == 1
    dnu = np.zeros(q.m2)
    st, it, rel = B.qp_pcg_reduced_solve(h.h, D, rhs, dnu, precond=2, tol=1e-5, maxit=20000)
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    ref = np.linalg.solve(K, rhs)
    assert np.linalg.norm(dnu - ref) / np.linalg.norm(ref) <= 2e-3
    h.close()
    q = qpgen.config_qp(0)
    with open(os.path.join(HERE, "golden", "oracle_config0.json")) as fh:
        gold = json.load(fh)
    o = _opts(B, 1, 0, form=form)
    o.factor_tc = 1
    h = B.QP.from_qpgen(q, o)
    st, f, its, _ = B.qp_ipm_solve(h.h)
    s = B.qp_get_stats(h.h)
    assert st == B.QP_OK and s["factor_tc"] == 1
    assert abs(f - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6
    assert abs(its - gold["ipm_iters"]) <= 2
    assert s["res_p"] <= 1e-8 and s["res_d"] <= 1e-8
    h.close()
