"""qp_opts.factor_bk: the Bunch-Kaufman LDL' of K0 = [H A'; A 0] on the GPU (the
paper's setup factorization, Sec. 6: SYTRF).  Its D must have K0's inertia
(n, m1) (Sec. 4.1), and M0 = [K0^{-1}]_11 formed from it drives the persistent
kernel's K0 solve (pcg_form 0) and the low-rank form's Z (pcg_form 3): reduced
solves against the direct solve of the explicit K_F, and whole IPM solves
against the FP64 oracle.  A Hessian scaled down by 1e3 makes Bunch-Kaufman take
2x2 pivots (|h_kk| below alpha times the largest |a_ik| of its column)."""
import json
import os

import numpy as np
import pytest

import qpgen
from oracle import reduced

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _opts(B, prec, form, pc=0):
    o = B.qp_opts_default()
    o.precision, o.pcg_form, o.precond, o.factor_bk = prec, form, pc, 1
    return o


@pytest.mark.parametrize("form", [0, 3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(60, 20, 150, 1e-2, 1e2), (300, 40, 1100, 1e-2, 1e2),
                                   (120, 70, 260, 1e-4, 1e-3), (64, 0, 96, 1e-2, 1e2)])
def test_bk_inertia_and_reduced_solve(B, prec, form, shape):
    n, m1, m2, lo, hi = shape
    if form == 3 and m1 == 0:
        pytest.skip("the low-rank form needs m1 > 0 to be low rank")
    if lo < 1e-3 and prec == 1:
        pytest.skip("H scaled to 1e-4..1e-3 puts K_F beyond FP32's 2e-3 bar; its pivots are tested in FP64")
    q = qpgen.dense_qp(n, m1, m2, seed=43, lam_lo=lo, lam_hi=hi)
    h = B.QP.from_qpgen(q, _opts(B, prec, form)).factor()
    s = B.qp_get_stats(h.h)
    assert (s["k0_inertia_pos"], s["k0_inertia_neg"]) == (n, m1)
    if lo < 1e-3:
        assert s["k0_pivots_2x2"] > 0                   # the scaled Hessian takes 2x2 pivots
    D, rhs = qpgen.pcg_inputs(m2, 7, 0.1, 10.0)
    tol = 1e-12 if prec == 0 else 1e-5
    dnu = np.zeros(m2)
    st, it, rel = B.qp_pcg_reduced_solve(h.h, D, rhs, dnu, precond=1, tol=tol, maxit=20000)
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    ref = np.linalg.solve(K, rhs)
    assert rel <= tol
    err = np.linalg.norm(dnu - ref) / np.linalg.norm(ref)
    assert err <= (1e-8 if prec == 0 else 2e-3), (it, err)
    h.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_bk_ipm_config0(B, prec):
    q = qpgen.config_qp(0)
    with open(os.path.join(HERE, "golden", "oracle_config0.json")) as fh:
        gold = json.load(fh)
    h = B.QP.from_qpgen(q, _opts(B, prec, 0))
    x = np.zeros(q.n)
    st, f, its, _ = B.qp_ipm_solve(h.h, x)
    s = B.qp_get_stats(h.h)
    assert st == B.QP_OK
    assert (s["k0_inertia_pos"], s["k0_inertia_neg"]) == (q.n, q.m1)
    assert abs(f - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6
    assert abs(its - gold["ipm_iters"]) <= 2
    h.close()


def test_bk_default_off(B):
    q = qpgen.config_qp(0)
    h = B.QP.from_qpgen(q, B.qp_opts_default()).factor()
    s = B.qp_get_stats(h.h)
    assert s["k0_inertia_pos"] == -1 and s["k0_pivots_2x2"] == -1
    h.close()
