"""The single-QP workloads at their full sizes, solved on the GPU in the launch
configuration bench.py times, against the FP64 oracle's golden optimum
(tests/golden, written by make_golden.py from oracle/ only): relative objective
1e-6, IPM iterations within 2, scaled residuals 1e-8, and the golden solution
samples (the first entries and the 2-norm of x) to 1e-5 relative."""
import json
import os

import numpy as np
import pytest

import qpgen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    from paper_2104_12916_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("cfg", [1, 2])
@pytest.mark.parametrize("prec", [1, 0])
def test_full_size_workload_matches_golden(B, cfg, prec):
    with open(os.path.join(HERE, "golden", f"oracle_config{cfg}.json")) as fh:
        gold = json.load(fh)
    q = qpgen.config_qp(cfg)
    assert (q.n, q.m1, q.m2) == (gold["n"], gold["m1"], gold["m2"])
    o = B.qp_opts_default()
    o.precision = prec
    h = B.QP.from_qpgen(q, o)
    x = np.zeros(q.n)
    st, f, its, _ = B.qp_ipm_solve(h.h, x)
    s = B.qp_get_stats(h.h)
    assert st == B.QP_OK
    assert abs(f - gold["f"]) / max(abs(gold["f"]), 1.0) <= 1e-6, (f, gold["f"])
    assert abs(its - gold["ipm_iters"]) <= 2, (its, gold["ipm_iters"])
    assert s["res_p"] <= 1e-8 and s["res_d"] <= 1e-8
    head = np.array(gold["x_head"])
    assert np.linalg.norm(x[:len(head)] - head) <= 1e-5 * max(1.0, np.linalg.norm(head))
    assert abs(np.linalg.norm(x) - gold["x_norm2"]) <= 1e-5 * gold["x_norm2"]
    h.close()
