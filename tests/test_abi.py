"""Host-only checks of the C-ABI library: it loads and exports every function
that include/pcgipm.h declares (no compute call, no GPU needed)."""
import os
import re

import pytest

from paper_2104_12916_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|size_t|double|unsigned long long|const char\s*\*)\s*\**\s*(qp_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(binding.EXPORTED) <= names


def test_host_only_calls(lib):
    o = binding.qp_opts_default()
    assert o.precision == binding.QP_PREC_FP32 and o.max_ipm == 100 and o.refine_max == 5
    assert binding.qp_strerror(binding.QP_ENOTCONVEX).startswith("H has")
    assert binding.qp_strerror(12345) == "unknown status"


def test_new_option_defaults(lib):
    o = binding.qp_opts_default()
    assert o.pcg_blocks == 0 and o.blocking_wait == 0 and o.mixed_fallback == 1
    assert o.pcg_form == binding.QP_FORM_AUTO and o.factor_tc == 0 and o.autotune == 1 and o.factor_bk == 0
    assert o.precond == binding.QP_PC_AUTO and o.pcg_mode == binding.QP_MODE_PARITY


def _bound(n, m1, m2, **kw):
    o = binding.qp_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return binding.qp_device_bytes_bound(n, m1, m2, o)


def test_device_bytes_bound_host_logic(lib):
    """The admission bound (host arithmetic only) covers what a handle must hold:
    the FP64 problem copies (H, A, A', C, C'), the operator factor, and the four
    m2 x m2 P_H matrices whenever P_H may be used; it grows with every size."""
    n, m1, m2 = 500, 100, 1200
    fp64_copies = 8 * (n * n + 2 * m1 * n + 2 * m2 * n)
    ph32 = 4 * 4 * m2 * m2
    auto = _bound(n, m1, m2)
    assert auto >= fp64_copies + ph32 + 8 * 2 * n * n      # + the FP64 factor (mixed may move there)
    pl = _bound(n, m1, m2, precond=binding.QP_PC_PL)
    assert pl < auto and pl >= fp64_copies                  # an explicit P_L never builds P_H
    assert _bound(n, m1, m2, mixed_fallback=0) < auto       # no FP64 operator or P_H to move to
    assert _bound(n, m1, m2, pcg_form=1) >= auto + 4 * 2 * (n + m1) * m2   # B and B' (FP32)
    assert _bound(n, m1, m2, pcg_form=0, factor_bk=1) >= _bound(n, m1, m2, pcg_form=0) + 8 * (n + m1) ** 2
    f64 = _bound(n, m1, m2, precision=binding.QP_PREC_FP64)
    assert f64 >= fp64_copies + 8 * 4 * m2 * m2
    for dn, dm1, dm2 in ((50, 0, 0), (0, 20, 0), (0, 0, 100)):
        assert _bound(n + dn, m1 + dm1, m2 + dm2) > auto
    assert binding.qp_device_bytes_bound(0, 0, 5, None) == 0          # invalid sizes
    assert binding.qp_device_bytes_bound(5, 6, 5, None) == 0


def test_device_calls_fail_cleanly_without_a_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: these calls would succeed")
    import numpy as np
    n, m1, m2 = 4, 1, 6
    H = np.eye(n)
    with pytest.raises(binding.QPError) as e:
        binding.qp_create(H, np.zeros(n), np.ones((m1, n)), np.zeros(m1), np.ones((m2, n)), np.zeros(m2))
    assert e.value.status == binding.QP_ECUDA
    with pytest.raises(binding.QPError) as e:
        binding.Server(budget_bytes=1 << 30, max_slots=2)
    assert e.value.status == binding.QP_ECUDA


def test_auto_form_resolution(lib):
    """QP_FORM_AUTO (host logic): the low-rank form when V = C Z streams at most
    half of what C', M0 and C stream (2 m2 r <= (2 m2 n + n^2) / 2, r = n - m1 in
    [1, 1024]), the M0 form otherwise -- seen through the admission bound, which
    sizes the form the handle will hold."""
    for n, m1, m2, want in ((3000, 2600, 6000, 3), (2000, 200, 4000, 0), (400, 200, 900, 3),
                            (400, 400, 900, 0), (3000, 1500, 4000, 0), (100, 40, 300, 0),
                            (100, 50, 300, 3), (1000, 300, 2000, 0)):
        auto = _bound(n, m1, m2, pcg_form=binding.QP_FORM_AUTO)
        assert auto == _bound(n, m1, m2, pcg_form=want), (n, m1, m2)
    assert _bound(100, 60, 300, pcg_form=3) != _bound(100, 60, 300, pcg_form=0)
    assert binding.qp_device_bytes_bound(10, 5, 20, None) > 0
