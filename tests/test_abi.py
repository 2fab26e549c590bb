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
