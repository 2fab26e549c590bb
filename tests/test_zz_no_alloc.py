"""The no-allocation entry point qp_kf_apply_static against qp_kf_apply.

qp_kf_apply_static serves callers that cannot allocate device memory (they run
under an allocator they do not own, or where cudaMalloc is not allowed, or on a
fixed memory budget): they pass the factored K0 and the vectors as device
arrays, and the intermediate vectors live in a fixed device array of the
library.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

import qpgen

pytestmark = pytest.mark.gpu


def _factor_arrays(q):
    """WH = R^{-T} (H = R'R) and Gt = L_S^{-1} A R^{-1} (L_S L_S' = A H^{-1} A'),
    the stored-factor layout the entry point documents."""
    L = np.linalg.cholesky(q.H)              # L = R'
    WH = np.linalg.inv(L)                    # R^{-T}, lower triangular
    WH = np.tril(WH)
    G = q.A @ WH.T                           # A R^{-1}
    LS = np.linalg.cholesky(G @ G.T)
    Gt = np.linalg.solve(LS, G)
    return WH, Gt


def test_kf_apply_static_matches_handle_path():
    torch = pytest.importorskip("torch")
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    q = qpgen.dense_qp(150, 40, 260, seed=77)
    WH, Gt = _factor_arrays(q)
    o = B.qp_opts_default()
    o.precision = B.QP_PREC_FP64
    h = B.QP.from_qpgen(q, o).factor()
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Cd, WHd, Gtd = t(q.C), t(WH), t(Gt)
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(3)
    for call in range(2):                    # two calls in a row share the scratch array
        D, _ = qpgen.pcg_inputs(q.m2, 40 + call)
        p = rng.standard_normal(q.m2)
        ref = np.zeros(q.m2)
        B.qp_kf_apply(h.h, D, p, ref)
        qd = torch.full((q.m2,), float("nan"), dtype=torch.float64, device=dev)
        B.qp_kf_apply_static(Cd, WHd, Gtd, t(D), t(p), qd, stream=stream)
        stream.synchronize()
        out = qd.cpu().numpy()
        assert np.all(np.isfinite(out))
        assert np.linalg.norm(out - ref) <= 1e-9 * np.linalg.norm(ref), call
    h.close()


def test_kf_apply_static_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    n = B.load().qp_kf_apply_static  # raw call: sizes are checked before any device work
    dev = torch.device("cuda", 0)
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    p = x.data_ptr()
    assert n(8193, 0, 4, p, p, None, p, p, p, None) == B.QP_EINVAL
    assert n(4, 5, 4, p, p, p, p, p, p, None) == B.QP_EINVAL
