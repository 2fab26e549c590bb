"""The no-allocation entry point qp_kf_apply_static, against qp_kf_apply and the oracle.

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
from oracle import reduced

pytestmark = pytest.mark.gpu


def _factor_arrays(q):
    """WH = R^{-T} (H = R'R) and Gt = L_S^{-1} A R^{-1} (L_S L_S' = A H^{-1} A'),
    the stored-factor layout the entry point documents (Gt is None when m1 = 0)."""
    L = np.linalg.cholesky(q.H)              # L = R'
    WH = np.tril(np.linalg.inv(L))           # R^{-T}, lower triangular
    if q.m1 == 0:
        return WH, None
    G = q.A @ WH.T                           # A R^{-1}
    LS = np.linalg.cholesky(G @ G.T)
    Gt = np.linalg.solve(LS, G)
    return WH, Gt


def _static_vs_references(q, seeds, tol=1e-9):
    """Two (or more) calls in a row through the entry point: each result is
    compared with qp_kf_apply on a handle of the same QP and with the oracle's
    K_F p (Sec. 5.2: C'p, a solve with F, a product with C, plus D p)."""
    torch = pytest.importorskip("torch")
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    WH, Gt = _factor_arrays(q)
    o = B.qp_opts_default()
    o.precision = B.QP_PREC_FP64
    h = B.QP.from_qpgen(q, o).factor()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(3)
    try:
        for call, seed in enumerate(seeds):  # calls in a row share the scratch array
            D, _ = qpgen.pcg_inputs(q.m2, seed)
            p = rng.standard_normal(q.m2)
            ref = np.zeros(q.m2)
            B.qp_kf_apply(h.h, D, p, ref)
            want = reduced.kf_apply(q.H, q.A, q.C, D, p)
            # inputs made on torch's current stream; the call runs on `stream`
            with torch.cuda.stream(stream):
                t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                Cd, WHd = t(q.C), t(WH)
                Gtd = None if Gt is None else t(Gt)
                Dd, pd = t(D), t(p)
                qd = torch.full((q.m2,), float("nan"), dtype=torch.float64, device=dev)
            stream.wait_stream(torch.cuda.current_stream())
            B.qp_kf_apply_static(Cd, WHd, Gtd, Dd, pd, qd, stream=stream)
            stream.synchronize()
            out = qd.cpu().numpy()
            assert np.all(np.isfinite(out)), call
            assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref), call
            assert np.linalg.norm(out - want) <= tol * np.linalg.norm(want), call
    finally:
        h.close()


def test_kf_apply_static_matches_handle_path_and_oracle():
    _static_vs_references(qpgen.dense_qp(150, 40, 260, seed=77), seeds=(40, 41))


def test_kf_apply_static_without_equalities():
    """m1 = 0: Gt is NULL and the K0 solve is R^{-1} R^{-T} alone (K0 = H)."""
    _static_vs_references(qpgen.dense_qp(120, 0, 200, seed=78), seeds=(42, 43))


def test_kf_apply_static_square_A_gives_D():
    """m1 = n: A is invertible, Hbar_A = H (Lemma 1), so K_F = D exactly
    (Sec. 4.1, eq. [schur-R]); the result is D p up to rounding."""
    torch = pytest.importorskip("torch")
    from paper_2104_12916_gb300 import binding as B, build
    build.build()
    q = qpgen.dense_qp(64, 64, 100, seed=79, lam_lo=0.5, lam_hi=2.0)
    WH, Gt = _factor_arrays(q)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    D, _ = qpgen.pcg_inputs(q.m2, 44)
    p = np.random.default_rng(5).standard_normal(q.m2)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    qd = torch.full((q.m2,), float("nan"), dtype=torch.float64, device=dev)
    B.qp_kf_apply_static(t(q.C), t(WH), t(Gt), t(D), t(p), qd)
    torch.cuda.synchronize()
    out = qd.cpu().numpy()
    scale = np.linalg.norm(q.C, 2) ** 2 * np.linalg.norm(np.linalg.inv(q.H), 2) * np.linalg.norm(p)
    assert np.linalg.norm(out - D * p) <= 1e-10 * scale


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


def test_kf_apply_static_wrapper_checks_shapes():
    """The binding checks every shape before the raw call (the C side sees only
    pointers and could not)."""
    torch = pytest.importorskip("torch")
    from paper_2104_12916_gb300 import binding as B
    dev = torch.device("cuda", 0)
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        B.qp_kf_apply_static(z(10, 6), z(6, 5), None, z(10), z(10), z(10))
    with pytest.raises(ValueError):
        B.qp_kf_apply_static(z(10, 6), z(6, 6), z(3, 5), z(10), z(10), z(10))
    with pytest.raises(ValueError):
        B.qp_kf_apply_static(z(10, 6), z(6, 6), None, z(10), z(9), z(10))
