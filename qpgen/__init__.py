"""Seeded synthetic convex-QP generator shared by the oracle, the tests and the bench.

This module only draws numbers. It holds none of the interior-point method's
arithmetic (no factorization, no KKT algebra, no Schur complement). Both the
CPU oracle and the CUDA path read the exact same arrays from it.

Problem form (Section 1, eq. (1.1) "qp"): minimise 1/2 x^T H x + c^T x subject to
A x = b and C x >= d, with H in R^{n x n} symmetric positive definite,
A in R^{m1 x n} of full row rank and C in R^{m2 x n}.

Workloads (the shapes the method is measured on):

* ``dense_qp``: H = Q diag(lam) Q^T with Q Haar-random orthogonal (QR of a
  Gaussian matrix with the sign of R's diagonal folded into Q, Mezzadri's
  method) and lam log-uniform in [lam_lo, lam_hi]; A, C, c, x0 iid N(0,1);
  b = A x0; d = C x0 - u with u ~ U(0.1, 1), so x0 is strictly feasible and the
  QP has a unique optimum.  Draw order: Q, lam, A, C, c, x0, u.
* ``orth_scaled`` A (few-degrees-of-freedom workload): the rows of A are an
  orthonormal basis (QR of a Gaussian A0^T) scaled by sigma log-uniform in
  [1e-2, 1], which makes the equality block ill-conditioned.
* ``batch_dims`` / ``serving_dims``: the size mixes of the batched and the
  served workloads.
* ``sparse_C``: 8 nonzeros per row, column indices drawn without replacement,
  values N(0,1), returned as CSR.
* ``tiny_qp``: the same recipe at n <= 6, m2 <= 10 for brute-force checks.
* ``syqp``: the paper's synthetic family SyQP^n_{m1} (Sec. 6, Test problems):
  simple bounds x >= 0 (C = I, d = 0); H block diagonal with 4 x 4 blocks M'M,
  M ~ U[0,1); A full rank and banded with band entries ~ U[0,1); c ~ U[0,1).
  The band width and the draw of b are not given there: row i of A covers the
  ``band`` columns from s_i = floor(i (n - w + 1) / m1), w = min(band, n - m1 + 1)
  (strictly increasing starts, so A has full row rank), and b = A x0 with
  x0 ~ U(0.5, 1.5) so that a strictly feasible point exists.  Draw order: the
  H blocks, the band of A, x0, c.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "QP", "dense_qp", "config_qp", "batch_dims", "serving_dims", "tiny_qp",
    "CONFIGS", "pcg_inputs", "arrival_times", "syqp",
]


@dataclasses.dataclass
class QP:
    """A convex QP  min 1/2 x'Hx + c'x  s.t.  Ax = b, Cx >= d  (FP64, row-major).

    ``C`` is dense (m2 x n) unless ``C_csr`` is given as (rowptr, colidx, val),
    in which case ``C`` is None.  ``x0`` is the strictly feasible point the
    generator built ``b`` and ``d`` from (not a solution).
    """
    H: np.ndarray
    c: np.ndarray
    A: np.ndarray
    b: np.ndarray
    C: np.ndarray | None
    d: np.ndarray
    x0: np.ndarray
    C_csr: tuple | None = None
    name: str = ""

    @property
    def n(self) -> int:
        return self.H.shape[0]

    @property
    def m1(self) -> int:
        return self.A.shape[0]

    @property
    def m2(self) -> int:
        return self.d.shape[0]

    def C_dense(self) -> np.ndarray:
        """C as a dense array (expands the CSR form if needed)."""
        if self.C is not None:
            return self.C
        rowptr, colidx, val = self.C_csr
        out = np.zeros((self.m2, self.n))
        for i in range(self.m2):
            out[i, colidx[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
        return out


def _haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    sgn = np.sign(np.diag(r))
    sgn[sgn == 0] = 1.0
    return q * sgn[None, :]


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def _sparse_rows(rng, m2, n, nnz_per_row):
    k = min(nnz_per_row, n)
    rowptr = np.arange(0, (m2 + 1) * k, k, dtype=np.int32)
    colidx = np.empty(m2 * k, dtype=np.int32)
    for i in range(m2):
        colidx[i * k:(i + 1) * k] = np.sort(rng.choice(n, size=k, replace=False))
    val = rng.standard_normal(m2 * k)
    return rowptr, colidx, val


def _csr_matvec(csr, m2, x):
    rowptr, colidx, val = csr
    out = np.zeros(m2)
    np.add.at(out, np.repeat(np.arange(m2), np.diff(rowptr)), val * x[colidx])
    return out


def dense_qp(n: int, m1: int, m2: int, seed: int, lam_lo: float = 1e-2,
             lam_hi: float = 1e2, a_kind: str = "gaussian", c_sparse_nnz: int = 0,
             name: str = "") -> QP:
    """Draw one QP with the recipe in the module docstring."""
    rng = np.random.default_rng(seed)
    Q = _haar_orthogonal(rng, n)
    lam = _log_uniform(rng, lam_lo, lam_hi, n)
    H = (Q * lam[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    if a_kind == "gaussian":
        A = rng.standard_normal((m1, n))
    elif a_kind == "orth_scaled":
        A0 = rng.standard_normal((m1, n))
        qa, _ = np.linalg.qr(A0.T)                       # n x m1, orthonormal columns
        sig = _log_uniform(rng, 1e-2, 1.0, m1)
        A = sig[:, None] * qa.T
    else:
        raise ValueError(a_kind)
    if c_sparse_nnz:
        C_csr = _sparse_rows(rng, m2, n, c_sparse_nnz)
        C = None
    else:
        C = rng.standard_normal((m2, n))
        C_csr = None
    c = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    u = rng.uniform(0.1, 1.0, m2)
    b = A @ x0
    Cx0 = C @ x0 if C is not None else _csr_matvec(C_csr, m2, x0)
    d = Cx0 - u
    return QP(H=H, c=c, A=A, b=b, C=C, d=d, x0=x0, C_csr=C_csr, name=name)


# The five workloads (dense few-equalities / few-dof singles, batched, served).
CONFIGS = {
    0: dict(n=120, m1=30, m2=200, seed=0, lam_lo=1e-2, lam_hi=1e2),
    1: dict(n=2000, m1=200, m2=4000, seed=1, lam_lo=1e-3, lam_hi=1e3),
    2: dict(n=3000, m1=2600, m2=6000, seed=2, lam_lo=1e-2, lam_hi=1e2,
            a_kind="orth_scaled"),
}


def config_qp(k: int, scale: float = 1.0) -> QP:
    """Single-QP workload k in {0, 1, 2}; ``scale`` < 1 shrinks n, m1, m2 alike
    (same recipe and seed) for quick checks of the same shape family."""
    cfg = dict(CONFIGS[k])
    if scale != 1.0:
        for key in ("n", "m1", "m2"):
            cfg[key] = max(2, int(round(cfg[key] * scale)))
    name = f"dense_n{cfg['n']}_m1_{cfg['m1']}_m2_{cfg['m2']}_seed{cfg['seed']}"
    return dense_qp(name=name, **cfg)


def batch_dims(i: int):
    """Sizes of QP i of the batched workload: n ~ U{64..512},
    m1 ~ U{ceil(0.1n)..floor(0.5n)}, m2 ~ U{n..3n}; drawn from seed i."""
    rng = np.random.default_rng(i)
    n = int(rng.integers(64, 513))
    m1 = int(rng.integers(math.ceil(0.1 * n), math.floor(0.5 * n) + 1))
    m2 = int(rng.integers(n, 3 * n + 1))
    return n, m1, m2, rng


def batch_qp(i: int) -> QP:
    """QP i of the batched workload (512 QPs of uneven size)."""
    n, m1, m2, _ = batch_dims(i)
    return dense_qp(n, m1, m2, seed=1_000_000 + i, lam_lo=1e-2, lam_hi=1e2,
                    name=f"batch{i}_n{n}_m1_{m1}_m2_{m2}")


def serving_dims(i: int):
    """Sizes of request i of the served workload: n log-uniform in [64, 4096],
    m1 = floor(n U(0.05, 0.9)), m2 = floor(n U(1, 3))."""
    rng = np.random.default_rng(10000 + i)
    n = int(round(float(_log_uniform(rng, 64, 4096, 1)[0])))
    m1 = max(1, int(math.floor(n * rng.uniform(0.05, 0.9))))
    m2 = max(1, int(math.floor(n * rng.uniform(1.0, 3.0))))
    return n, m1, m2


def serving_qp(i: int) -> QP:
    """Request i of the served workload (sparse C, 8 nonzeros per row)."""
    n, m1, m2 = serving_dims(i)
    return dense_qp(n, m1, m2, seed=2_000_000 + i, lam_lo=1e-2, lam_hi=1e2,
                    c_sparse_nnz=8, name=f"serve{i}_n{n}_m1_{m1}_m2_{m2}")


def arrival_times(count: int, rate_per_s: float, seed: int = 4) -> np.ndarray:
    """Poisson arrival stream: cumulative exponential gaps at ``rate_per_s``."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def tiny_qp(seed: int) -> QP:
    """A QP small enough for active-set enumeration: n in 2..6,
    m1 in 1..n-1, m2 in 1..10; same value recipe as ``dense_qp``."""
    rng = np.random.default_rng(500_000 + seed)
    n = int(rng.integers(2, 7))
    m1 = int(rng.integers(1, n))
    m2 = int(rng.integers(1, 11))
    return dense_qp(n, m1, m2, seed=600_000 + seed, name=f"tiny{seed}")


def pcg_inputs(m2: int, seed: int, d_lo: float = 1e-2, d_hi: float = 1e2):
    """Inputs of one reduced solve K_F dnu = rhs: a positive diagonal D
    (log-uniform in [d_lo, d_hi], the shape of V^{-1}S inside the IPM) and a
    N(0,1) right-hand side."""
    rng = np.random.default_rng(900_000 + seed)
    D = _log_uniform(rng, d_lo, d_hi, m2)
    rhs = rng.standard_normal(m2)
    return D, rhs


def syqp(n: int, m1: int, seed: int = 0, band: int = 3) -> QP:
    """SyQP^n_{m1} of the paper's synthetic family (see the module docstring)."""
    if not (1 <= m1 <= n):
        raise ValueError("SyQP needs 1 <= m1 <= n")
    rng = np.random.default_rng(3_000_000 + seed)
    H = np.zeros((n, n))
    for k in range(0, n, 4):
        b = min(4, n - k)
        M = rng.uniform(0.0, 1.0, (b, b))
        H[k:k + b, k:k + b] = M.T @ M
    w = min(band, n - m1 + 1)
    A = np.zeros((m1, n))
    for i in range(m1):
        s0 = (i * (n - w + 1)) // m1
        A[i, s0:s0 + w] = rng.uniform(0.0, 1.0, w)
    x0 = rng.uniform(0.5, 1.5, n)
    c = rng.uniform(0.0, 1.0, n)
    C = np.eye(n)
    return QP(H=H, c=c, A=A, b=A @ x0, C=C, d=np.zeros(n), x0=x0, name=f"syqp{n}_{m1}_s{seed}")
