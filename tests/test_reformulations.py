"""The exact reformulations the persistent PCG kernel uses, checked in FP64
against the definition of K_F (eq. [ineq-const-reduced], oracle.reduced):

* the K0 solve as one product with M0 = [K0^{-1}]_11 = R^{-1}R^{-T} - Et'Et;
* the low-rank form: M0 has rank n - m1 (Sec. 4.3, Lemma 2: H - Hbar_A has rank
  n - m1, and M0 = H^{-1}(H - Hbar_A)H^{-1}), so M0 = Z Z' with Z n x (n - m1)
  and K_F = D + (C Z)(C Z)';

* the K0 solve as two products with the inverse factor: with H = R'R,
  Gt = L_S^{-1} A R^{-1} (L_S L_S' = A H^{-1} A') and Et = Gt R^{-T}, the top
  block of K0^{-1}[u; 0] is R^{-1} z1 + Et' z2 with z1 = R^{-T} u, z2 = -Et u;
* the W-form: with B1 = R^{-T} C' and B2 = Et C',
  K_F = D + B1'B1 - B2'B2 (the closed form of eq. [schur-R])."""
import numpy as np
import pytest

import qpgen
from oracle import reduced


def _factors(q):
    R = np.linalg.cholesky(q.H).T                 # H = R'R, R upper
    Rinv = np.linalg.inv(R)
    G = q.A @ Rinv
    LS = np.linalg.cholesky(G @ G.T)
    Gt = np.linalg.solve(LS, G)
    Et = Gt @ Rinv.T
    return Rinv, Et


@pytest.mark.parametrize("shape", [(40, 10, 70), (33, 0, 50), (25, 20, 60)])
def test_two_phase_k0_solve(shape):
    n, m1, m2 = shape
    q = qpgen.dense_qp(n, m1, m2, seed=5)
    Rinv, Et = _factors(q) if m1 else (np.linalg.inv(np.linalg.cholesky(q.H).T), np.zeros((0, n)))
    u = np.random.default_rng(1).standard_normal(n)
    K0 = np.block([[q.H, q.A.T], [q.A, np.zeros((m1, m1))]]) if m1 else q.H
    top = np.linalg.solve(K0, np.concatenate([u, np.zeros(m1)]))[:n]
    z1 = Rinv.T @ u
    z2 = -Et @ u
    y = Rinv @ z1 + Et.T @ z2
    assert np.linalg.norm(y - top) <= 1e-10 * np.linalg.norm(top)


@pytest.mark.parametrize("shape", [(40, 10, 70), (25, 20, 60)])
def test_wform_equals_definition(shape):
    n, m1, m2 = shape
    q = qpgen.dense_qp(n, m1, m2, seed=6)
    D, _ = qpgen.pcg_inputs(m2, 3)
    Rinv, Et = _factors(q)
    B1 = Rinv.T @ q.C.T
    B2 = Et @ q.C.T
    Kw = np.diag(D) + B1.T @ B1 - B2.T @ B2
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    assert np.linalg.norm(Kw - K) <= 1e-10 * np.linalg.norm(K)


@pytest.mark.parametrize("shape", [(40, 10, 70), (33, 0, 50), (25, 20, 60)])
def test_k0_inverse_block_equals_definition(shape):
    n, m1, m2 = shape
    q = qpgen.dense_qp(n, m1, m2, seed=7)
    Rinv = np.linalg.inv(np.linalg.cholesky(q.H).T)
    Et = _factors(q)[1] if m1 else np.zeros((0, n))
    M0 = Rinv @ Rinv.T - Et.T @ Et
    K0 = np.block([[q.H, q.A.T], [q.A, np.zeros((m1, m1))]]) if m1 else q.H
    want = np.linalg.inv(K0)[:n, :n]
    assert np.linalg.norm(M0 - want) <= 1e-10 * np.linalg.norm(want)
    D, _ = qpgen.pcg_inputs(m2, 4)
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    assert np.linalg.norm(np.diag(D) + q.C @ M0 @ q.C.T - K) <= 1e-10 * np.linalg.norm(K)


def _pivoted_cholesky(M, r):
    """M = Z Z' by r steps of the outer-product Cholesky on the largest
    remaining diagonal entry (a textbook method, written out independently of
    the CUDA kernel)."""
    n = M.shape[0]
    Z = np.zeros((n, r))
    d = np.diag(M).copy()
    for k in range(r):
        p = int(np.argmax(d))
        col = M[:, p] - Z[:, :k] @ Z[p, :k]
        Z[:, k] = col / np.sqrt(d[p])
        d -= Z[:, k] ** 2
        d[p] = -np.inf
    return Z


@pytest.mark.parametrize("shape", [(40, 10, 70), (30, 24, 90), (20, 0, 40)])
def test_low_rank_form_equals_definition(shape):
    n, m1, m2 = shape
    q = qpgen.dense_qp(n, m1, m2, seed=8)
    M0 = np.linalg.inv(np.block([[q.H, q.A.T], [q.A, np.zeros((m1, m1))]]))[:n, :n] if m1 else np.linalg.inv(q.H)
    sv = np.linalg.svd(M0, compute_uv=False)
    assert np.sum(sv > 1e-10 * sv[0]) == n - m1              # Lemma 2: rank n - m1
    Z = _pivoted_cholesky(M0, n - m1)
    D, _ = qpgen.pcg_inputs(m2, 5)
    V = q.C @ Z
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    assert np.linalg.norm(np.diag(D) + V @ V.T - K) <= 1e-9 * np.linalg.norm(K)
