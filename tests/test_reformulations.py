"""The two exact reformulations the persistent PCG kernel uses, checked in FP64
against the definition of K_F (eq. [ineq-const-reduced], oracle.reduced):

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
