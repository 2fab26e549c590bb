"""The method's reduced-system quantities, written out by their definitions (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every function states the passage it follows.  Nothing here is blocked, fused
or reordered beyond the definition: inverses are dense ``numpy.linalg.solve``
calls on the matrices the paper names.
"""
from __future__ import annotations

import numpy as np


def F_matrix(H, A):
    """F = [-H A'; A 0], Sec. 4.1, eq. [f-def]."""
    n, m1 = H.shape[0], A.shape[0]
    F = np.zeros((n + m1, n + m1))
    F[:n, :n] = -H
    F[:n, n:] = A.T
    F[n:, :n] = A
    return F


def kf_explicit(H, A, C, D):
    """K_F = D - [C 0] F^{-1} [C'; 0], Sec. 4.1, eq. [ineq-const-reduced]."""
    n, m1 = H.shape[0], A.shape[0]
    F = F_matrix(H, A)
    rhs = np.zeros((n + m1, C.shape[0]))
    rhs[:n, :] = C.T
    X = np.linalg.solve(F, rhs)
    return np.diag(D) - C @ X[:n, :]


def kf_closed_form(H, A, C, D):
    """K_F = D + C H^{-1} (H - Hbar_A) H^{-1} C' with Hbar_A = A' F_H^{-1} A and
    F_H = A H^{-1} A', Sec. 4.1, eqs. [f-inv] and [schur-R] (explicit inverses)."""
    Hinv = np.linalg.inv(H)
    if A.shape[0]:
        F_H = A @ Hinv @ A.T
        Hbar = A.T @ np.linalg.inv(F_H) @ A
    else:
        Hbar = np.zeros_like(H)
    return np.diag(D) + C @ Hinv @ (H - Hbar) @ Hinv @ C.T


def hbar_A(H, A):
    """Hbar_A = A' (A H^{-1} A')^{-1} A, Sec. 4.3, Lemma 1."""
    Hinv = np.linalg.inv(H)
    return A.T @ np.linalg.inv(A @ Hinv @ A.T) @ A


def kf_apply(H, A, C, D, p):
    """K_F p computed as the paper's three steps (Sec. 5.2): C'p, a solve with F,
    a product with C; plus the diagonal term D p."""
    n, m1 = H.shape[0], A.shape[0]
    rhs = np.concatenate([C.T @ p, np.zeros(m1)])
    y = np.linalg.solve(F_matrix(H, A), rhs)
    return D * p - C @ y[:n]


def r_nu(H, A, C, r_g, r_e, r_a):
    """r_nu = -r_a + [C 0] F^{-1} [r_g; r_e], Sec. 4.1, eq. [ineq-const-reduced]."""
    n = H.shape[0]
    y = np.linalg.solve(F_matrix(H, A), np.concatenate([r_g, r_e]))
    return -r_a + C @ y[:n]


def recover(H, A, C, r_g, r_e, dnu):
    """(dx, dlam) from F [dx; dlam] = -[r_g + C' dnu; r_e], Sec. 4.1, eq. [schur-delta-x]."""
    n = H.shape[0]
    z = np.linalg.solve(F_matrix(H, A), -np.concatenate([r_g + C.T @ dnu, r_e]))
    return z[:n], z[n:]


def newton_direction(H, A, C, s, nu, r_g, r_e, r_i, r_c):
    """Full Newton direction through the reduced system (direct K_F solve):
    D = V^{-1}S (eq. [diag-d]), r_a = r_i + V^{-1} r_c (eq. [augmented]),
    K_F dnu = r_nu (eq. [ineq-const-reduced]), recovery (eq. [schur-delta-x]),
    ds = -V^{-1} r_c - D dnu (eq. [delz])."""
    D = s / nu
    r_a = r_i + r_c / nu
    K = kf_explicit(H, A, C, D)
    dnu = np.linalg.solve(K, r_nu(H, A, C, r_g, r_e, r_a))
    dx, dlam = recover(H, A, C, r_g, r_e, dnu)
    ds = -r_c / nu - D * dnu
    return dx, dlam, dnu, ds


def P_L(D):
    """Low-degree-of-freedom preconditioner P_L = D, Sec. 4.2, eq. [preconditioner-1]."""
    return np.diag(D)


def P_H(H, C, D, exact=True):
    """High-degree-of-freedom preconditioner P_H = D + C H^{-1} C',
    Sec. 4.2, eq. [preconditioner-2]; ``exact=False`` replaces H^{-1} by
    diag(H)^{-1}, the choice of the experiments (Sec. 5.2, PH-KF variant)."""
    if exact:
        T = C @ np.linalg.solve(H, C.T)
    else:
        T = (C / np.diag(H)[None, :]) @ C.T
    return np.diag(D) + T


def pcg(apply_K, apply_Minv, rhs, tol, maxit):
    """Textbook preconditioned CG from a zero initial guess, stopping when
    ||r||_2 <= tol ||rhs||_2 (Sec. 6 setup: zero start, relative residual test).

    Returns (x, iterations, relres_history).  The iteration count is the number
    of products with K."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = float(np.linalg.norm(rhs))
    hist = [1.0]
    if bnorm == 0.0:
        return x, 0, hist
    z = apply_Minv(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < maxit:
        q = apply_K(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if rel <= tol:
            break
        z = apply_Minv(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist

