"""Exact optimum of a tiny strictly convex QP by active-set enumeration.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For every subset W of the inequality rows, solve the equality-constrained QP
with A and C_W as equalities (its KKT system: H x + c - A'lam - C_W' nu_W = 0,
A x = b, C_W x = d_W; Sec. 2 KKT conditions with the inactive multipliers set to
zero).  W is kept when x is feasible (C x >= d - tol) and the multipliers are
dual feasible (nu_W >= -tol).  Because H is positive definite the optimum is
unique, so every kept W gives the same x; the one with the smallest objective is
returned.  Cost 2^m2 small solves: meant for n <= 6, m2 <= 10.
"""
from __future__ import annotations

import itertools

import numpy as np


def bruteforce(H, c, A, b, C, d, tol=1e-9):
    n, m1, m2 = H.shape[0], A.shape[0], C.shape[0]
    best = None
    for size in range(0, min(m2, n - m1) + 1):
        for W in itertools.combinations(range(m2), size):
            W = list(W)
            Aw = np.vstack([A, C[W]]) if W else A
            bw = np.concatenate([b, d[W]]) if W else b
            k = Aw.shape[0]
            if k and np.linalg.matrix_rank(Aw) < k:
                continue
            K = np.zeros((n + k, n + k))
            K[:n, :n] = H
            K[:n, n:] = -Aw.T
            K[n:, :n] = Aw
            sol = np.linalg.solve(K, np.concatenate([-c, bw]))
            x, y = sol[:n], sol[n:]
            if np.any(C @ x < d - tol):
                continue
            if np.any(y[m1:] < -tol):
                continue
            f = 0.5 * float(x @ H @ x) + float(c @ x)
            if best is None or f < best[0]:
                nu = np.zeros(m2)
                nu[W] = y[m1:]
                best = (f, x, y[:m1], nu, W)
    if best is None:
        raise RuntimeError("no KKT point found (infeasible QP?)")
    f, x, lam, nu, W = best
    return dict(f=f, x=x, lam=lam, nu=nu, active=W)
