"""Oracle interior-point method: FP64, full KKT system factored at every iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

What it follows
---------------
* Sec. 2, eq. [nonlinear] / [duality]: perturbed KKT conditions with slack s > 0,
  multipliers nu > 0, duality measure mu = s'nu / m2 and centering sigma in [0, 1].
* Sec. 2, eq. [sym-indef-KKT] with right-hand side eq. [rhs-KKT4]: the symmetrised
  4x4 Newton system in (dx, dlam, dnu, ds).  ``variant="kkt4"`` assembles it and
  factors it with dense LU (partial pivoting) once per iteration.
* Sec. 2.1, eqs. [delz], [diag-d], [augmented]: ds eliminated with D = V^{-1} S,
  giving the first augmented 3x3 system with r_a = r_i + V^{-1} r_c.
  ``variant="kkt3"`` factors that symmetric indefinite matrix with LAPACK sytrf
  (Bunch-Kaufman) and recovers ds from eq. [delz].

Readings where the paper is silent (it fixes sigma in [0,1] only)
-----------------------------------------------------------------
* Start point: x0, lam0 from the equality-only QP (K0 [x; -lam] = [-c; b] with
  K0 = [H A'; A 0]); s0 = max(C x0 - d, 1) elementwise; nu0 = 1.
* Mehrotra predictor-corrector (the paper's IPM reference, Nocedal & Wright
  ch. 16): affine step with sigma = 0; sigma = (mu_aff / mu)^3; the corrector
  solves once more with r_c = S V e + dS_aff dV_aff e - sigma mu e, reusing the
  same factorization.
* One step length for primal and dual variables (H couples them),
  fraction-to-boundary tau = 0.995 on (s, nu); the affine step uses tau = 1.
* Stop when res_p = max(|r_e|_inf/(1+|b|_inf), |r_i|_inf/(1+|d|_inf)) <= tol_feas,
  res_d = |r_g|_inf / (1 + |c|_inf + |H|_inf) <= tol_feas and
  mu <= tol_mu (1 + |f|); defaults 1e-10, 1e-10, 1e-11; at most 100 iterations.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack

TAU = 0.995


@dataclasses.dataclass
class IPMResult:
    x: np.ndarray
    lam: np.ndarray
    nu: np.ndarray
    s: np.ndarray
    f: float
    iters: int
    status: str
    history: list


def objective(H, c, x):
    """f(x) = 1/2 x'Hx + c'x (Sec. 1, eq. [qp])."""
    return 0.5 * float(x @ (H @ x)) + float(c @ x)


def kkt_residuals(H, c, A, b, C, d, x, lam, nu, s):
    """r_g, r_e, r_i of eq. [rhs-KKT4] (r_c depends on sigma and is formed by the caller)."""
    r_g = -H @ x - c + A.T @ lam + C.T @ nu
    r_e = A @ x - b
    r_i = C @ x - d - s
    return r_g, r_e, r_i


def _ninf(v):
    return float(np.max(np.abs(v))) if v.size else 0.0


def scaled_residuals(H, c, b, d, r_g, r_e, r_i):
    """Scaled primal and dual infeasibility used by the stopping rule."""
    res_p = max(_ninf(r_e) / (1.0 + _ninf(b)), _ninf(r_i) / (1.0 + _ninf(d)))
    h_inf = float(np.max(np.sum(np.abs(H), axis=1)))
    res_d = _ninf(r_g) / (1.0 + _ninf(c) + h_inf)
    return res_p, res_d


def max_step(s, ds, nu, dnu):
    """Largest alpha with s + alpha ds >= 0 and nu + alpha dnu >= 0 (inf if unbounded)."""
    a = np.inf
    neg = ds < 0
    if np.any(neg):
        a = min(a, float(np.min(-s[neg] / ds[neg])))
    neg = dnu < 0
    if np.any(neg):
        a = min(a, float(np.min(-nu[neg] / dnu[neg])))
    return a


def k0_matrix(H, A):
    """K0 = [H A'; A 0], the equality-only KKT matrix."""
    n, m1 = H.shape[0], A.shape[0]
    K = np.zeros((n + m1, n + m1))
    K[:n, :n] = H
    K[:n, n:] = A.T
    K[n:, :n] = A
    return K


def start_point(H, c, A, b, C, d):
    """Equality-only QP solution for (x0, lam0); s0 = max(C x0 - d, 1); nu0 = 1."""
    n, m1 = H.shape[0], A.shape[0]
    sol = np.linalg.solve(k0_matrix(H, A), np.concatenate([-c, b]))
    x = sol[:n]
    lam = -sol[n:]
    s = np.maximum(C @ x - d, 1.0)
    nu = np.ones(C.shape[0])
    return x, lam, nu, s


class _KKT4:
    """Full 4x4 Newton matrix of eq. [sym-indef-KKT], dense LU."""

    def __init__(self, H, A, C, s, nu):
        n, m1, m2 = H.shape[0], A.shape[0], C.shape[0]
        N = n + m1 + 2 * m2
        K = np.zeros((N, N))
        i1, i2, i3 = n, n + m1, n + m1 + m2
        K[:i1, :i1] = -H
        K[:i1, i1:i2] = A.T
        K[:i1, i2:i3] = C.T
        K[i1:i2, :i1] = A
        K[i2:i3, :i1] = C
        K[i2:i3, i3:] = -np.eye(m2)
        K[i3:, i2:i3] = np.diag(s)
        K[i3:, i3:] = np.diag(nu)
        self.idx = (i1, i2, i3)
        self.lu = sla.lu_factor(K)

    def solve(self, r_g, r_e, r_i, r_c, nu):
        i1, i2, i3 = self.idx
        z = sla.lu_solve(self.lu, -np.concatenate([r_g, r_e, r_i, r_c]))
        return z[:i1], z[i1:i2], z[i2:i3], z[i3:]


class _KKT3:
    """First augmented 3x3 system of eq. [augmented], LAPACK sytrf/sytrs."""

    def __init__(self, H, A, C, s, nu):
        n, m1, m2 = H.shape[0], A.shape[0], C.shape[0]
        N = n + m1 + m2
        K = np.zeros((N, N))
        i1, i2 = n, n + m1
        K[:i1, :i1] = -H
        K[:i1, i1:i2] = A.T
        K[:i1, i2:] = C.T
        K[i1:i2, :i1] = A
        K[i2:, :i1] = C
        self.D = s / nu                                  # eq. [diag-d]
        K[i2:, i2:] = np.diag(self.D)
        self.idx = (i1, i2)
        ldu, ipiv, info = lapack.dsytrf(K, lower=1, lwork=max(1, 64 * N))
        if info < 0:
            raise RuntimeError(f"dsytrf argument error {info}")
        self.ldu, self.ipiv = ldu, ipiv

    def solve(self, r_g, r_e, r_i, r_c, nu):
        i1, i2 = self.idx
        r_a = r_i + r_c / nu                             # eq. [augmented], r_a
        rhs = -np.concatenate([r_g, r_e, r_a])
        z, info = lapack.dsytrs(self.ldu, self.ipiv, rhs[:, None], lower=1)
        z = z[:, 0]
        dx, dlam, dnu = z[:i1], z[i1:i2], z[i2:]
        ds = -r_c / nu - self.D * dnu                    # eq. [delz]
        return dx, dlam, dnu, ds


def solve(H, c, A, b, C, d, variant="kkt4", tol_feas=1e-10, tol_mu=1e-11,
          max_ipm=100, newton=None) -> IPMResult:
    """Mehrotra predictor-corrector IPM on min 1/2x'Hx+c'x s.t. Ax=b, Cx>=d.

    ``newton`` (optional) replaces the direction solver: a factory
    ``newton(H, A, C, s, nu)`` returning an object with
    ``solve(r_g, r_e, r_i, r_c, nu) -> (dx, dlam, dnu, ds)``.
    """
    m2 = C.shape[0]
    x, lam, nu, s = start_point(H, c, A, b, C, d)
    factory = newton or {"kkt4": _KKT4, "kkt3": _KKT3}[variant]
    history = []
    status = "max_iter"
    k = 0
    while True:
        r_g, r_e, r_i = kkt_residuals(H, c, A, b, C, d, x, lam, nu, s)
        mu = float(s @ nu) / m2
        f = objective(H, c, x)
        res_p, res_d = scaled_residuals(H, c, b, d, r_g, r_e, r_i)
        rec = dict(k=k, mu=mu, res_p=res_p, res_d=res_d, f=f)
        history.append(rec)
        if res_p <= tol_feas and res_d <= tol_feas and mu <= tol_mu * (1.0 + abs(f)):
            status = "optimal"
            break
        if k >= max_ipm:
            break
        kkt = factory(H, A, C, s, nu)
        # predictor (affine scaling), sigma = 0
        r_c = s * nu
        dx_a, dl_a, dn_a, ds_a = kkt.solve(r_g, r_e, r_i, r_c, nu)
        a_aff = min(1.0, max_step(s, ds_a, nu, dn_a))
        mu_aff = float((s + a_aff * ds_a) @ (nu + a_aff * dn_a)) / m2
        sigma = (mu_aff / mu) ** 3
        # corrector with the second-order term
        r_c = s * nu + ds_a * dn_a - sigma * mu
        dx, dl, dn, ds = kkt.solve(r_g, r_e, r_i, r_c, nu)
        alpha = min(1.0, TAU * max_step(s, ds, nu, dn))
        rec.update(sigma=sigma, alpha=alpha, alpha_aff=a_aff)
        x = x + alpha * dx
        lam = lam + alpha * dl
        nu = nu + alpha * dn
        s = s + alpha * ds
        k += 1
    return IPMResult(x=x, lam=lam, nu=nu, s=s, f=objective(H, c, x), iters=k,
                     status=status, history=history)


def solve_qp(qp, **kw) -> IPMResult:
    """``solve`` on a qpgen.QP (expands a CSR C to dense)."""
    return solve(qp.H, qp.c, qp.A, qp.b, qp.C_dense(), qp.d, **kw)


def kkt_report(H, c, A, b, C, d, x, lam, nu, s):
    """Optimality measures at a point (KKT conditions of Sec. 2, eq. [nonlinear] with sigma=0)."""
    r_g, r_e, r_i = kkt_residuals(H, c, A, b, C, d, x, lam, nu, s)
    res_p, res_d = scaled_residuals(H, c, b, d, r_g, r_e, r_i)
    return dict(res_p=res_p, res_d=res_d, mu=float(s @ nu) / C.shape[0],
                min_s=float(np.min(s)) if s.size else 0.0,
                min_nu=float(np.min(nu)) if nu.size else 0.0,
                f=objective(H, c, x))
