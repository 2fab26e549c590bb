"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: exact enumeration, a closed form,
a theorem of the paper, an invariant, or a special case that reduces to a
textbook solve.  Tolerances are derived in the test from the stopping rule or
from the conditioning of the case.
"""
import numpy as np
import pytest

import qpgen
from oracle import bruteforce, ipm, reduced


# ---------------------------------------------------------------- exact optimum
@pytest.mark.parametrize("variant", ["kkt4", "kkt3"])
def test_ipm_matches_active_set_enumeration(variant):
    """200 tiny QPs: the IPM optimum equals the enumerated exact optimum.

    The stopping rule allows a duality gap s'nu = m2 mu <= m2 1e-11 (1+|f|), so the
    objective may differ by ~m2 1e-11 relative (m2 <= 10 -> 1e-10).  For x the gap
    only bounds the H-norm error, |x - x*|_H^2 <= 2 (gap + residual terms), which
    is loose near a weakly active constraint; x is held to 1e-7 here and the
    exactness of the IPM's limit point is pinned by the tight-tolerance test."""
    for seed in range(200):
        q = qpgen.tiny_qp(seed)
        bf = bruteforce.bruteforce(q.H, q.c, q.A, q.b, q.C, q.d)
        r = ipm.solve_qp(q, variant=variant)
        assert r.status == "optimal", seed
        ex = np.linalg.norm(r.x - bf["x"]) / max(1.0, np.linalg.norm(bf["x"]))
        ef = abs(r.f - bf["f"]) / max(1.0, abs(bf["f"]))
        assert ex <= 1e-7, (seed, ex)
        assert ef <= 1e-10, (seed, ef)


def test_ipm_tight_tolerance_reaches_exact_optimum():
    """With tighter stopping tolerances the IPM converges onto the enumerated
    optimum to near rounding level, multipliers included (LICQ holds)."""
    for seed in range(40):
        q = qpgen.tiny_qp(seed)
        bf = bruteforce.bruteforce(q.H, q.c, q.A, q.b, q.C, q.d)
        r = ipm.solve_qp(q, tol_feas=1e-13, tol_mu=1e-15)
        sc = max(1.0, np.linalg.norm(bf["x"]))
        assert np.linalg.norm(r.x - bf["x"]) / sc <= 1e-11, seed
        assert np.linalg.norm(r.nu - bf["nu"]) / max(1.0, np.linalg.norm(bf["nu"])) <= 1e-9, seed
        assert np.linalg.norm(r.lam - bf["lam"]) / max(1.0, np.linalg.norm(bf["lam"])) <= 1e-9, seed


def test_no_active_inequalities_reduces_to_equality_qp():
    """If every inequality is slack at the optimum (d pushed far below Cx), the
    optimum is the equality-constrained QP solution H x + c = A'lam, Ax = b,
    obtained here with one dense solve of [H -A'; A 0]."""
    q = qpgen.config_qp(0, scale=0.25)
    n, m1 = q.n, q.m1
    K = np.block([[q.H, -q.A.T], [q.A, np.zeros((m1, m1))]])
    sol = np.linalg.solve(K, np.concatenate([-q.c, q.b]))
    d = q.C @ sol[:n] - 10.0 - np.abs(q.C @ sol[:n])
    r = ipm.solve(q.H, q.c, q.A, q.b, q.C, d)
    assert r.status == "optimal"
    assert np.linalg.norm(r.x - sol[:n]) <= 1e-8 * max(1.0, np.linalg.norm(sol[:n]))
    assert np.linalg.norm(r.lam - sol[n:]) <= 1e-8 * max(1.0, np.linalg.norm(sol[n:]))
    assert np.max(np.abs(r.nu)) <= 1e-9


def test_kkt_conditions_at_oracle_output():
    """Sec. 2 KKT conditions hold at the returned point of the dense workload (n=120)."""
    q = qpgen.config_qp(0)
    r = ipm.solve_qp(q)
    rep = ipm.kkt_report(q.H, q.c, q.A, q.b, q.C, q.d, r.x, r.lam, r.nu, r.s)
    assert r.status == "optimal"
    assert rep["res_p"] <= 1e-10 and rep["res_d"] <= 1e-10
    assert rep["mu"] <= 1e-11 * (1 + abs(rep["f"]))
    assert rep["min_s"] > 0 and rep["min_nu"] > 0
    # primal feasibility of the original inequality (s is the slack)
    assert np.min(q.C @ r.x - q.d) >= -1e-9


def test_kkt3_and_kkt4_give_the_same_iterates():
    """The 3x3 LDL^T variant eliminates ds exactly (eq. [delz]): same iteration
    count and the same optimum as the 4x4 LU variant."""
    q = qpgen.config_qp(0)
    a = ipm.solve_qp(q, variant="kkt4")
    b = ipm.solve_qp(q, variant="kkt3")
    assert a.iters == b.iters
    assert np.linalg.norm(a.x - b.x) <= 1e-9 * np.linalg.norm(a.x)
    for ha, hb in zip(a.history, b.history):
        assert abs(ha["mu"] - hb["mu"]) <= 1e-8 * max(ha["mu"], 1e-12)


# ------------------------------------------------------ the reduction (Sec. 4.1)
def _iterates(q, count):
    """The first ``count`` oracle iterates (x, lam, nu, s) and their residuals."""
    out = []

    class Tap:
        def __init__(self, H, A, C, s, nu):
            self.k = ipm._KKT4(H, A, C, s, nu)
            out.append((s.copy(), nu.copy()))

        def solve(self, *a):
            return self.k.solve(*a)

    ipm.solve(q.H, q.c, q.A, q.b, q.C, q.d, newton=Tap, max_ipm=count)
    return out


def test_reduced_direction_equals_full_newton_direction():
    """Sec. 4.1: solving K_F dnu = r_nu and recovering (dx, dlam) from
    eq. [schur-delta-x] and ds from eq. [delz] gives exactly the direction of
    the full 4x4 system (eq. [sym-indef-KKT]).  Checked at the first 8 IPM
    iterates, where max(D)/min(D) stays below ~1e8 so that both dense solves
    are accurate to ~1e-12."""
    q = qpgen.config_qp(0, scale=0.3)
    rng = np.random.default_rng(5)
    for s, nu in _iterates(q, 8):
        r_g, r_e, r_i = (rng.standard_normal(q.n), rng.standard_normal(q.m1),
                         rng.standard_normal(q.m2))
        r_c = s * nu - 0.1 * float(s @ nu) / q.m2
        full = ipm._KKT4(q.H, q.A, q.C, s, nu).solve(r_g, r_e, r_i, r_c, nu)
        red = reduced.newton_direction(q.H, q.A, q.C, s, nu, r_g, r_e, r_i, r_c)
        for u, v in zip(full, red):
            assert np.linalg.norm(u - v) <= 1e-10 * np.linalg.norm(u)


def _small_case(seed, n=14, m1=5, m2=25, dlo=1e-2, dhi=1e2):
    q = qpgen.dense_qp(n, m1, m2, seed=seed)
    D, _ = qpgen.pcg_inputs(m2, seed, dlo, dhi)
    return q, D


def test_kf_closed_form_matches_definition():
    """eq. [ineq-const-reduced] (Schur complement of F) equals eq. [schur-R]
    (closed form through F_H = A H^{-1} A'), written with explicit inverses."""
    for seed in range(5):
        q, D = _small_case(seed, n=40, m1=12, m2=60)
        K1 = reduced.kf_explicit(q.H, q.A, q.C, D)
        K2 = reduced.kf_closed_form(q.H, q.A, q.C, D)
        assert np.linalg.norm(K1 - K2) <= 1e-10 * np.linalg.norm(K1)


def test_kf_apply_matches_explicit_matrix():
    """The three-step product (C'p, F solve, C y) equals K_F p."""
    q, D = _small_case(3)
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    p = np.random.default_rng(0).standard_normal(q.m2)
    assert np.allclose(reduced.kf_apply(q.H, q.A, q.C, D, p), K @ p, rtol=1e-11, atol=1e-11)


def test_kf_is_symmetric_positive_definite():
    """Sec. 4.1: K_F = D + (PSD term) is SPD and K_F - D is PSD."""
    for seed in range(5):
        q, D = _small_case(seed)
        K = reduced.kf_explicit(q.H, q.A, q.C, D)
        assert np.allclose(K, K.T, atol=1e-10 * np.abs(K).max())
        ev = np.linalg.eigvalsh(0.5 * (K + K.T))
        assert ev.min() > 0
        evm = np.linalg.eigvalsh(0.5 * (K + K.T) - np.diag(D))
        assert evm.min() >= -1e-10 * abs(evm).max()


def test_F_inertia():
    """Sec. 4.1: F has n negative and m1 positive eigenvalues (Haynsworth)."""
    q, _ = _small_case(1)
    ev = np.linalg.eigvalsh(reduced.F_matrix(q.H, q.A))
    assert int(np.sum(ev < 0)) == q.n and int(np.sum(ev > 0)) == q.m1


def test_lemma_ranks():
    """Lemma 1: rank(Hbar_A) <= m1; Lemma 2: rank(H - Hbar_A) <= n - m1
    (both attained for generic A)."""
    q, _ = _small_case(2, n=20, m1=7, m2=10)
    Hb = reduced.hbar_A(q.H, q.A)
    assert np.linalg.matrix_rank(Hb, tol=1e-9 * np.abs(Hb).max()) == q.m1
    R = q.H - Hb
    assert np.linalg.matrix_rank(R, tol=1e-9 * np.abs(q.H).max()) == q.n - q.m1


def _eig_precond(K, P):
    L = np.linalg.cholesky(P)
    Li = np.linalg.inv(L)
    return np.linalg.eigvalsh(Li @ K @ Li.T)


@pytest.mark.parametrize("seed", range(4))
def test_theorem1_PL_spectrum(seed):
    """Theorem 1: P_L^{-1/2} K_F P_L^{-1/2} = I + X has at most n-m1 non-unit
    eigenvalues, all >= 1."""
    q, D = _small_case(seed, n=16, m1=10, m2=30, dlo=1e-1, dhi=1e1)
    ev = _eig_precond(reduced.kf_explicit(q.H, q.A, q.C, D), reduced.P_L(D))
    nonunit = np.abs(ev - 1.0) > 1e-8 * ev.max()
    assert int(nonunit.sum()) <= q.n - q.m1
    assert ev.min() >= 1.0 - 1e-9


@pytest.mark.parametrize("seed", range(4))
def test_theorem2_PH_spectrum(seed):
    """Theorem 2: P_H^{-1/2} K_F P_H^{-1/2} = I - Y has at most m1 non-unit
    eigenvalues, all in (0, 1] (exact H^{-1} in P_H)."""
    q, D = _small_case(seed, n=16, m1=4, m2=30, dlo=1e-1, dhi=1e1)
    ev = _eig_precond(reduced.kf_explicit(q.H, q.A, q.C, D), reduced.P_H(q.H, q.C, D))
    nonunit = np.abs(ev - 1.0) > 1e-8
    assert int(nonunit.sum()) <= q.m1
    assert ev.min() > 0 and ev.max() <= 1.0 + 1e-9


def _pcg_iters(q, D, which, tol=1e-10):
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    rhs = np.random.default_rng(1).standard_normal(q.m2)
    if which == "PL":
        Minv = lambda r: r / D
    elif which == "PH":
        P = reduced.P_H(q.H, q.C, D)
        Minv = lambda r: np.linalg.solve(P, r)
    else:
        Minv = lambda r: r
    x, it, _ = reduced.pcg(lambda p: K @ p, Minv, rhs, tol, 10 * q.m2)
    return it, np.linalg.norm(x - np.linalg.solve(K, rhs)) / np.linalg.norm(np.linalg.solve(K, rhs))


def test_corollaries_cg_iteration_bounds():
    """Corollary 1 (P_L: <= n-m1+1 iterations) and Corollary 2 (P_H: <= m1+1).

    In exact arithmetic CG terminates at the bound.  In FP64 the unit-eigenvalue
    cluster is perturbed by rounding and the Krylov polynomial, whose roots sit on
    the few small non-unit eigenvalues, amplifies that perturbation (Sec. 6.2 notes
    the same deviation), so the count is taken at a 1e-6 relative residual with
    one iteration of slack.  Unpreconditioned CG needs many more."""
    q, D = _small_case(7, n=30, m1=24, m2=60, dlo=0.5, dhi=2.0)
    it, err = _pcg_iters(q, D, "PL", tol=1e-6)
    assert it <= (q.n - q.m1) + 1 + 1 and err < 1e-3
    q, D = _small_case(8, n=30, m1=3, m2=60, dlo=0.5, dhi=2.0)
    it, err = _pcg_iters(q, D, "PH", tol=1e-6)
    assert it <= q.m1 + 1 + 1 and err < 1e-3
    itu, _ = _pcg_iters(q, D, "none", tol=1e-6)
    assert itu > 3 * (q.m1 + 2)


def test_degenerate_cases_reduce_to_one_iteration():
    """m1 = n makes H - Hbar_A = 0, so K_F = D = P_L exactly; m1 = 0 makes
    K_F = D + C H^{-1} C' = P_H exactly.  PCG then stops after one iteration."""
    q, D = _small_case(9, n=12, m1=12, m2=20)
    assert _pcg_iters(q, D, "PL")[0] == 1
    q, D = _small_case(10, n=12, m1=0, m2=20)
    assert _pcg_iters(q, D, "PH")[0] == 1


def test_pcg_matches_direct_solve():
    """The textbook PCG reaches the direct solution of K_F within its tolerance
    times the condition number."""
    q, D = _small_case(11, n=30, m1=10, m2=50)
    for which in ("PL", "PH", "none"):
        it, err = _pcg_iters(q, D, which, tol=1e-12)
        assert err <= 1e-7, which


# ----------------------------------------------- mutations the pins must catch
def test_pins_catch_a_sign_error_in_K_F():
    """A planted mistake in the oracle (K_F with + F^{-1} instead of -) breaks
    the SPD / Theorem-1 facts: this shows those pins can fail."""
    q, D = _small_case(4, n=16, m1=10, m2=30, dlo=1e-1, dhi=1e1)
    good = reduced.kf_explicit(q.H, q.A, q.C, D)
    bad = 2 * np.diag(D) - good                     # D + [C 0] F^{-1} [C'; 0]
    ev = _eig_precond(bad, reduced.P_L(D))
    assert ev.min() < 1.0 - 1e-6


def test_pins_catch_the_garbled_r_a():
    """The text of Sec. 5.2 writes r_a = r_i - D r_c; eq. [augmented] defines
    r_a = r_i + V^{-1} r_c.  Planting the former breaks the full-vs-reduced
    direction agreement, so the oracle follows eq. [augmented]."""
    q = qpgen.config_qp(0, scale=0.3)
    s, nu = _iterates(q, 2)[-1]
    rng = np.random.default_rng(2)
    r_g, r_e, r_i = rng.standard_normal(q.n), rng.standard_normal(q.m1), rng.standard_normal(q.m2)
    r_c = s * nu
    full = ipm._KKT4(q.H, q.A, q.C, s, nu).solve(r_g, r_e, r_i, r_c, nu)
    D = s / nu
    K = reduced.kf_explicit(q.H, q.A, q.C, D)
    dnu_bad = np.linalg.solve(K, reduced.r_nu(q.H, q.A, q.C, r_g, r_e, r_i - D * r_c))
    assert np.linalg.norm(dnu_bad - full[2]) > 1e-3 * np.linalg.norm(full[2])


# ------------------------------------- P_H with diag(H)^{-1} (the experiments' variant)
def test_PH_diag_variant_equals_exact_for_diagonal_H():
    """With a diagonal H, diag(H)^{-1} = H^{-1}, so the variant of Sec. 5.2 (PH-KF)
    coincides with the P_H of eq. [preconditioner-2]."""
    rng = np.random.default_rng(5)
    h = rng.uniform(0.3, 7.0, 9)
    C = rng.standard_normal((13, 9))
    D = rng.uniform(0.1, 2.0, 13)
    exact = reduced.P_H(np.diag(h), C, D, exact=True)
    diag = reduced.P_H(np.diag(h), C, D, exact=False)
    assert np.allclose(diag, exact, rtol=1e-13, atol=1e-13)


def test_PH_diag_variant_hand_computed():
    """A case worked by hand.  H = [[2,1,0],[1,4,1],[0,1,5]] (its off-diagonal
    entries must be ignored), C = [[1,0,2],[0,1,-1]], D = (0.5, 0.25):
      C diag(H)^{-1} C' = [[1/2 + 4/5, -2/5], [-2/5, 1/4 + 1/5]] = [[1.3, -0.4], [-0.4, 0.45]],
      P_H(diag) = D + that = [[1.8, -0.4], [-0.4, 0.7]].
    The exact P_H differs: det(H) = 33, adj(H) = [[19,-5,1],[-5,10,-2],[1,-2,7]], so
      C H^{-1} C' = (1/33) [[51, -24], [-24, 21]],
      P_H(exact) = [[0.5 + 51/33, -24/33], [-24/33, 0.25 + 21/33]]."""
    H = np.array([[2.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.0, 1.0, 5.0]])
    C = np.array([[1.0, 0.0, 2.0], [0.0, 1.0, -1.0]])
    D = np.array([0.5, 0.25])
    assert np.allclose(reduced.P_H(H, C, D, exact=False), [[1.8, -0.4], [-0.4, 0.7]], rtol=0, atol=1e-15)
    want = np.array([[0.5 + 51 / 33, -24 / 33], [-24 / 33, 0.25 + 21 / 33]])
    assert np.allclose(reduced.P_H(H, C, D, exact=True), want, rtol=0, atol=1e-14)


def test_pins_catch_diag_H_instead_of_its_inverse():
    """A planted slip, C diag(H) C' in place of C diag(H)^{-1} C', misses the
    hand-computed values above (so that pin can fail)."""
    H = np.array([[2.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.0, 1.0, 5.0]])
    C = np.array([[1.0, 0.0, 2.0], [0.0, 1.0, -1.0]])
    D = np.array([0.5, 0.25])
    bad = np.diag(D) + (C * np.diag(H)[None, :]) @ C.T
    assert not np.allclose(bad, [[1.8, -0.4], [-0.4, 0.7]], rtol=0, atol=1e-3)
