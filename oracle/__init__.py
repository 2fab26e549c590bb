"""FP64 CPU oracle for the preconditioned inexact IPM (Karim & Solomonik).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package; only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code,
constants or helpers with the CUDA library: the two only read the same seeded
inputs from ``qpgen``.

Citations name the paper's section and the equation's LaTeX label, written
eq. [label] (for example eq. [ineq-const-reduced] in Sec. 4.1).

Modules
-------
ipm         Primal-dual Mehrotra predictor-corrector IPM that factors the full
            unreduced 4x4 Newton system (Sec. 2, eqs. [sym-indef-KKT] and
            [rhs-KKT4]) with dense LU at every iteration; an LDL^T variant on the
            first augmented 3x3 system (Sec. 2.1, eq. [augmented]) for the larger
            workloads.
reduced     The method's own quantities written out by definition: F (eq. [f-def]),
            K_F and r_nu (eq. [ineq-const-reduced]), the recovery of (dx, dlam)
            (eq. [schur-delta-x]), the closed form through F_H (eq. [schur-R]),
            P_L (eq. [preconditioner-1]), P_H (eq. [preconditioner-2]) and a
            textbook preconditioned CG.
bruteforce  Active-set enumeration for tiny QPs (the exact optimum).

All functions use numpy/scipy in float64.  Pins (tests that fix the oracle to
something other than itself) live in tests/test_oracle_*.py.
"""
