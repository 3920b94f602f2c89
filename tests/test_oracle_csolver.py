"""Pins of the oracle's C/OpenMP block-triangular FGMRES (oracle/csolve.c), the CPU baseline of
the benchmark: its solution against the sparse direct solve (SuperLU), and each of its steps
against the Python oracle's on the same seeded inputs (operator, V-cycle, B_T^{-1}, and the
FGMRES iteration count and iterate)."""
import numpy as np
import pytest

from oracle import basis, csolver, kl, krylov, mg, precond, sg as osg
from paper_1304_1755_gb300 import inputs


def _system(n, M, p, fam, sigma, mean="one", nu=(1, 1)):
    coef = kl.kl_coefficients(n, M, sigma)
    if mean == "lognormal":
        coef[0] = inputs.lognormal_cells(2, n, 0.2)
    s = osg.build(n, M, p, fam, coef)
    h = mg.Hierarchy(s.K[0], n, nu1=nu[0], nu2=nu[1])
    return s, h, csolver.CSolver(s, h)


CASES = [(9, 2, 3, basis.HERMITE, 0.3, "one", (1, 1)), (33, 2, 2, basis.LEGENDRE, 0.3, "one", (1, 1)),
         (17, 3, 2, basis.LEGENDRE, 0.25, "lognormal", (2, 1))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}M{c[1]}p{c[2]}{c[5]}")
def test_c_steps_match_python_oracle(case):
    s, h, c = _system(*case)
    X = inputs.uniform(61, s.P * s.Nx)
    assert np.abs(c.apply(X) - osg.apply(s, X)).max() <= 1e-14 * np.abs(X).max() * 8
    Xm = X.reshape(s.P, s.Nx)
    assert np.abs(c.vcycles(X, s.P).reshape(s.P, -1) - h.vcycle(Xm.T).T).max() <= 1e-13 * np.abs(X).max()
    sol = precond.DiagSolver(s.K[0], h)
    for tr in (False, True):
        ref = precond.block_tri_inv(s, sol, X, transpose=tr)
        assert np.abs(c.precond_bt(X, transpose=tr) - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}M{c[1]}p{c[2]}{c[5]}")
def test_c_fgmres_matches_direct_solution(case):
    s, h, c = _system(*case)
    F = osg.rhs(s, inputs.rhs_nodes(1, s.n))
    A = osg.assemble(s)
    Ustar = osg.solve_direct(A, F)
    U, its, rr, rc, _ = c.fgmres(F, restart=30, tol=1e-12)
    assert rc == 0 and rr <= 1e-12
    assert np.linalg.norm(U - Ustar) <= 1e-8 * np.linalg.norm(Ustar)
    sol = precond.DiagSolver(s.K[0], h)
    U2, its2, _ = krylov.gmres(lambda v: A @ v, lambda r: precond.block_tri_inv(s, sol, r), F, tol=1e-12,
                               restart=30, flexible=True)
    assert its == its2
    assert np.linalg.norm(U - U2) <= 1e-10 * np.linalg.norm(U2)


def test_c_fgmres_restart_and_maxit():
    s, h, c = _system(33, 2, 2, basis.LEGENDRE, 0.3)
    F = osg.rhs(s)
    U, its, rr, rc, _ = c.fgmres(F, restart=3, tol=1e-10)
    assert rc == 0 and rr <= 1e-10 and its > 3
    _, its2, _, rc2, _ = c.fgmres(F, restart=3, maxit=4, tol=1e-14)
    assert rc2 == 1 and its2 == 4
    Z, its0, rr0, rc0, _ = c.fgmres(np.zeros_like(F))
    assert rc0 == 0 and its0 == 0 and not Z.any()


def test_c_oracle_uses_threads():
    assert csolver.threads() >= 1


def test_c_adjoint_fgmres_matches_direct_transpose_solution():
    s, h, c = _system(17, 3, 2, basis.LEGENDRE, 0.25, "lognormal", (1, 1))
    F = inputs.uniform(62, s.P * s.Nx)
    A = osg.assemble(s)
    Ustar = osg.solve_direct(A.T.tocsr(), F)
    U, its, rr, rc, _ = c.fgmres(F, restart=30, tol=1e-12, transpose=True)
    assert rc == 0 and rr <= 1e-12
    assert np.linalg.norm(U - Ustar) <= 1e-8 * np.linalg.norm(Ustar)
