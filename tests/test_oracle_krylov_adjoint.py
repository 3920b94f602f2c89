"""Pins of the oracle's Krylov drivers (Sec. 4.2, 6) against the direct solve and
the ideal-Schur two-iteration property, and of its adjoint gradient against
central finite differences of the objective."""
import numpy as np

from oracle import adjoint, basis, kl, krylov, mg, precond, sg
from paper_1304_1755_gb300 import inputs


def _c1():
    n, M, p, sigma = 33, 2, 2, 0.3
    s = sg.build(n, M, p, basis.LEGENDRE, kl.kl_coefficients(n, M, sigma))
    A = sg.assemble(s)
    F = sg.rhs(s)
    hier = mg.Hierarchy(s.K[0], n)
    solver = precond.DiagSolver(s.K[0], hier)
    return s, A, F, solver


def test_preconditioned_solvers_match_direct_c1():
    s, A, F, solver = _c1()
    Ud = sg.solve_direct(A, F)
    Av = lambda v: A @ v
    BT = lambda r: precond.block_tri_inv(s, solver, r)
    BD = lambda r: precond.block_diag_inv(s, solver, r)
    runs = {
        "BT-FGMRES": krylov.gmres(Av, BT, F, tol=1e-12, restart=30, flexible=True),
        "BT-GMRES": krylov.gmres(Av, BT, F, tol=1e-12, restart=30),
        "BD-GMRES": krylov.gmres(Av, BD, F, tol=1e-12, restart=30),
        "BT-GPCG": krylov.gpcg1(Av, BT, F, tol=1e-12),
        "BD-PCG": krylov.pcg(Av, BD, F, tol=1e-12),
    }
    for name, (U, its, rr) in runs.items():
        assert rr <= 1e-12, name
        assert np.linalg.norm(U - Ud) / np.linalg.norm(Ud) < 1e-9, name
        assert its < 60, name
    # block-triangular needs fewer iterations than block-diagonal (Sec. 6, Tables 2-3)
    assert runs["BT-FGMRES"][1] < runs["BD-GMRES"][1]


def test_ideal_schur_gmres_two_iterations():
    n, M, p = 5, 2, 2
    s = sg.build(n, M, p, basis.LEGENDRE, kl.kl_coefficients(n, M, 0.4))
    A = sg.assemble(s).toarray()
    Ph = basis.n_basis(M, p - 1) * s.Nx
    Ah, W, D = A[:Ph, :Ph], A[Ph:, :Ph], A[Ph:, Ph:]
    S = D - W @ np.linalg.solve(Ah, W.T)
    Bt = np.block([[Ah, np.zeros_like(W.T)], [W, S]])
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x, its, rr = krylov.gmres(lambda v: A @ v, lambda r: np.linalg.solve(Bt, r), b, tol=1e-11, restart=10)
    assert its <= 2 and rr <= 1e-10


def test_adjoint_gradient_matches_central_differences():
    n, M, p, sigma = 9, 2, 2, 0.4
    abar = inputs.lognormal_cells(2, n, 0.2)
    unit = kl.kl_coefficients(n, M, 1.0)

    def J_of(ab, sg_):
        coef = unit.copy()
        coef[0] = ab
        coef[1:] *= sg_
        s_ = sg.build(n, M, p, basis.LEGENDRE, coef)
        U = sg.solve_direct(sg.assemble(s_), sg.rhs(s_))
        return adjoint.objective(s_, U)[0]

    coef = unit.copy()
    coef[0] = abar
    coef[1:] *= sigma
    s = sg.build(n, M, p, basis.LEGENDRE, coef)
    J, U, Lam, g_abar, g_sigma = adjoint.solve_and_gradients(s, unit)
    assert abs(J - J_of(abar, sigma)) < 1e-15
    eps = 1e-5
    for seed in range(100, 104):
        d = inputs.normal(seed, abar.shape)
        fd = (J_of(abar + eps * d, sigma) - J_of(abar - eps * d, sigma)) / (2 * eps)
        assert abs(fd - g_abar @ d) < 1e-7 * abs(fd) + 1e-14
    fd = (J_of(abar, sigma + eps) - J_of(abar, sigma - eps)) / (2 * eps)
    assert abs(fd - g_sigma) < 1e-7 * abs(fd)


def test_block_gauss_seidel_and_bs_pcg_match_direct():
    s, A, F, solver = _c1()
    Ud = sg.solve_direct(A, F)
    Av = lambda v: A @ v
    U, its, rr = krylov.block_gauss_seidel(Av, lambda r: precond.block_tri_inv(s, solver, r), F, tol=1e-12)
    assert rr <= 1e-12 and np.linalg.norm(U - Ud) / np.linalg.norm(Ud) < 1e-9
    # one step from zero is exactly the block-triangular preconditioner applied to F
    U1, _, _ = krylov.block_gauss_seidel(Av, lambda r: precond.block_tri_inv(s, solver, r), F, maxit=1)
    assert np.allclose(U1, precond.block_tri_inv(s, solver, F), atol=1e-15)
    U, its2, rr = krylov.pcg(Av, lambda r: precond.block_sym_inv(s, solver, r), F, tol=1e-12)
    assert rr <= 1e-12 and np.linalg.norm(U - Ud) / np.linalg.norm(Ud) < 1e-9
    assert its2 < its
