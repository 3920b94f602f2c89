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
    for seed in range(100, 120):                          # the 20 seeded directions of the C4 check
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


def _small(sigma=0.3):
    """A small SG system (n = 9, M = 2, p = 2: 294 unknowns) with dense A and the two block
    preconditioners as dense matrices (exact K_0 solves), for the Krylov optimality pins."""
    n, M, p = 9, 2, 2
    s = sg.build(n, M, p, basis.LEGENDRE, kl.kl_coefficients(n, M, sigma))
    A = sg.assemble(s).toarray()
    solver = precond.DiagSolver(s.K[0])                   # sparse LU of K_0
    N = A.shape[0]
    BTinv = np.column_stack([precond.block_tri_inv(s, solver, e) for e in np.eye(N)])
    BDinv = np.column_stack([precond.block_diag_inv(s, solver, e) for e in np.eye(N)])
    b = np.random.default_rng(11).standard_normal(N)
    return A, BTinv, BDinv, b


def _krylov_basis(Op, v, k):
    """Orthonormal basis of span{v, Op v, ..., Op^(k-1) v} (Gram-Schmidt twice per vector)."""
    Q = np.zeros((len(v), k))
    w = v.copy()
    for j in range(k):
        for _ in range(2):
            w = w - Q[:, :j] @ (Q[:, :j].T @ w)
        Q[:, j] = w / np.linalg.norm(w)
        w = Op @ Q[:, j]
    return Q


def test_gmres_iterate_minimises_the_residual_over_the_krylov_space():
    """Right-preconditioned GMRES after k steps (no restart) returns the x in
    x0 + M K_k(A M, r0) of least residual norm: brute-force least squares on that space."""
    A, BTinv, _, b = _small()
    AM = A @ BTinv
    for k in (1, 2, 3, 5):
        x, its, _ = krylov.gmres(lambda v: A @ v, lambda r: BTinv @ r, b, tol=1e-300, restart=30, maxit=k)
        assert its == k
        Q = _krylov_basis(AM, b, k)
        y = np.linalg.lstsq(AM @ Q, b, rcond=None)[0]
        best = np.linalg.norm(b - AM @ (Q @ y))
        assert abs(np.linalg.norm(b - A @ x) - best) <= 1e-10 * np.linalg.norm(b)


def test_flexible_gmres_with_a_fixed_preconditioner_is_gmres():
    """With the same linear preconditioner at every step, flexible GMRES builds the same iterate."""
    A, BTinv, _, b = _small()
    for k in (2, 4, 7):
        x1 = krylov.gmres(lambda v: A @ v, lambda r: BTinv @ r, b, tol=1e-300, restart=30, maxit=k)[0]
        x2 = krylov.gmres(lambda v: A @ v, lambda r: BTinv @ r, b, tol=1e-300, restart=30, maxit=k, flexible=True)[0]
        assert np.linalg.norm(x1 - x2) <= 1e-11 * np.linalg.norm(x1)


def test_pcg_iterate_minimises_the_energy_error_over_the_krylov_space():
    """PCG with the SPD block-diagonal preconditioner after k steps returns the x in
    K_k(M A, M b) of least A-norm error (x0 = 0): brute force by the projected normal equations."""
    A, _, BDinv, b = _small()
    xs = np.linalg.solve(A, b)
    MA = BDinv @ A
    for k in (1, 2, 4, 6):
        x = krylov.pcg(lambda v: A @ v, lambda r: BDinv @ r, b, tol=1e-300, maxit=k)[0]
        Q = _krylov_basis(MA, BDinv @ b, k)
        y = np.linalg.solve(Q.T @ A @ Q, Q.T @ A @ xs)
        xb = Q @ y
        en = lambda z: np.sqrt((xs - z) @ A @ (xs - z))
        assert abs(en(x) - en(xb)) <= 1e-9 * en(np.zeros_like(b))


def test_gpcg1_with_a_symmetric_preconditioner_is_pcg():
    """GPCG[1] orthogonalises each new direction against the previous one only; with a symmetric
    positive definite preconditioner the conjugacy to all older directions holds by itself, so
    its iterates are those of PCG."""
    A, _, BDinv, b = _small()
    for k in (1, 3, 6, 9):
        x1 = krylov.gpcg1(lambda v: A @ v, lambda r: BDinv @ r, b, tol=1e-300, maxit=k)[0]
        x2 = krylov.pcg(lambda v: A @ v, lambda r: BDinv @ r, b, tol=1e-300, maxit=k)[0]
        assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x2)


def test_block_gauss_seidel_error_is_the_matrix_power():
    """The stationary iteration x <- x + B_T^-1 (b - A x) leaves the error (I - B_T^-1 A)^k e_0."""
    A, BTinv, _, b = _small()
    xs = np.linalg.solve(A, b)
    E = np.eye(A.shape[0]) - BTinv @ A
    for k in (1, 2, 5):
        x = krylov.block_gauss_seidel(lambda v: A @ v, lambda r: BTinv @ r, b, tol=1e-300, maxit=k)[0]
        e = np.linalg.matrix_power(E, k) @ (0 - xs)
        assert np.linalg.norm((x - xs) - e) <= 1e-10 * np.linalg.norm(xs)


def test_left_gmres_iterate_minimises_the_preconditioned_residual():
    """Left-preconditioned GMRES after k steps (no restart) returns the x in K_k(M A, M b) of least
    preconditioned residual ||M (b - A x)||: brute-force least squares on that space."""
    A, BTinv, _, b = _small()
    MA = BTinv @ A
    Mb = BTinv @ b
    for k in (1, 2, 4, 6):
        x, its, _ = krylov.gmres_left(lambda v: A @ v, lambda r: BTinv @ r, b, tol=1e-300, restart=30, maxit=k)
        assert its == k
        Q = _krylov_basis(MA, Mb, k)
        y = np.linalg.lstsq(MA @ Q, Mb, rcond=None)[0]
        best = np.linalg.norm(Mb - MA @ (Q @ y))
        assert abs(np.linalg.norm(Mb - MA @ x) - best) <= 1e-10 * np.linalg.norm(Mb)
