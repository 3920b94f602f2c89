"""Pins of the oracle's SG system (Eq. tensor-product, Sec. 3) against symmetry,
the sigma = 0 reduction, a Kronecker special case with a closed-form solution,
stochastic collocation and Monte Carlo means, and unpreconditioned GMRES."""
import math

import numpy as np
import scipy.sparse.linalg as spla

from oracle import basis, fem, kl, sg
from paper_1304_1755_gb300 import inputs


def _c1_like(n=9, M=2, p=2, sigma=0.3, family=basis.LEGENDRE):
    return sg.build(n, M, p, family, kl.kl_coefficients(n, M, sigma))


def test_matrix_free_apply_equals_assembled_and_symmetric():
    s = sg.build(9, 3, 3, basis.HERMITE, inputs.random_cell_coefficients(5, 9, 3))
    A = sg.assemble(s)
    X = inputs.uniform(6, s.P * s.Nx)
    assert np.allclose(sg.apply(s, X), A @ X, rtol=0, atol=1e-13)
    assert abs(A - A.T).max() < 1e-15


def test_sigma_zero_reduces_to_deterministic_problem():
    s = _c1_like(sigma=0.0)
    U = sg.solve_direct(sg.assemble(s), sg.rhs(s)).reshape(s.P, s.Nx)
    u0 = spla.spsolve(s.K[0].tocsc(), fem.load_vector(s.n))
    assert np.allclose(U[0], u0, atol=1e-15)
    assert np.abs(U[1:]).max() == 0.0


def test_kronecker_special_case_closed_form():
    """M = 1, spatially constant mode b_1 = 1: A = (I + sigma G_1) (x) K_0, so
    U* = ((I + sigma G_1)^{-1} e_0) (x) (K_0^{-1} F_0)."""
    n, p, sigma = 9, 4, 0.2
    coef = np.vstack([np.ones((n - 1) ** 2), sigma * np.ones((n - 1) ** 2)])
    for fam in (basis.LEGENDRE, basis.HERMITE):
        s = sg.build(n, 1, p, fam, coef)
        U = sg.solve_direct(sg.assemble(s), sg.rhs(s)).reshape(s.P, s.Nx)
        e0 = np.zeros(s.P)
        e0[0] = 1.0
        a = np.linalg.solve(np.eye(s.P) + sigma * s.G[1], e0)
        u0 = spla.spsolve(s.K[0].tocsc(), fem.load_vector(n))
        assert np.allclose(U, np.outer(a, u0), atol=1e-14 * np.abs(u0).max())


def _deterministic_solve(n, coef, xi):
    a = coef[0] + np.tensordot(xi, coef[1:], axes=1)
    K = fem.assemble_stiffness(n, a)
    return spla.spsolve(K.tocsc(), fem.load_vector(n))


def test_mean_and_variance_converge_to_collocation():
    """SG mean U_0 and variance sum_{i>=1} U_i^2 against tensor Gauss-Legendre quadrature of
    deterministic solves (stochastic collocation); the gap shrinks spectrally in p."""
    n, M, sigma = 9, 2, 0.3
    coef = kl.kl_coefficients(n, M, sigma)
    x, w = np.polynomial.legendre.leggauss(14)
    xi1, w1 = math.sqrt(3.0) * x, w / 2
    mean = np.zeros((n - 2) ** 2)
    second = np.zeros_like(mean)
    for a, wa in zip(xi1, w1):
        for b, wb in zip(xi1, w1):
            u = _deterministic_solve(n, coef, np.array([a, b]))
            mean += wa * wb * u
            second += wa * wb * u * u
    var = second - mean ** 2
    errs = []
    for p in (1, 2, 4, 6):
        s = sg.build(n, M, p, basis.LEGENDRE, coef)
        U = sg.solve_direct(sg.assemble(s), sg.rhs(s)).reshape(s.P, s.Nx)
        errs.append((np.abs(U[0] - mean).max() / np.abs(mean).max(),
                     np.abs((U[1:] ** 2).sum(0) - var).max() / np.abs(var).max()))
    assert errs[-1][0] < 1e-7 and errs[-1][1] < 1e-5
    assert all(errs[i + 1][0] < errs[i][0] for i in range(3))
    assert all(errs[i + 1][1] < errs[i][1] for i in range(3))


def test_mean_against_monte_carlo():
    n, M, sigma, N = 17, 2, 0.3, 4000
    coef = kl.kl_coefficients(n, M, sigma)
    g = inputs.rng(11)
    xis = g.uniform(-math.sqrt(3.0), math.sqrt(3.0), size=(N, M))
    samples = np.array([_deterministic_solve(n, coef, xi) for xi in xis])
    mc_mean, mc_std = samples.mean(0), samples.std(0)
    s = sg.build(n, M, 4, basis.LEGENDRE, coef)
    U = sg.solve_direct(sg.assemble(s), sg.rhs(s)).reshape(s.P, s.Nx)
    assert np.all(np.abs(U[0] - mc_mean) <= 4 * mc_std / math.sqrt(N) + 1e-6 * np.abs(mc_mean).max())


def test_plain_gmres_matches_direct():
    s = sg.build(33, 2, 2, basis.LEGENDRE, kl.kl_coefficients(33, 2, 0.3))
    A = sg.assemble(s)
    F = sg.rhs(s)
    Ud = sg.solve_direct(A, F)
    Ug, its, rr = sg.gmres_plain(lambda v: A @ v, F, tol=1e-12, restart=100, maxit=20000)
    assert rr <= 1e-12
    assert np.linalg.norm(Ug - Ud) / np.linalg.norm(Ud) < 1e-9
