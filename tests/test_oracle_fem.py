"""Pins of the oracle's Q1 stiffness matrices (Eq. def-stiffness) and of the
multigrid transfer operators against closed forms and independent quadrature."""
import numpy as np

from oracle import fem, mg
from paper_1304_1755_gb300 import inputs


def test_reference_element_matrix_textbook():
    K = fem.q1_reference_stiffness()
    ref = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    assert np.allclose(K, ref, atol=1e-15)
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-15)


def test_laplacian_spectrum_closed_form():
    for n in (9, 17):
        K0 = fem.assemble_stiffness(n, np.ones((n - 1) ** 2)).toarray()
        ev = np.sort(np.linalg.eigvalsh(K0))
        assert np.allclose(ev, fem.laplacian_q1_eigenvalues(n), atol=1e-12)


def test_energy_matches_independent_quadrature():
    """u^T K u = sum_e c_e int_e |grad u_h|^2 with u_h bilinear, by 3x3 Gauss per cell."""
    n = 9
    c = inputs.random_cell_coefficients(3, n, 0)[0]
    u = inputs.uniform(4, (n - 2) ** 2)
    K = fem.assemble_stiffness(n, c)
    h = 1.0 / (n - 1)
    U = np.zeros((n, n))
    U[1:-1, 1:-1] = u.reshape(n - 2, n - 2)          # U[vy, vx]
    x, w = np.polynomial.legendre.leggauss(3)
    x, w = 0.5 * x + 0.5, 0.5 * w
    energy = 0.0
    for cy in range(n - 1):
        for cx in range(n - 1):
            sw, se, ne, nw = U[cy, cx], U[cy, cx + 1], U[cy + 1, cx + 1], U[cy + 1, cx]
            for i in range(3):
                for j in range(3):
                    s, t = x[i], x[j]
                    dx = ((se - sw) * (1 - t) + (ne - nw) * t) / h
                    dy = ((nw - sw) * (1 - s) + (ne - se) * s) / h
                    energy += c[cx + cy * (n - 1)] * w[i] * w[j] * h * h * (dx * dx + dy * dy)
    assert abs(u @ (K @ u) - energy) < 1e-12 * abs(energy)


def test_galerkin_coarse_operator_of_constant_q1_is_q1():
    for n in (9, 17, 33):
        Kf = fem.assemble_stiffness(n, np.ones((n - 1) ** 2))
        P = mg.prolongation((n + 1) // 2)
        Kc = fem.assemble_stiffness((n + 1) // 2, np.ones(((n + 1) // 2 - 1) ** 2))
        assert abs(P.T @ Kf @ P - Kc).max() < 1e-13


def test_prolongation_reproduces_bilinear_functions():
    nc = 9
    nf = 2 * nc - 1
    P = mg.prolongation(nc)
    xc = np.linspace(0, 1, nc)[1:-1]
    Xc, Yc = np.meshgrid(xc, xc)
    g = lambda X, Y: (2 * X - 1) * (3 * Y + 1)                         # a bilinear function
    uc = g(Xc, Yc).reshape(-1)
    xf = np.linspace(0, 1, nf)[1:-1]
    Xf, Yf = np.meshgrid(xf, xf)
    # away from the boundary ring, bilinear interpolation of a bilinear function is exact
    uf = (P @ uc).reshape(nf - 2, nf - 2)
    ref = g(Xf, Yf)
    assert np.allclose(uf[2:-2, 2:-2], ref[2:-2, 2:-2], atol=1e-14)


def test_load_vector_f1_is_hat_integral():
    n = 17
    F = fem.load_vector(n)
    assert np.allclose(F, (1.0 / 16) ** 2)
