"""Pins of the oracle's Karhunen-Loeve expansion (Sec. 2.1, Eqs. truncated-KLE,
exponential-covariance) against the integral equation, Mercer's theorem and the
covariance trace -- all computed by independent quadrature here."""
import math

import numpy as np
import pytest

from oracle import kl


def _kernel_apply(b, s, a=0.5):
    """int_{-a}^{a} exp(-|s - t|) b(t) dt by Gauss-Legendre split at the kink t = s."""
    x, w = np.polynomial.legendre.leggauss(60)
    total = 0.0
    for lo, hi in ((-a, s), (s, a)):
        if hi - lo <= 0:
            continue
        t = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        total += 0.5 * (hi - lo) * np.sum(w * np.exp(-np.abs(s - t)) * b(t))
    return total


def test_1d_eigenpairs_solve_integral_equation():
    lam, om, par = kl.kl_1d(8)
    assert np.all(np.diff(lam) < 0)
    for k in range(8):
        b = lambda t, k=k: kl.eval_1d(om[k], par[k], t)
        for s in (-0.41, -0.1, 0.0, 0.23, 0.5):
            assert abs(_kernel_apply(b, s) - lam[k] * b(s)) < 1e-12


def test_1d_modes_orthonormal():
    lam, om, par = kl.kl_1d(8)
    x, w = np.polynomial.legendre.leggauss(80)
    t, w = 0.5 * x, 0.5 * w
    B = np.array([kl.eval_1d(om[k], par[k], t) for k in range(8)])
    gram = (B * w) @ B.T
    assert np.allclose(gram, np.eye(8), atol=1e-13)


def test_trace_of_covariance_is_one():
    # int C(s,s) ds = 1 on an interval of length 1; tail of sum lambda ~ 2/(pi^2 N)
    N = 400
    lam, _, _ = kl.kl_1d(N)
    tail = 1.0 - lam.sum()
    assert 0.5 * 2 / (math.pi ** 2 * N) < tail < 1.5 * 2 / (math.pi ** 2 * N)


def test_mercer_reconstruction():
    N = 600
    lam, om, par = kl.kl_1d(N)
    s, t = 0.17, -0.31
    approx = sum(lam[k] * kl.eval_1d(om[k], par[k], s) * kl.eval_1d(om[k], par[k], t) for k in range(N))
    assert abs(approx - math.exp(-abs(s - t))) < 2e-3


def test_2d_modes_sorted_with_tie_rule():
    modes = kl.kl_2d_modes(6)
    lams = [m[0] for m in modes]
    assert all(lams[i] >= lams[i + 1] for i in range(5))
    # equal products: lower x1-mode index first
    assert (modes[1][1], modes[1][2]) == (0, 1) and (modes[2][1], modes[2][2]) == (1, 0)
    assert (modes[3][1], modes[3][2]) == (0, 2) and (modes[4][1], modes[4][2]) == (2, 0)


def test_coefficients_layout_and_variance():
    n, M, sigma = 17, 4, 0.3
    c = kl.kl_coefficients(n, M, sigma)
    assert c.shape == (M + 1, 16 * 16)
    assert np.all(c[0] == 1.0)
    # pointwise variance of the truncated field sum_k c_k^2 <= sigma^2 (Bessel), cell mean close to
    # sigma^2 * sum lambda_k (orthonormal modes)
    var = np.sum(c[1:] ** 2, axis=0)
    assert np.all(var <= sigma ** 2 * (1 + 1e-12))
    lam2 = kl.kl_eigenvalues(M)
    assert abs(var.mean() - sigma ** 2 * lam2.sum()) < 0.02 * sigma ** 2
    # cell index e = cx + cy (n-1): mode 2 is (x1 mode 0, x2 mode 1) -> odd in x2, even in x1
    c2 = c[2].reshape(16, 16)
    assert np.allclose(c2, -c2[::-1, :], atol=1e-15)
    assert np.allclose(c2, c2[:, ::-1], atol=1e-15)


@pytest.mark.parametrize("n,M,sigma", [(5, 2, 0.3), (9, 4, 0.5), (9, 6, 0.4)])
def test_min_coefficient_at_corners_by_enumeration(n, M, sigma):
    """The closed form c_0 - sqrt3 sum|c_k| against brute force over all 2^M corners of the xi box,
    per cell, and no point inside the box below it."""
    import itertools
    coef = kl.kl_coefficients(n, M, sigma)
    coef[0] = 1.0 + 0.3 * np.sin(np.arange(coef.shape[1]))        # a non-constant mean as well
    r = math.sqrt(3.0)
    corners = np.array(list(itertools.product((-r, r), repeat=M)))  # (2^M, M)
    a_corners = coef[0][None, :] + corners @ coef[1:]               # (2^M, cells)
    assert kl.min_coefficient_at_corners(coef) == pytest.approx(a_corners.min(), abs=1e-14)
    inside = np.random.default_rng(3).uniform(-r, r, size=(500, M))
    assert (coef[0][None, :] + inside @ coef[1:]).min() >= a_corners.min() - 1e-14
    # another radius (a Hermite reference radius) scales the fluctuation part only
    half = coef[0] - 2.0 * np.abs(coef[1:]).sum(axis=0)
    assert kl.min_coefficient_at_corners(coef, 2.0) == pytest.approx(half.min(), abs=1e-14)
