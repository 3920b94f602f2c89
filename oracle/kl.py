"""Truncated Karhunen-Loeve expansion of the exponential covariance (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.1, Eq. (truncated-KLE):  a_m(x, xi) = abar(x) + sum_k sqrt(lambda_k) b_k(x) xi_k,
with (lambda_k, b_k) the eigenpairs of the covariance operator.
Eq. (exponential-covariance):   Cov(x, y) = sigma^2 exp(-|x - y| / L).

On the unit square the covariance is taken in its separable L1 form
exp(-|x1-y1|/L - |x2-y2|/L), so each 2-D eigenpair is a product of two 1-D
eigenpairs of the kernel exp(-|s-t|/L) on an interval of length 1.  The 1-D
problem on (-a, a) (a = 1/2, c = 1/L) has the classical solution
  even modes  b(y) = cos(w y) / sqrt(a + sin(2 w a) / (2 w)),   c - w tan(w a) = 0
  odd  modes  b(y) = sin(w y) / sqrt(a - sin(2 w a) / (2 w)),   w + c tan(w a) = 0
  lambda = 2 c / (w^2 + c^2).
sigma multiplies the unit-variance modes (the covariance carries sigma^2), so the
per-cell coefficient of mode k is c_k(e) = sigma sqrt(lambda_k) b_k(x_e) with x_e
the cell centre (coefficients are constant per Q1 cell).

Ties between 2-D modes (lambda_i lambda_j == lambda_j lambda_i) are broken by
putting the lower x1-mode index first.

Pins: the integral equation residual by independent quadrature, sum of 1-D
eigenvalues -> 1 (trace of the unit-variance covariance on a unit interval),
orthonormality of the modes; the coercivity minimum by enumeration of the corners of
the xi box.
"""
import math

import numpy as np
from scipy.optimize import brentq


def kl_1d(n_modes, corr_len=1.0, half_length=0.5):
    """First ``n_modes`` eigenpairs of exp(-|s-t|/L) on (-a, a), by decreasing lambda.

    Returns (lam, omega, parity) arrays; parity 0 = even (cos), 1 = odd (sin).
    """
    a = half_length
    c = 1.0 / corr_len
    lam, om, par = [], [], []
    k = 0
    while len(lam) < n_modes:
        # even root: w a in (k pi, k pi + pi/2)
        lo, hi = (k * math.pi) / a, (k * math.pi + math.pi / 2) / a
        eps = 1e-10 * hi
        f = lambda w: c - w * math.tan(w * a)
        w = brentq(f, lo + eps, hi - eps, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
        om.append(w), par.append(0), lam.append(2 * c / (w * w + c * c))
        if len(lam) >= n_modes:
            break
        # odd root: w a in (k pi + pi/2, k pi + pi)
        lo, hi = (k * math.pi + math.pi / 2) / a, (k * math.pi + math.pi) / a
        eps = 1e-10 * hi
        g = lambda w: w + c * math.tan(w * a)
        w = brentq(g, lo + eps, hi - eps, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
        om.append(w), par.append(1), lam.append(2 * c / (w * w + c * c))
        k += 1
    return np.array(lam), np.array(om), np.array(par)


def eval_1d(omega, parity, y, half_length=0.5):
    """Normalised 1-D eigenfunction at centred coordinate y (|y| <= a)."""
    a = half_length
    if parity == 0:
        return np.cos(omega * y) / math.sqrt(a + math.sin(2 * omega * a) / (2 * omega))
    return np.sin(omega * y) / math.sqrt(a - math.sin(2 * omega * a) / (2 * omega))


def kl_2d_modes(M, corr_len=1.0):
    """The M leading separable 2-D modes: list of (lambda, i, j) with 1-D mode indices."""
    lam1, _, _ = kl_1d(M + 1, corr_len)
    pairs = []
    for i in range(M + 1):
        for j in range(M + 1):
            pairs.append((lam1[i] * lam1[j], i, j))
    pairs.sort(key=lambda t: (-t[0], t[1]))
    return pairs[:M]


def kl_coefficients(n, M, sigma, abar=None, corr_len=1.0):
    """Per-cell coefficients c_k(e), k = 0..M, on the (n-1)^2 Q1 cells of [0,1]^2.

    Returns an (M+1, (n-1)^2) FP64 array, cell e = cx + cy (n-1); row 0 is the
    mean field abar (1 when not given), row k >= 1 is sigma sqrt(lambda_k) b_k(x_e).
    """
    nc1 = n - 1
    h = 1.0 / nc1
    lam1, om1, par1 = kl_1d(M + 1, corr_len)
    modes = kl_2d_modes(M, corr_len)
    centres = (np.arange(nc1) + 0.5) * h - 0.5          # centred coordinates
    coef = np.zeros((M + 1, nc1 * nc1))
    coef[0] = 1.0 if abar is None else np.asarray(abar, dtype=np.float64).reshape(-1)
    for k, (lam, i, j) in enumerate(modes, start=1):
        bx = eval_1d(om1[i], par1[i], centres)
        by = eval_1d(om1[j], par1[j], centres)
        coef[k] = sigma * math.sqrt(lam) * np.outer(by, bx).reshape(-1)   # row = cy, col = cx
    return coef


def kl_eigenvalues(M, corr_len=1.0):
    """lambda_k, k = 1..M, of the leading separable 2-D modes."""
    return np.array([m[0] for m in kl_2d_modes(M, corr_len)])


def kl_mode_sup(M, corr_len=1.0):
    """||b_k||_inf of each 2-D mode over the unit square (product of 1-D sups)."""
    lam1, om1, par1 = kl_1d(M + 1, corr_len)
    y = np.linspace(-0.5, 0.5, 20001)
    sup1 = [np.max(np.abs(eval_1d(om1[i], par1[i], y))) for i in range(M + 1)]
    return np.array([sup1[i] * sup1[j] for (_, i, j) in kl_2d_modes(M, corr_len)])


def min_coefficient_at_corners(coef, xi_max=math.sqrt(3.0)):
    """Coercivity check (Eq. assumption, Remark after Eq. exponential-covariance).

    Minimum over the cells of a = c_0 + sum_k c_k xi_k over the box |xi_k| <= xi_max
    (xi_max = sqrt3 is the support of the unit-variance uniform variables of the
    Legendre chaos).  a is linear in xi, so the minimum over the box sits at the
    corner xi_k = -xi_max sign(c_k), where it equals c_0 - xi_max sum_k |c_k|.
    Hermite variables are unbounded; there xi_max is a chosen reference radius.
    """
    return float(np.min(coef[0] - xi_max * np.sum(np.abs(coef[1:]), axis=0)))
