"""Pins of the oracle's gPC basis and stochastic matrices (Sec. 2.2, Eq.
def-stochastic, Sec. 3.2-3.3, Table 1) against Gauss quadrature of the
triple products with independently built orthonormal polynomials."""
import json
import math
import os
from itertools import product

import numpy as np
import pytest

from oracle import basis

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _ortho_1d(family, nmax):
    """Orthonormal 1-D polynomials as callables plus a quadrature rule for the density."""
    if family == basis.LEGENDRE:
        x, w = np.polynomial.legendre.leggauss(nmax + 4)
        xi, w = math.sqrt(3.0) * x, w / 2.0              # U(-sqrt3, sqrt3)
        polys = [lambda t, n=n: math.sqrt(2 * n + 1) * np.polynomial.legendre.legval(t / math.sqrt(3.0), [0] * n + [1])
                 for n in range(nmax + 1)]
    else:
        x, w = np.polynomial.hermite_e.hermegauss(nmax + 4)
        xi, w = x, w / math.sqrt(2 * math.pi)            # N(0, 1)
        polys = [lambda t, n=n: np.polynomial.hermite_e.hermeval(t, [0] * n + [1]) / math.sqrt(math.factorial(n))
                 for n in range(nmax + 1)]
    return xi, w, polys


def test_n_basis_formula_and_paper_example():
    ex = GOLD["n_basis_example"]
    assert basis.n_basis(ex["m"], ex["p"]) == ex["N_xi"]
    for M in range(1, 7):
        for p in range(0, 5):
            al = basis.multi_indices(M, p)
            assert len(al) == basis.n_basis(M, p) == len(set(al))
            degs = [sum(a) for a in al]
            assert degs == sorted(degs) and max(degs) == p


@pytest.mark.parametrize("family", [basis.LEGENDRE, basis.HERMITE])
def test_g_matrices_match_tensor_quadrature(family):
    M, p = 2, 3
    al = basis.multi_indices(M, p)
    G = basis.g_matrices(al, family)
    xi, w, polys = _ortho_1d(family, p + 1)
    # full tensor-product quadrature in M = 2 dimensions (no separability assumed)
    P = len(al)
    for k in range(M + 1):
        ref = np.zeros((P, P))
        for (q1, x1), (q2, x2) in product(enumerate(xi), enumerate(xi)):
            wt = w[q1] * w[q2]
            xs = (x1, x2)
            psi = np.array([polys[a[0]](x1) * polys[a[1]](x2) for a in al])
            f = 1.0 if k == 0 else xs[k - 1]
            ref += wt * f * np.outer(psi, psi)
        assert np.allclose(G[k], ref, atol=1e-12), k


@pytest.mark.parametrize("family", [basis.LEGENDRE, basis.HERMITE])
def test_g_matrices_separable_quadrature_M4(family):
    M, p = 4, 3
    al = basis.multi_indices(M, p)
    G = basis.g_matrices(al, family)
    xi, w, polys = _ortho_1d(family, p + 1)
    V = np.array([[polys[n](x) for x in xi] for n in range(p + 2)])   # (deg, quad)
    mass = (V * w) @ V.T
    first = (V * w * xi) @ V.T
    for k in range(1, M + 1):
        for i, a in enumerate(al):
            for j, b in enumerate(al):
                v = 1.0
                for l in range(M):
                    v *= first[a[l], b[l]] if l == k - 1 else mass[a[l], b[l]]
                assert abs(G[k][i, j] - v) < 1e-12


def test_structure_no_coupling_within_degree_level():
    al = basis.multi_indices(4, 4)
    G = basis.g_matrices(al, basis.LEGENDRE)
    deg = np.array([sum(a) for a in al])
    for k in range(1, 5):
        assert np.all(np.diag(G[k]) == 0.0)
        nz = np.argwhere(G[k] != 0.0)
        assert np.all(np.abs(deg[nz[:, 0]] - deg[nz[:, 1]]) == 1)
        assert np.all(np.abs(G[k] - G[k].T) == 0.0)
        # each row has at most 2 entries in G_k (i - e_k and i + e_k)
        assert np.max(np.count_nonzero(G[k], axis=1)) <= 2


def test_table1_block_counts():
    t = GOLD["table1"]
    m, p = t["m"], t["p"]
    Nx = (t["h_inv"] - 1) ** 2
    nnz5 = 5 * Nx - 4 * (t["h_inv"] - 1)          # 5-point pattern of the paper's P1 K_k
    al = basis.multi_indices(m, p)
    P, Phat = len(al), basis.n_basis(m, p - 1)
    G = basis.g_matrices(al, basis.LEGENDRE)
    pattern = sum((Gk != 0).astype(int) for Gk in G[1:]) > 0
    blocks_A = P + int(pattern.sum())
    blocks_W = int(pattern[Phat:, :Phat].sum())
    blocks_Ahat = Phat + int(pattern[:Phat, :Phat].sum())
    assert P * Nx == t["size_A"] == t["size_BD"]
    assert Phat * Nx == t["size_Ahat"] == t["cols_W"]
    assert (P - Phat) * Nx == t["size_D"] == t["rows_W"]
    assert (P - Phat) * nnz5 == t["nnz_D"]
    assert P * nnz5 == t["nnz_BD"]
    assert (blocks_A, blocks_W, blocks_Ahat) == (1218, 336, 420)
    # the paper's nnz counts sit just below block count x pattern (a few exact zeros of K_k dropped)
    for blocks, nnz in ((blocks_A, t["nnz_A"]), (blocks_W, t["nnz_W"]), (blocks_Ahat, t["nnz_Ahat"])):
        assert 0 <= blocks * nnz5 - nnz <= 1e-4 * nnz
    assert t["nnz_Ahat"] + 2 * t["nnz_W"] + t["nnz_D"] == t["nnz_A"]
