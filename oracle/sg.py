"""Stochastic Galerkin system A U = F (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (tensor-product): A = G_0 (x) K_0 + sum_{k=1}^M G_k (x) K_k, G_0 = I by
orthonormality (Sec. 3.2).  Unknowns are ordered PC-major,
U[i*N_x + s] = coefficient of psi_i phi_s, i.e. the block rows of the
Kronecker form (Eq. PCE_u).  The right-hand side is F = e_0 (x) F_0: the
forcing f is deterministic, so only the mean block E[f psi_i] = delta_i0 f
survives.

Solvers here define the exact result U* = A^{-1} F: a sparse direct
factorisation (SuperLU) of the assembled matrix and a plain unpreconditioned
restarted GMRES (Saad-Schultz; cited in Sec. 4.2).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, fem


@dataclass
class SGSystem:
    n: int
    M: int
    p: int
    family: int
    coef: np.ndarray                      # (M+1, Nc)
    alphas: list = field(default_factory=list)
    G: list = field(default_factory=list)
    K: list = field(default_factory=list)

    @property
    def P(self):
        return len(self.alphas)

    @property
    def Nx(self):
        return (self.n - 2) ** 2


def build(n, M, p, family, coef):
    """Basis, stochastic matrices G_k and stiffness matrices K_k of one SG system."""
    coef = np.asarray(coef, dtype=np.float64)
    assert coef.shape == (M + 1, (n - 1) ** 2)
    alphas = basis.multi_indices(M, p)
    G = basis.g_matrices(alphas, family)
    K = fem.stiffness_matrices(n, coef)
    return SGSystem(n, M, p, family, coef, alphas, G, K)


def assemble(sys):
    """Global CSR matrix  sum_k kron(G_k, K_k)  (Eq. tensor-product)."""
    A = sp.kron(sp.csr_matrix(sys.G[0]), sys.K[0], format="csr")
    for k in range(1, sys.M + 1):
        A = A + sp.kron(sp.csr_matrix(sys.G[k]), sys.K[k], format="csr")
    return A.tocsr()


def apply(sys, X):
    """Y = A X without assembling A:  Y_i = sum_k sum_j G_k(i,j) K_k X_j.

    X, Y are flat PC-major vectors of length P*N_x (or (P, N_x) arrays).
    """
    Xm = np.asarray(X, dtype=np.float64).reshape(sys.P, sys.Nx)
    Y = np.zeros_like(Xm)
    for k in range(sys.M + 1):
        KX = (sys.K[k] @ Xm.T).T              # rows: K_k X_j
        Y += sys.G[k] @ KX
    return Y.reshape(-1)


def rhs(sys, f_nodes=None):
    """F = e_0 (x) F_0 with F_0 the (lumped) load vector."""
    F = np.zeros((sys.P, sys.Nx))
    F[0] = fem.load_vector(sys.n, f_nodes)
    return F.reshape(-1)


def solve_direct(A, F):
    """U* = A^{-1} F by sparse LU (library primitive)."""
    return spla.spsolve(A.tocsc(), F)


def gmres_plain(apply_A, b, tol=1e-10, restart=50, maxit=5000):
    """Unpreconditioned restarted GMRES, x0 = 0 (Saad-Schultz, cited in Sec. 4.2).

    Stops when the true relative residual ||b - A x|| / ||b|| <= tol.
    Returns (x, iterations, relres).
    """
    from .krylov import gmres
    return gmres(apply_A, None, b, tol=tol, restart=restart, maxit=maxit)
