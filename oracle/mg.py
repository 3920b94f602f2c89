"""Geometric multigrid V-cycle on the mean operator K_0 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.1: each diagonal block K_0 of B_D is inverted approximately by
multigrid; Sec. 4.2: the diagonal blocks of B_T are solved inexactly by the
standard V-cycle; Sec. 6 uses one V-cycle per diagonal block.  The smoother
here is damped Jacobi (omega = 8/9 by default) with nu1 pre- and nu2
post-smoothing steps; the paper's own runs use point Gauss-Seidel V(2,2).

Hierarchy: vertex grids n_0 = n, n_{l+1} = (n_l + 1)/2, down to n = 3 (one
interior node), which is solved exactly.  Prolongation P_l is bilinear
interpolation of coarse-vertex values, restriction is P_l^T, and coarse
operators are Galerkin products A_{l+1} = P_l^T A_l P_l.  All matrices are
assembled (scipy.sparse), so every step can be read off directly.

Pins: Galerkin coarse operator of the constant-coefficient Q1 stencil equals
the Q1 stencil on the coarse grid; the V-cycle with equal pre/post smoothing
is a symmetric operator; the high-frequency Jacobi smoothing factor of the
Q1 stencil at omega = 8/9 is 1/3; the two-grid convergence factor equals the
local Fourier analysis of the same cycle (1/9 for V(1,1) at omega = 8/9)
for several smoother weights and sweep counts.
"""
import numpy as np
import scipy.sparse as sp


def grid_sizes(n, coarsest=3):
    sizes = [n]
    while sizes[-1] > coarsest:
        assert (sizes[-1] - 1) % 2 == 0, "n must be 2^L + 1"
        sizes.append((sizes[-1] + 1) // 2)
    return sizes


def prolongation(nc):
    """Bilinear interpolation from the interior of an nc-grid to the interior of a (2nc-1)-grid."""
    nf = 2 * nc - 1
    mf, mc = nf - 2, nc - 2
    rows, cols, vals = [], [], []
    for vy in range(1, nf - 1):
        for vx in range(1, nf - 1):
            r = (vx - 1) + (vy - 1) * mf
            xs = [(vx // 2, 1.0)] if vx % 2 == 0 else [((vx - 1) // 2, 0.5), ((vx + 1) // 2, 0.5)]
            ys = [(vy // 2, 1.0)] if vy % 2 == 0 else [((vy - 1) // 2, 0.5), ((vy + 1) // 2, 0.5)]
            for cxv, wx in xs:
                for cyv, wy in ys:
                    if 1 <= cxv <= nc - 2 and 1 <= cyv <= nc - 2:
                        rows.append(r)
                        cols.append((cxv - 1) + (cyv - 1) * mc)
                        vals.append(wx * wy)
    return sp.csr_matrix((vals, (rows, cols)), shape=(mf * mf, mc * mc))


class Hierarchy:
    """Assembled operators A_l, prolongations P_l and Jacobi diagonals of one V-cycle."""

    def __init__(self, K0, n, nu1=1, nu2=1, omega=8.0 / 9.0, coarsest=3):
        self.sizes = grid_sizes(n, coarsest)
        self.nu1, self.nu2, self.omega = nu1, nu2, omega
        self.A = [sp.csr_matrix(K0)]
        self.P = []
        for l in range(len(self.sizes) - 1):
            Pl = prolongation(self.sizes[l + 1])
            self.P.append(Pl)
            self.A.append((Pl.T @ self.A[l] @ Pl).tocsr())
        self.Dinv = [1.0 / A.diagonal() for A in self.A]
        self.coarse_inv = np.linalg.inv(self.A[-1].toarray())

    def vcycle(self, b, level=0):
        """One V(nu1, nu2) cycle from a zero initial guess; b is (N_l,) or (N_l, nrhs)."""
        A = self.A[level]
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        Dinv = self.Dinv[level] if b.ndim == 1 else self.Dinv[level][:, None]
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = x + self.omega * Dinv * (b - A @ x)
        r = b - A @ x
        bc = self.P[level].T @ r
        xc = self.vcycle(bc, level + 1)
        x = x + self.P[level] @ xc
        for _ in range(self.nu2):
            x = x + self.omega * Dinv * (b - A @ x)
        return x
