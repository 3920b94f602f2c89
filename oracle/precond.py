"""Block preconditioners B_D and B_T of the SG matrix (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.1: B_D = G_0 (x) K_0 (mean-based, block diagonal); each diagonal
block is inverted approximately by a multigrid V-cycle.
Sec. 4.2: B_T = the lower block-triangular part of A, i.e. one block
Gauss-Seidel step from a zero initial guess; its diagonal blocks are solved
inexactly by the standard V-cycle.

Reading taken (the paper states B_T for the 2x2 split of Eq.
(hierarchical_structure) and calls it the lower block-triangular part of A):
B_T is the full lower block-triangular part of A in the degree-graded PC
order, which is the 2x2 split applied recursively down to degree 0.  Its
inverse is applied by plain block forward substitution over the PC index:
  T_i = R_i - sum_{j<i} A_ij Z_j,   Z_i ~= A_ii^{-1} T_i,
with A_ij = sum_k G_k(i,j) K_k and A_ii = K_0 (G_k(i,i) = 0 for symmetric
densities).  B_T^T is applied by backward substitution with A_ji^T.

Diagonal solve options: a V-cycle (``Hierarchy.vcycle``) or the exact
sparse LU of K_0 (used for the spectral checks of Sec. 5).
"""
import numpy as np

from . import basis
import scipy.sparse.linalg as spla


class DiagSolver:
    def __init__(self, K0, hierarchy=None):
        self.hier = hierarchy
        self.lu = None if hierarchy is not None else spla.splu(K0.tocsc())

    def __call__(self, b):
        if self.hier is not None:
            return self.hier.vcycle(b)
        return self.lu.solve(b)


def block_diag_inv(sys, solver, R):
    """Z = B_D^{-1} R: every PC block solved with the mean operator K_0."""
    Rm = np.asarray(R, dtype=np.float64).reshape(sys.P, sys.Nx)
    Z = solver(Rm.T).T
    return np.ascontiguousarray(Z).reshape(-1)


def _offdiag_block_apply(sys, i, j, Zj, transpose=False):
    """A_ij Zj (or A_ji^T Zj) for i != j, skipping zero Kronecker factors."""
    out = None
    for k in range(1, sys.M + 1):
        g = sys.G[k][j, i] if transpose else sys.G[k][i, j]
        if g != 0.0:
            Kk = sys.K[k].T if transpose else sys.K[k]
            t = g * (Kk @ Zj)
            out = t if out is None else out + t
    return out


def block_tri_inv(sys, solver, R, transpose=False):
    """Z = B_T^{-1} R (forward substitution) or B_T^{-T} R (backward substitution)."""
    Rm = np.asarray(R, dtype=np.float64).reshape(sys.P, sys.Nx)
    Z = np.zeros_like(Rm)
    order = range(sys.P - 1, -1, -1) if transpose else range(sys.P)
    for i in order:
        T = Rm[i].copy()
        others = range(i + 1, sys.P) if transpose else range(i)
        for j in others:
            c = _offdiag_block_apply(sys, i, j, Z[j], transpose)
            if c is not None:
                T -= c
        Z[i] = solver(T)
    return Z.reshape(-1)


def block_sym_inv(sys, solver, R):
    """Z = B_S^{-1} R for the symmetric block Gauss-Seidel preconditioner of Sec. 4.2,
    B_S = B_T diag(A)^{-1} B_T^T with diag(A) = I (x) K_0:  a lower sweep, the exact
    diagonal blocks K_0, then an upper sweep."""
    Z1 = block_tri_inv(sys, solver, R).reshape(sys.P, sys.Nx)
    Z2 = (sys.K[0] @ Z1.T).T
    return block_tri_inv(sys, solver, np.ascontiguousarray(Z2).reshape(-1), transpose=True)


def block_sym_recursive_inv(sys, solver, R):
    """Z = B_S^{-1} R with the 2 x 2 form of Sec. 4.2 applied recursively over the degree levels:
    B_S = [A_hat 0; W D] diag(A_hat, D)^{-1} [A_hat W^T; 0 D] gives
      y_low = A_hat^{-1} R_low,  y_p = D^{-1} (R_p - W y_low),  z_low = A_hat^{-1} (R_low - W^T y_p),
    and A_hat^{-1} is replaced by the same preconditioner one degree lower, down to degree 0, whose
    block is K_0 (D = I (x) K_0 on every degree level).  Each call of the solver takes the blocks of one
    degree level at once."""
    off = basis.degree_levels(sys.alphas)
    P, Nx = sys.P, sys.Nx
    Rm = np.asarray(R, dtype=np.float64).reshape(P, Nx)

    def couple(Y, rows, cols):
        """sum_k G_k[rows, cols] (x) K_k applied to the blocks Y of the columns."""
        out = np.zeros((len(rows), Nx))
        for k in range(1, sys.M + 1):
            Gk = sys.G[k][np.ix_(rows, cols)]
            if np.any(Gk):
                out += Gk @ (sys.K[k] @ Y.T).T
        return out

    def rec(q, Rq):                                       # Rq: blocks of degrees 0..q, in order
        hi = np.arange(off[q], off[q + 1])
        if q == 0:
            return solver(Rq.T).T
        low = np.arange(0, off[q])
        y_low = rec(q - 1, Rq[:off[q]])
        y_hi = solver((Rq[off[q]:] - couple(y_low, hi, low)).T).T
        z_low = rec(q - 1, Rq[:off[q]] - couple(y_hi, low, hi))
        return np.vstack([z_low, y_hi])

    return rec(len(off) - 2, Rm).reshape(-1)


def block_tri_exact_inv(sys, solver, R, inner_tol=1e-13, inner_restart=40):
    """Z = B_T^{-1} R for the 2 x 2 split of Theorem 1 with the lower-degree block A_hat solved to
    ``inner_tol`` (GMRES on A_hat, right-preconditioned by the flat B_T of A_hat) and the degree-p
    blocks by ``solver``:  Z_low = A_hat^{-1} R_low,  Z_p = D^{-1} (R_p - W Z_low).  An analysis tool
    (Sec. 4.2, Theorem 1): with an exact ``solver`` its preconditioned spectrum is the theorem's."""
    from . import krylov
    from .sg import SGSystem, apply as sg_apply
    off = basis.degree_levels(sys.alphas)
    P, Nx = sys.P, sys.Nx
    nlow = off[-2]
    Rm = np.asarray(R, dtype=np.float64).reshape(P, Nx)
    low = SGSystem(sys.n, sys.M, sys.p - 1, sys.family, sys.coef, list(sys.alphas[:nlow]),
                   [G[:nlow, :nlow] for G in sys.G], sys.K)
    Zlow, _, rr = krylov.gmres(lambda v: sg_apply(low, v), lambda r: block_tri_inv(low, solver, r),
                               Rm[:nlow].reshape(-1), tol=inner_tol, restart=inner_restart, maxit=2000)
    Zlow = Zlow.reshape(nlow, Nx)
    T = Rm[nlow:].copy()
    hi, lo = np.arange(nlow, P), np.arange(nlow)
    for k in range(1, sys.M + 1):
        Gk = sys.G[k][np.ix_(hi, lo)]
        if np.any(Gk):
            T -= Gk @ (sys.K[k] @ Zlow.T).T
    Zp = solver(T.T).T
    return np.vstack([Zlow, Zp]).reshape(-1)
