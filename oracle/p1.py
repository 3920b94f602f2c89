"""The paper's own discretisation: linear triangles and a point Gauss-Seidel V-cycle (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 6 solves the test problem on D = (-0.5, 0.5)^2 with linear finite elements on a uniform
triangulation of mesh size h and approximates every diagonal block by one geometric multigrid
V(2,2) cycle with point Gauss-Seidel smoothing.  The paper gives no further detail; the readings
used here are:

* every square cell of the uniform grid is cut by its SW-NE diagonal into a lower-right and an
  upper-left right triangle; the KL coefficient of a triangle is taken at its centroid, so each
  K_k is the P1 stiffness matrix of a piecewise-constant coefficient.  On these right triangles
  the coupling across a diagonal vanishes (the opposite angles are right angles), so every K_k
  has the 5-point pattern, which is what the nonzero counts of the paper's Table 1 imply;
* the load vector is lumped, F_i = h^2 f(x_i) (six triangles of area h^2/2 share a vertex);
* prolongation is linear interpolation on the nested triangulations (a fine vertex on a coarse
  edge, the diagonals included, takes the mean of the edge's two end points), restriction its
  transpose, coarse operators Galerkin products, the coarsest grid (one interior vertex) solved
  exactly;
* pre-smoothing is forward lexicographic Gauss-Seidel and post-smoothing backward Gauss-Seidel,
  which makes the cycle a symmetric operator (PCG with B_D needs a symmetric preconditioner);
  ``order="rb"`` takes the red-black order instead (the multicolour reading of a parallel point
  Gauss-Seidel): the unknowns of colour (x + y) mod 2 = 0 first, then colour 1, each colour in
  lexicographic order, and the backward sweep in the reverse of that order.

For B_T the module also has the reading that the paper's counts support best: the 2 x 2 split of
Eq. hierarchical_structure with the lower-degree block A_hat approximated by one V(2,2) of a point
Gauss-Seidel multigrid on the coupled system A_hat itself (``CoupledGSHierarchy``,
``block_tri_2x2_inv``), and the degree-p blocks by K_0 cycles.

Pins: the element matrices against the gradients of the barycentric basis; the assembled K_0
against the 5-point Laplacian and the nonzero count of Table 1; the symmetry of the cycle and its
two-grid factor against a local Fourier analysis of lexicographic Gauss-Seidel; the iteration
counts the paper prints in Tables 2 and 3 for its test problem.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis, kl, mg
from .sg import SGSystem


def triangle_element_matrices():
    """P1 stiffness element matrices (coefficient 1, any h) of the two right triangles of a cell:
    lower-right (SW, SE, NE), right angle at SE, and upper-left (SW, NE, NW), right angle at NW."""
    lower = np.array([[0.5, -0.5, 0.0], [-0.5, 1.0, -0.5], [0.0, -0.5, 0.5]])
    upper = np.array([[0.5, 0.0, -0.5], [0.0, 0.5, -0.5], [-0.5, -0.5, 1.0]])
    return lower, upper


def triangle_coefficients(n, M, sigma, corr_len=1.0):
    """Coefficients c_k(T), k = 0..M, at the centroids of the 2 (n-1)^2 triangles: triangle 2e is
    the lower-right and 2e + 1 the upper-left triangle of cell e = cx + cy (n-1); row 0 is the
    mean 1, row k >= 1 is sigma sqrt(lambda_k) b_k(centroid) (same separable modes as ``kl``)."""
    nc1 = n - 1
    h = 1.0 / nc1
    lam1, om1, par1 = kl.kl_1d(M + 1, corr_len)
    modes = kl.kl_2d_modes(M, corr_len)
    base = np.arange(nc1) * h - 0.5
    coef = np.zeros((M + 1, 2 * nc1 * nc1))
    coef[0] = 1.0
    for k, (lam, i, j) in enumerate(modes, start=1):
        for t, (ox, oy) in enumerate(((2.0 / 3.0, 1.0 / 3.0), (1.0 / 3.0, 2.0 / 3.0))):
            bx = kl.eval_1d(om1[i], par1[i], base + ox * h)
            by = kl.eval_1d(om1[j], par1[j], base + oy * h)
            coef[k, t::2] = sigma * np.sqrt(lam) * np.outer(by, bx).reshape(-1)
    return coef


def assemble_p1(n, tri_coef):
    """Interior-node P1 stiffness matrix for the per-triangle coefficients tri_coef (2 (n-1)^2)."""
    m = n - 2
    lower, upper = triangle_element_matrices()
    rows, cols, vals = [], [], []
    nc1 = n - 1
    for cy in range(nc1):
        for cx in range(nc1):
            e = cx + cy * nc1
            sw, se, ne, nw = (cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)
            for Ke, verts, a in ((lower, (sw, se, ne), tri_coef[2 * e]), (upper, (sw, ne, nw), tri_coef[2 * e + 1])):
                idx = [(vx - 1) + (vy - 1) * m if 1 <= vx <= n - 2 and 1 <= vy <= n - 2 else -1 for vx, vy in verts]
                for r in range(3):
                    for c in range(3):
                        if idx[r] >= 0 and idx[c] >= 0 and Ke[r, c] != 0.0:
                            rows.append(idx[r]), cols.append(idx[c]), vals.append(a * Ke[r, c])
    K = sp.csr_matrix((vals, (rows, cols)), shape=(m * m, m * m))
    K.sum_duplicates()
    K.eliminate_zeros()
    return K


def build(n, M, p, family, sigma, corr_len=1.0):
    """SG system of the paper's discretisation (the same chaos space and G_k as ``sg.build``)."""
    tc = triangle_coefficients(n, M, sigma, corr_len)
    alphas = basis.multi_indices(M, p)
    G = basis.g_matrices(alphas, family)
    K = [assemble_p1(n, tc[k]) for k in range(M + 1)]
    return SGSystem(n, M, p, family, tc, alphas, G, K)


def rhs(sys, f=None):
    """F = e_0 (x) F_0 with the lumped load F_0,i = h^2 f(x_i); f defaults to the paper's
    2 (0.5 - x^2 - y^2) on (-0.5, 0.5)^2."""
    n = sys.n
    h = 1.0 / (n - 1)
    xs = np.arange(1, n - 1) * h - 0.5
    X, Y = np.meshgrid(xs, xs)
    fv = 2.0 * (0.5 - X ** 2 - Y ** 2) if f is None else f(X, Y)
    F = np.zeros((sys.P, sys.Nx))
    F[0] = h * h * fv.reshape(-1)
    return F.reshape(-1)


def prolongation(nc):
    """Linear interpolation from the interior of an nc-grid to the interior of the (2 nc - 1)-grid
    of the nested triangulation (SW-NE diagonals)."""
    nf = 2 * nc - 1
    mf, mc = nf - 2, nc - 2
    rows, cols, vals = [], [], []
    for vy in range(1, nf - 1):
        for vx in range(1, nf - 1):
            r = (vx - 1) + (vy - 1) * mf
            if vx % 2 == 0 and vy % 2 == 0:
                src = [(vx // 2, vy // 2, 1.0)]
            elif vy % 2 == 0:
                src = [((vx - 1) // 2, vy // 2, 0.5), ((vx + 1) // 2, vy // 2, 0.5)]
            elif vx % 2 == 0:
                src = [(vx // 2, (vy - 1) // 2, 0.5), (vx // 2, (vy + 1) // 2, 0.5)]
            else:                                           # centre of a coarse cell: on its SW-NE diagonal
                src = [((vx - 1) // 2, (vy - 1) // 2, 0.5), ((vx + 1) // 2, (vy + 1) // 2, 0.5)]
            for cxv, cyv, w in src:
                if 1 <= cxv <= nc - 2 and 1 <= cyv <= nc - 2:
                    rows.append(r), cols.append((cxv - 1) + (cyv - 1) * mc), vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(mf * mf, mc * mc))


def red_black_order(n):
    """Permutation of the (n-2)^2 interior vertices of an n-grid (index (x-1) + (y-1)(n-2)): the
    vertices with (x + y) even in lexicographic order, then those with (x + y) odd."""
    m = n - 2
    vx, vy = np.meshgrid(np.arange(1, n - 1), np.arange(1, n - 1))
    colour = ((vx + vy) % 2).reshape(-1)
    return np.concatenate([np.nonzero(colour == 0)[0], np.nonzero(colour == 1)[0]])


class GSHierarchy:
    """V(nu1, nu2) cycle with forward Gauss-Seidel pre- and backward Gauss-Seidel post-smoothing, in
    lexicographic (``order="lex"``) or red-black (``order="rb"``) order of the unknowns."""

    def __init__(self, K0, n, nu1=2, nu2=2, coarsest=3, order="lex"):
        self.sizes = mg.grid_sizes(n, coarsest)
        self.nu1, self.nu2 = nu1, nu2
        self.A = [sp.csr_matrix(K0)]
        self.P = []
        for l in range(len(self.sizes) - 1):
            Pl = prolongation(self.sizes[l + 1])
            self.P.append(Pl)
            self.A.append((Pl.T @ self.A[l] @ Pl).tocsr())
        # the sweep order of each level as a permutation (identity for the lexicographic order)
        self.perm = [np.arange(A.shape[0]) if order == "lex" else red_black_order(nl)
                     for A, nl in zip(self.A, self.sizes)]
        # D + L and D + U of the permuted matrix as sparse LU factors with the natural order (plain
        # triangular solves): one forward / backward Gauss-Seidel sweep in that order
        Ap = [A[q][:, q] for A, q in zip(self.A[:-1], self.perm)]
        self.low = [spla.splu(sp.tril(A).tocsc(), permc_spec="NATURAL", diag_pivot_thresh=0.0) for A in Ap]
        self.up = [spla.splu(sp.triu(A).tocsc(), permc_spec="NATURAL", diag_pivot_thresh=0.0) for A in Ap]
        self.coarse_inv = np.linalg.inv(self.A[-1].toarray())

    def _sweep(self, factor, level, x, b):
        q = self.perm[level]
        d = np.zeros_like(x)
        d[q] = factor.solve((b - self.A[level] @ x)[q])
        return x + d

    def vcycle(self, b, level=0):
        """One cycle from a zero initial guess; b is (N_l,) or (N_l, nrhs)."""
        A = self.A[level]
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = self._sweep(self.low[level], level, x, b)
        bc = self.P[level].T @ (b - A @ x)
        x = x + self.P[level] @ self.vcycle(bc, level + 1)
        for _ in range(self.nu2):
            x = self._sweep(self.up[level], level, x, b)
        return x


class CoupledGSHierarchy:
    """V(nu1, nu2) point Gauss-Seidel multigrid on the coupled SG matrix of the PC rows ``rows``,
    sum_k G_k[rows, rows] (x) K_k (the lower-degree block A_hat of Eq. hierarchical_structure): the
    same spatial hierarchy for every PC block (prolongation I (x) P_h, Galerkin coarse operators),
    forward Gauss-Seidel over all unknowns in PC-major order before the coarse correction and backward
    after it, the coarsest grid solved exactly."""

    def __init__(self, sys, rows, nu1=2, nu2=2, coarsest=3):
        rows = np.asarray(rows)
        sizes = mg.grid_sizes(sys.n, coarsest)
        A0 = sum(sp.kron(sp.csr_matrix(sys.G[k][np.ix_(rows, rows)]), sys.K[k]) for k in range(sys.M + 1))
        self.A = [sp.csr_matrix(A0)]
        self.P = []
        for l in range(len(sizes) - 1):
            Pl = sp.kron(sp.identity(len(rows)), prolongation(sizes[l + 1])).tocsr()
            self.P.append(Pl)
            self.A.append((Pl.T @ self.A[l] @ Pl).tocsr())
        self.low = [spla.splu(sp.tril(A).tocsc(), permc_spec="NATURAL", diag_pivot_thresh=0.0) for A in self.A[:-1]]
        self.up = [spla.splu(sp.triu(A).tocsc(), permc_spec="NATURAL", diag_pivot_thresh=0.0) for A in self.A[:-1]]
        self.coarse_inv = np.linalg.inv(self.A[-1].toarray())
        self.nu1, self.nu2 = nu1, nu2

    def vcycle(self, b, level=0):
        A = self.A[level]
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = x + self.low[level].solve(b - A @ x)
        x = x + self.P[level] @ self.vcycle(self.P[level].T @ (b - A @ x), level + 1)
        for _ in range(self.nu2):
            x = x + self.up[level].solve(b - A @ x)
        return x


def block_tri_2x2_inv(sys, ahat_cycle, solver, R):
    """Z = B_T^{-1} R for the 2 x 2 split of Sec. 4.2, B_T = [A_hat 0; W D], with A_hat^{-1} replaced
    by one cycle of ``ahat_cycle`` (a CoupledGSHierarchy on the degrees < p) and D^{-1} = I (x) K_0^{-1}
    by ``solver`` block by block:  Z_low = cycle(R_low),  Z_p = D^{-1} (R_p - W Z_low)."""
    off = basis.degree_levels(sys.alphas)
    P, Nx = sys.P, sys.Nx
    nlow = off[-2]
    Rm = np.asarray(R, dtype=np.float64).reshape(P, Nx)
    Zlow = ahat_cycle.vcycle(Rm[:nlow].reshape(-1)).reshape(nlow, Nx)
    T = Rm[nlow:].copy()
    hi, low = np.arange(nlow, P), np.arange(nlow)
    for k in range(1, sys.M + 1):
        Gk = sys.G[k][np.ix_(hi, low)]
        if np.any(Gk):
            T -= Gk @ (sys.K[k] @ Zlow.T).T
    Zp = solver(T.T).T
    return np.vstack([Zlow, Zp]).reshape(-1)


class MulticolourCoupledGSHierarchy(CoupledGSHierarchy):
    """The coupled cycle with the parallel (multicolour) Gauss-Seidel order: an unknown (PC row i,
    node (x, y)) has colour 2 (deg(i) mod 2) + ((x + y) mod 2).  The K_k are 5-point, so a coupling
    between two nodes joins opposite node parities, and G_k (k >= 1) couples only degrees one apart
    (G_0 = I), so no two unknowns of one colour are coupled and a colour is updated at once.
    Pre-smoothing visits the colours 0, 1, 2, 3 and post-smoothing 3, 2, 1, 0 (a symmetric cycle)."""

    def __init__(self, sys, rows, nu1=2, nu2=2, coarsest=3):
        super().__init__(sys, rows, nu1, nu2, coarsest)
        rows = np.asarray(rows)
        degs = np.array([sum(sys.alphas[i]) for i in rows])
        sizes = mg.grid_sizes(sys.n, coarsest)
        self.colours, self.dinv = [], []
        for l, nl in enumerate(sizes[:-1]):
            m = nl - 2
            vx, vy = np.meshgrid(np.arange(m), np.arange(m))
            parity = ((vx + vy) % 2).reshape(-1)
            colour = np.repeat(degs % 2, m * m) * 2 + np.tile(parity, len(rows))
            self.colours.append([np.nonzero(colour == c)[0] for c in range(4)])
            self.dinv.append(1.0 / self.A[l].diagonal())

    def _sweep(self, level, x, b, order):
        A = self.A[level]
        for c in order:
            idx = self.colours[level][c]
            d = self.dinv[level][idx] if b.ndim == 1 else self.dinv[level][idx][:, None]
            x[idx] += d * (b[idx] - A[idx] @ x)
        return x

    def vcycle(self, b, level=0):
        A = self.A[level]
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            x = self._sweep(level, x, b, (0, 1, 2, 3))
        x = x + self.P[level] @ self.vcycle(self.P[level].T @ (b - A @ x), level + 1)
        for _ in range(self.nu2):
            x = self._sweep(level, x, b, (3, 2, 1, 0))
        return x
