"""Q1 finite-element stiffness matrices on the unit square (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (def-stiffness): K_0(r,s) = int abar grad phi_s . grad phi_r,
K_k(r,s) = sqrt(lambda_k) int b_k grad phi_s . grad phi_r.  With the KL
coefficient constant on each cell (cell-centre value, times sigma), every K_k
is  sum_e c_k(e) K_ref^(e),  K_ref the bilinear element matrix of the
Laplacian on one square cell (scale invariant in 2-D).

Grid: n vertices per side on [0,1]^2, h = 1/(n-1), homogeneous Dirichlet
boundary (Eq. model-problem).  Interior node s = (vx-1) + (vy-1)(n-2) for
vertex (vx, vy), 1 <= vx, vy <= n-2; cell e = cx + cy (n-1) with corners
SW (cx,cy), SE (cx+1,cy), NE (cx+1,cy+1), NW (cx,cy+1) in that
(counter-clockwise) local order.

Pins: closed-form eigenvalues of K_0 for abar = 1, symmetry, constant
nullspace of K_ref, Galerkin coarse operator of constant Q1 is Q1.
"""
import numpy as np
import scipy.sparse as sp


def q1_reference_stiffness():
    """K_ref(r,s) = int_[0,1]^2 grad phi_r . grad phi_s by 2x2 Gauss quadrature (exact)."""
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0) * 0.5 + 0.5
    w = np.array([0.5, 0.5])
    # bilinear basis in (x, y) on the unit cell, local order SW, SE, NE, NW
    def grads(x, y):
        return np.array([
            [-(1 - y), -(1 - x)],
            [(1 - y), -x],
            [y, x],
            [-y, (1 - x)],
        ])
    K = np.zeros((4, 4))
    for i in range(2):
        for j in range(2):
            G = grads(g[i], g[j])
            K += w[i] * w[j] * G @ G.T
    return K


def cell_corner_nodes(n):
    """(Nc, 4) array of interior-node indices of each cell's corners; -1 on the boundary."""
    nc1 = n - 1
    m = n - 2
    cx, cy = np.meshgrid(np.arange(nc1), np.arange(nc1))
    cx, cy = cx.reshape(-1), cy.reshape(-1)

    def node(vx, vy):
        inside = (vx >= 1) & (vx <= n - 2) & (vy >= 1) & (vy <= n - 2)
        return np.where(inside, (vx - 1) + (vy - 1) * m, -1)

    return np.stack([node(cx, cy), node(cx + 1, cy), node(cx + 1, cy + 1), node(cx, cy + 1)], axis=1)


def assemble_stiffness(n, cell_coef):
    """K = sum_e cell_coef[e] K_ref^(e) on the interior nodes, as CSR (FP64)."""
    Kref = q1_reference_stiffness()
    corners = cell_corner_nodes(n)
    Nx = (n - 2) ** 2
    rows, cols, vals = [], [], []
    cc = np.asarray(cell_coef, dtype=np.float64).reshape(-1)
    for a in range(4):
        for b in range(4):
            ra, cb = corners[:, a], corners[:, b]
            keep = (ra >= 0) & (cb >= 0)
            rows.append(ra[keep]), cols.append(cb[keep]), vals.append(cc[keep] * Kref[a, b])
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(Nx, Nx))
    return K.tocsr()


def stiffness_matrices(n, coef):
    """[K_0, ..., K_M] from the (M+1, Nc) per-cell coefficient array."""
    return [assemble_stiffness(n, coef[k]) for k in range(coef.shape[0])]


def node_mass_weights(n):
    """m_s = int phi_s dx = h^2 for every interior Q1 hat function."""
    h = 1.0 / (n - 1)
    return np.full((n - 2) ** 2, h * h)


def load_vector(n, f_nodes=None):
    """F_0(s) = int f phi_s, with f given at interior nodes and lumped: h^2 f_s.

    For f = 1 this is exact (int phi_s = h^2).
    """
    m = node_mass_weights(n)
    if f_nodes is None:
        return m.copy()
    return m * np.asarray(f_nodes, dtype=np.float64).reshape(-1)


def laplacian_q1_eigenvalues(n):
    """Closed-form spectrum of K_0 (abar = 1): (2/3)(4 - c_j - c_k - 2 c_j c_k), c_j = cos(j pi h)."""
    h = 1.0 / (n - 1)
    j = np.arange(1, n - 1)
    c = np.cos(j * np.pi * h)
    cj, ck = np.meshgrid(c, c)
    return np.sort(((2.0 / 3.0) * (4 - cj - ck - 2 * cj * ck)).reshape(-1))
