"""Pins of the oracle's version of the paper's own discretisation (Sec. 6: linear triangles,
point Gauss-Seidel V(2,2)) and of the iteration counts the paper prints for it (Tables 2 and 3,
`tests/golden/paper_examples.json`)."""
import json
import os

import numpy as np
import pytest

from oracle import basis, krylov, p1, precond, sg

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def test_element_matrices_from_barycentric_gradients():
    """area x grad(lambda_i) . grad(lambda_j) for the two right triangles of a unit cell, with the
    gradients of the barycentric coordinates from the rotated opposite edges (any h gives the same)."""
    def element(verts):
        v = np.array(verts, dtype=float)
        d1, d2 = v[1] - v[0], v[2] - v[0]
        area = 0.5 * abs(d1[0] * d2[1] - d1[1] * d2[0])
        grads = []
        for i in range(3):
            a, b = v[(i + 1) % 3], v[(i + 2) % 3]
            e = b - a
            g = np.array([e[1], -e[0]]) / (2 * area)
            if np.dot(g, v[i] - a) < 0:                    # point towards vertex i
                g = -g
            grads.append(g)
        G = np.array(grads)
        return area * G @ G.T
    lower, upper = p1.triangle_element_matrices()
    assert np.allclose(element([(0, 0), (1, 0), (1, 1)]), lower, atol=1e-15)
    assert np.allclose(element([(0, 0), (1, 1), (0, 1)]), upper, atol=1e-15)


def test_k0_is_the_five_point_laplacian_and_the_kl_blocks_keep_its_pattern():
    """Constant coefficient: the 5-point stencil (4, -1); the KL blocks have the same pattern, so one
    block has (n-2)^2 + 4 (n-2)(n-3) nonzeros: 19,593 at h = 1/64, nnz(B_D)/P of Table 1."""
    n = 65
    s = p1.build(n, 6, 1, basis.LEGENDRE, 0.3)
    m = n - 2
    K0 = s.K[0].tocsr()
    assert np.allclose(K0.diagonal(), 4.0)
    assert K0.nnz == m * m + 4 * m * (m - 1)
    t1 = GOLDEN["table1"]
    assert K0.nnz * 210 == t1["nnz_BD"]
    for K in s.K[1:]:
        K = K.tocsr()
        assert K.nnz <= K0.nnz
        pattern = set(zip(*K0.nonzero()))
        assert set(zip(*K.nonzero())) <= pattern                 # inside the 5-point pattern
    vals = K0.tocoo()
    offd = vals.data[vals.row != vals.col]
    assert np.allclose(offd, -1.0)


def test_gauss_seidel_cycle_is_symmetric_and_contracting():
    """Forward Gauss-Seidel before and backward after the coarse correction: the V(2,2) cycle is a
    symmetric operator (as PCG with B_D needs) and contracts the K_0 error (factor 0.14 here; a
    sanity band, the cycle has no closed-form factor)."""
    n = 17
    s = p1.build(n, 1, 1, basis.LEGENDRE, 0.0)
    H = p1.GSHierarchy(s.K[0], n)
    N = s.K[0].shape[0]
    B = H.vcycle(np.eye(N))
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    E = np.eye(N) - B @ s.K[0].toarray()
    assert max(abs(np.linalg.eigvals(E))) < 0.2


def _counts(n, M, p, sigma, methods):
    s = p1.build(n, M, p, basis.LEGENDRE, sigma)
    F = p1.rhs(s)
    solver = precond.DiagSolver(s.K[0], p1.GSHierarchy(s.K[0], n))
    Ax = lambda v: sg.apply(s, v)
    bt = lambda r: precond.block_tri_inv(s, solver, r)
    run = {
        "Block-GS": lambda: krylov.block_gauss_seidel(Ax, bt, F, tol=1e-10, maxit=400),
        "BD-PCG": lambda: krylov.pcg(Ax, lambda r: precond.block_diag_inv(s, solver, r), F, tol=1e-10, maxit=400),
        "BT-GPCG": lambda: krylov.gpcg1(Ax, bt, F, tol=1e-10, maxit=400),
        "BT-GMRes": lambda: krylov.gmres(Ax, bt, F, tol=1e-10, restart=10, maxit=400),
        "BS-PCG": lambda: krylov.pcg(Ax, lambda r: precond.block_sym_recursive_inv(s, solver, r), F, tol=1e-10,
                                     maxit=400),
    }
    out = {}
    for name in methods:
        x, its, rr = run[name]()
        assert rr <= 1e-10, name
        out[name] = its
    return out


def test_table2_uniform_iterations_with_the_papers_discretisation():
    """Table 2: at sigma = 0.1 the counts do not depend on h, p or m (h = 1/32 and 1/64, p = 2 and 3,
    m = 4 and 6), and they are the paper's to within one iteration (BD-PCG 13, BT-GPCG 9, BS-PCG 9,
    BT-GMRes 8), also at h = 1/128."""
    names = ["BD-PCG", "BT-GPCG", "BS-PCG", "BT-GMRes"]
    runs = [_counts(n, M, p, 0.1, names) for n, M, p in ((33, 4, 2), (33, 6, 2), (33, 4, 3), (65, 4, 2))]
    for r in runs[1:]:
        assert r == runs[0]
    for name in names:
        assert abs(runs[0][name] - GOLDEN["table2"][name]) <= 1, (name, runs[0][name])
    fine = _counts(129, 4, 2, 0.1, names)                 # h = 1/128
    for name in names:
        assert abs(fine[name] - GOLDEN["table2"][name]) <= 1, (name, fine[name])


@pytest.mark.parametrize("sigma,methods", [
    (0.1, ["Block-GS", "BD-PCG", "BT-GPCG", "BT-GMRes", "BS-PCG"]),
    (0.2, ["BD-PCG", "BS-PCG"]),
])
def test_table3_iterations_with_the_papers_discretisation(sigma, methods):
    """Table 3 (h = 1/64, m = 6, p = 4): the oracle with the paper's discretisation needs the paper's
    iteration counts to within one, for every method at sigma = 0.1 and for the mean-based and the
    symmetric preconditioner at sigma = 0.2 (the block-triangular methods need more than the paper
    at larger sigma; the counts are recorded in the design notes)."""
    t3 = GOLDEN["table3"]
    col = t3["sigma"].index(sigma)
    got = _counts(65, 6, 4, sigma, methods)
    for name in methods:
        assert abs(got[name] - t3[name][col][0]) <= 1, (name, got[name], t3[name][col][0])


def test_recursive_symmetric_preconditioner_is_the_dense_recursion():
    """block_sym_recursive_inv against the 2 x 2 symmetric block Gauss-Seidel inverse written as dense
    matrices, M_q = [[M + M W^T D^-1 W M, -M W^T D^-1], [-D^-1 W M, D^-1]] with M = M_{q-1} and
    M_0 = K_0^-1 (exact K_0 solves, n = 7, M = 2, p = 3); the operator is symmetric positive definite."""
    s = sg.build(7, 2, 3, basis.LEGENDRE, np.vstack([np.ones(36), 0.3 * np.random.default_rng(5).standard_normal((2, 36))]))
    solver = precond.DiagSolver(s.K[0])
    A = sg.assemble(s).toarray()
    Nx = s.Nx
    off = basis.degree_levels(s.alphas)
    K0inv = np.linalg.inv(s.K[0].toarray())
    Mq = np.kron(np.eye(off[1]), K0inv)
    for q in range(1, len(off) - 1):
        lo, hi = slice(0, off[q] * Nx), slice(off[q] * Nx, off[q + 1] * Nx)
        W = A[hi, lo]
        Dinv = np.kron(np.eye(off[q + 1] - off[q]), K0inv)
        top = np.hstack([Mq + Mq @ W.T @ Dinv @ W @ Mq, -Mq @ W.T @ Dinv])
        bot = np.hstack([-Dinv @ W @ Mq, Dinv])
        Mq = np.vstack([top, bot])
    N = A.shape[0]
    Z = np.column_stack([precond.block_sym_recursive_inv(s, solver, e) for e in np.eye(N)])
    assert np.abs(Z - Mq).max() <= 1e-10 * np.abs(Mq).max()
    assert np.abs(Z - Z.T).max() <= 1e-10 * np.abs(Z).max()
    assert np.linalg.eigvalsh(0.5 * (Z + Z.T)).min() > 0


@pytest.mark.parametrize("sigma", [0.1, 0.2, 0.3])
def test_table3_block_triangular_with_a_coupled_cycle_on_the_lower_degrees(sigma):
    """Reading of B_T that the paper's counts support: the 2 x 2 split with A_hat (all degrees < p,
    coupled) approximated by one point Gauss-Seidel V(2,2) of the coupled system and the degree-p
    blocks by K_0 cycles.  GPCG[1], and GMRes(10) run as a left-preconditioned GMRES that stops on the
    preconditioned residual, then need the paper's counts to within one (the flat block substitution
    with right-preconditioned GMRES needs 12 and 11 at sigma = 0.2 against the paper's 10 and 9); block
    Gauss-Seidel too, for sigma <= 0.2 (26 against 24 at sigma = 0.3)."""
    n = 65
    s = p1.build(n, 6, 4, basis.LEGENDRE, sigma)
    F = p1.rhs(s)
    off = basis.degree_levels(s.alphas)
    cyc = p1.CoupledGSHierarchy(s, np.arange(off[-2]))
    solver = precond.DiagSolver(s.K[0], p1.GSHierarchy(s.K[0], n))
    bt = lambda r: p1.block_tri_2x2_inv(s, cyc, solver, r)
    Ax = lambda v: sg.apply(s, v)
    t3 = GOLDEN["table3"]
    col = t3["sigma"].index(sigma)
    got = {"BT-GPCG": krylov.gpcg1(Ax, bt, F, tol=1e-10, maxit=400),
           "BT-GMRes": krylov.gmres_left(Ax, bt, F, tol=1e-10, restart=10, maxit=400)}
    if sigma <= 0.2:
        got["Block-GS"] = krylov.block_gauss_seidel(Ax, bt, F, tol=1e-10, maxit=400)
    for name, (x, its, rr) in got.items():
        assert rr <= (1e-10 if name != "BT-GMRes" else 1e-7)   # left GMRES stops on the preconditioned residual
        assert abs(its - t3[name][col][0]) <= 1, (name, its, t3[name][col][0])


def _lfa_gs_two_grid(nu1, nu2, ngrid=96):
    """Local Fourier analysis of the two-grid cycle with lexicographic Gauss-Seidel on the 5-point
    stencil (symbol 4 - 2 cos t1 - 2 cos t2): forward sweeps amplify a mode by
    (e^{i t1} + e^{i t2}) / (4 - e^{-i t1} - e^{-i t2}), backward sweeps by the conjugate form; linear
    interpolation on the triangulation has the symbol 1 + cos t1 + cos t2 + cos(t1 + t2) per harmonic;
    restriction its transpose, Galerkin coarse symbol.  Largest spectral radius over the low frequencies."""
    A = lambda t1, t2: 4 - 2 * np.cos(t1) - 2 * np.cos(t2)
    Sf = lambda t1, t2: (np.exp(1j * t1) + np.exp(1j * t2)) / (4 - np.exp(-1j * t1) - np.exp(-1j * t2))
    Sb = lambda t1, t2: (np.exp(-1j * t1) + np.exp(-1j * t2)) / (4 - np.exp(1j * t1) - np.exp(1j * t2))
    Pr = lambda t1, t2: 1 + np.cos(t1) + np.cos(t2) + np.cos(t1 + t2)
    ts = (np.arange(ngrid) + 0.5) / ngrid * np.pi - np.pi / 2
    rho = 0.0
    for t1 in ts:
        for t2 in ts:
            H = [(t1, t2), (t1 + np.pi, t2), (t1, t2 + np.pi), (t1 + np.pi, t2 + np.pi)]
            a = np.array([A(*h) for h in H])
            pr = np.array([Pr(*h) for h in H])
            K = np.eye(4) - np.outer(pr, pr * a) / np.sum(pr * a * pr)
            M = np.diag([Sb(*h) ** nu2 for h in H]) @ K @ np.diag([Sf(*h) ** nu1 for h in H])
            rho = max(rho, float(max(abs(np.linalg.eigvals(M)))))
    return rho


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 2), (2, 1)])
def test_gauss_seidel_two_grid_factor_matches_local_fourier_analysis(nu1, nu2):
    """The oracle's P1 two-grid cycle (forward / backward Gauss-Seidel, linear interpolation on the
    triangulation, Galerkin coarse grid) contracts by the LFA factor, within 3 % below it on the
    65 x 65 Dirichlet grid (V(2,2): 0.1327)."""
    n = 65
    s = p1.build(n, 1, 1, basis.LEGENDRE, 0.0)
    H = p1.GSHierarchy(s.K[0], n, nu1=nu1, nu2=nu2, coarsest=(n + 1) // 2)
    K0 = s.K[0]
    e = np.random.default_rng(0).standard_normal(K0.shape[0])
    for _ in range(60):
        e_new = e - H.vcycle(K0 @ e)
        r = np.linalg.norm(e_new) / np.linalg.norm(e)
        e = e_new / np.linalg.norm(e_new)
    rl = _lfa_gs_two_grid(nu1, nu2)
    assert 0.97 * rl <= r <= 1.005 * rl, (r, rl)


def test_four_colour_order_has_no_coupling_inside_a_colour():
    """The colours of MulticolourCoupledGSHierarchy are independent sets of the coupled lower-degree
    matrix on every level (each colour block of A is diagonal), so a colour sweep is an exact Gauss-Seidel
    step; the cycle (colours 0-3 before, 3-0 after) is a symmetric operator."""
    n = 9
    s = p1.build(n, 2, 3, basis.LEGENDRE, 0.3)
    off = basis.degree_levels(s.alphas)
    cyc = p1.MulticolourCoupledGSHierarchy(s, np.arange(off[-2]))
    for l, cols in enumerate(cyc.colours):
        A = cyc.A[l].tocsr()
        assert sum(len(c) for c in cols) == A.shape[0]
        for c in cols:
            sub = A[c][:, c].tocoo()
            assert np.all(sub.row[np.abs(sub.data) > 0] == sub.col[np.abs(sub.data) > 0])
    N = cyc.A[0].shape[0]
    B = cyc.vcycle(np.eye(N))
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()


def test_red_black_sweep_is_gauss_seidel_in_colour_order():
    """``order="rb"``: one forward sweep of the oracle (a triangular solve of the permuted matrix) is
    the point Gauss-Seidel update written out node by node, colour 0 then colour 1, and, the colours
    being independent sets of the 5-point matrix, also a Jacobi step on each colour in turn; the
    backward sweep visits colour 1 first.  The cycle is symmetric and contracts the K_0 error."""
    n = 9
    s = p1.build(n, 1, 1, basis.LEGENDRE, 0.0)
    H = p1.GSHierarchy(s.K[0], n, order="rb")
    rng = np.random.default_rng(3)
    for l, nl in enumerate(H.sizes[:-1]):
        A = H.A[l].toarray()
        m = nl - 2
        x0, b = rng.standard_normal(m * m), rng.standard_normal(m * m)
        colour = [((t % m) + (t // m)) % 2 for t in range(m * m)]
        for forward, fac in ((True, H.low[l]), (False, H.up[l])):
            got = H._sweep(fac, l, x0.copy(), b)
            x = x0.copy()                               # node by node, in the sweep's order
            order = [t for c in ((0, 1) if forward else (1, 0)) for t in range(m * m) if colour[t] == c]
            if not forward:
                order = [t for c in (1, 0) for t in reversed(range(m * m)) if colour[t] == c]
            for t in order:
                x[t] = (b[t] - sum(A[t, u] * x[u] for u in range(m * m) if u != t)) / A[t, t]
            assert np.abs(got - x).max() <= 1e-13
            y = x0.copy()                               # colour by colour, Jacobi on each colour
            for c in ((0, 1) if forward else (1, 0)):
                idx = [t for t in range(m * m) if colour[t] == c]
                y[idx] += (b - A @ y)[idx] / np.diag(A)[idx]
            assert np.abs(got - y).max() <= 1e-13
    n = 17
    s = p1.build(n, 1, 1, basis.LEGENDRE, 0.0)
    H = p1.GSHierarchy(s.K[0], n, order="rb")
    N = s.K[0].shape[0]
    B = H.vcycle(np.eye(N))
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    E = np.eye(N) - B @ s.K[0].toarray()
    assert max(abs(np.linalg.eigvals(E))) < 0.2
