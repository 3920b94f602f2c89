"""Parity at the full bandwidth-scale size (1025^2 grid, M = 6 Hermite, p = 4: 219,771,090
unknowns), in the configuration the bench times (FGMRES(20) with an FP64 Arnoldi basis and
Gram-Schmidt and the double-float outer operator, BF16-storage preconditioner with FP32
output) and in the all-double-float Krylov variant: the library's load vector must equal the
oracle's, the GPU solve must reach a true relative residual of 1e-8,
and the FP64 residual the library computes must agree, at 4096 sampled (PC row, node) pairs,
with the oracle's own evaluation of F - A U at those pairs (Eq. tensor-product, written out
per node from the Q1 element matrix and the closed-form G_k).  The oracle cannot solve or even
assemble this system, so the check is on sampled outputs plus the residual property."""
import numpy as np
import pytest
from scipy import sparse

from oracle import basis, fem, kl
from paper_1304_1755_gb300 import inputs, sg

pytestmark = pytest.mark.gpu

N_, M_, P_DEG, SIG = 1025, 6, 4, 0.2


def _sampled_residual(coef, Gs, U, F, rows, nodes, n):
    """r[i, s] = F[i, s] - sum_k sum_j G_k[i, j] (K_k U_j)_s for the sampled pairs, in FP64 (one
    pair at a time), with the absolute sum of the terms (the scale of the rounding error)."""
    Kref = fem.q1_reference_stiffness()
    m = n - 2
    r = np.empty(len(rows))
    scale = np.empty(len(rows))
    Gcsr = [sparse.csr_matrix(G) for G in Gs]
    for q, (i, s) in enumerate(zip(rows, nodes)):
        vx, vy = s % m + 1, s // m + 1                    # vertex coordinates of the node
        acc, sc = F[i, s], abs(F[i, s])
        # the four cells around the node (SW corner (cx, cy)) and the node's corner in each
        for cx, cy, a in ((vx - 1, vy - 1, 2), (vx, vy - 1, 3), (vx - 1, vy, 1), (vx, vy, 0)):
            e = cx + cy * (n - 1)
            corners = []
            for wx, wy in ((cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)):
                inside = 1 <= wx <= n - 2 and 1 <= wy <= n - 2
                corners.append((wx - 1) + (wy - 1) * m if inside else -1)
            for k, G in enumerate(Gcsr):
                for j, g in zip(G.indices[G.indptr[i]:G.indptr[i + 1]], G.data[G.indptr[i]:G.indptr[i + 1]]):
                    z = [U[j, c] if c >= 0 else 0.0 for c in corners]
                    t = sum(Kref[a, b] * z[b] for b in range(4))
                    acc -= g * coef[k, e] * t
                    sc += abs(g * coef[k, e]) * sum(abs(Kref[a, b] * z[b]) for b in range(4))
        r[q], scale[q] = acc, sc
    return r, scale


@pytest.mark.parametrize("arith", [sg.ARITH_F64_DFOP, sg.ARITH_DF64], ids=["f64_dfop", "df64"])
def test_c3_fullsize_residual_at_sampled_outputs(arith):
    import torch
    n, M, p = N_, M_, P_DEG
    coef = kl.kl_coefficients(n, M, SIG)
    alphas = basis.multi_indices(M, p)
    Gs = basis.g_matrices(alphas, basis.HERMITE)          # G_0 = I, G_1 .. G_M
    h = sg.Handle(n, M, p, sg.HERMITE, coef, stream=torch.cuda.current_stream())
    N = h.P * h.Nx
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    h.rhs(F)
    torch.cuda.synchronize()
    F0 = F[:h.Nx].cpu().numpy()
    assert np.array_equal(F0, fem.load_vector(n)) and float(F[h.Nx:].abs().max()) == 0.0
    U = torch.zeros_like(F)
    info = h.solve(F, U, method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=20, maxit=200, tol=1e-8,
                   pc_prec=sg.BF16Z, arith=arith)
    assert info.status == 0 and info.relres_true <= 1e-8
    R = torch.empty_like(F)
    h.residual(F, U, R)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(R) / torch.linalg.norm(F)) <= 1e-8
    rng = inputs.rng(77)
    rows = rng.integers(0, h.P, 4096)
    nodes = rng.integers(0, h.Nx, 4096)
    Uh = U.cpu().numpy().reshape(h.P, h.Nx)
    Fh = F.cpu().numpy().reshape(h.P, h.Nx)
    Rs = R.cpu().numpy().reshape(h.P, h.Nx)[rows, nodes]
    r_or, scale = _sampled_residual(coef, Gs, Uh, Fh, rows, nodes, n)
    assert np.all(np.abs(Rs - r_or) <= 1e-13 * scale + 1e-300)
    h.close()
