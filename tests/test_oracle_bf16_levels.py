"""Why BF16 storage of the V-cycle's levels costs the configured bandwidth-scale solve Krylov
iterations, checked on the CPU with the oracle: the oracle's V(1,1) cycle with its coarse-level
right-hand sides b_l and/or corrections x_l rounded to BF16 (round to nearest even, as the library's
stores do) at the points where the library stores them, inside the oracle's block-triangular FGMRES.
Rounding the restricted residuals costs nothing; rounding the corrections costs iterations, because
the rounding noise of a coarse correction is smooth on the finer grids (their smoothers leave it) and
the operator amplifies it."""
import numpy as np

from oracle import basis, kl, krylov, mg, precond, sg as osg


def _bf16(x):
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    u = ((u + (((u >> 16) & 1) + 0x7FFF)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


class _RoundedCycle(mg.Hierarchy):
    """The oracle's V-cycle with b_l and/or x_l (levels 1 .. the last one with n > 33, as the library keeps
    them in global memory) rounded to BF16."""

    def __init__(self, K0, n, round_b, round_x):
        super().__init__(K0, n)
        self.round_b, self.round_x = round_b, round_x
        self.lc = next(i for i, m in enumerate(self.sizes) if m <= 33)

    def vcycle(self, b, level=0):
        A = self.A[level]
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        Dinv = self.Dinv[level] if b.ndim == 1 else self.Dinv[level][:, None]
        x = self.omega * Dinv * b
        bc = self.P[level].T @ (b - A @ x)
        if self.round_b and level + 1 <= self.lc:
            bc = _bf16(bc)
        xc = self.vcycle(bc, level + 1)
        if self.round_x and level + 1 <= self.lc:
            xc = _bf16(xc)
        x = x + self.P[level] @ xc
        return x + self.omega * Dinv * (b - A @ x)


def test_bf16_rounding_of_corrections_costs_iterations_and_of_residuals_does_not():
    n, M, p = 257, 4, 3
    s = osg.build(n, M, p, basis.LEGENDRE, kl.kl_coefficients(n, M, 0.3))
    F = osg.rhs(s)
    A = lambda v: osg.apply(s, v)
    its = {}
    for tag, rb, rx in (("fp64", False, False), ("bf16 b", True, False), ("bf16 x", False, True)):
        solver = precond.DiagSolver(s.K[0], _RoundedCycle(s.K[0], n, rb, rx))
        _, its[tag], rr = krylov.gmres(A, lambda r: precond.block_tri_inv(s, solver, r), F, tol=1e-8, restart=30,
                                       maxit=100, flexible=True)
        assert rr <= 1e-8
    assert its["bf16 b"] == its["fp64"]
    assert its["bf16 x"] > its["fp64"]
