"""GPU adjoint gradients (C4 shape on a 33x33 copy: M = 4 Legendre, p = 3, sigma = 0.4,
lognormal mean coefficient) through the torch.autograd.Function, against the oracle's FP64
adjoint (direct solves) and against central finite differences of the GPU objective.

Tolerance: both solves run to a relative residual of 1e-12, so J, U and Lam carry relative
errors of order kappa * 1e-12 ~ 1e-9; gradients are compared at 1e-7 relative."""
import numpy as np
import pytest

from oracle import adjoint as oadj, basis, kl, sg as osg
from paper_1304_1755_gb300 import inputs

pytestmark = pytest.mark.gpu

N_, M_, P_, SIG = 33, 4, 3, 0.4


def _oracle():
    unit = kl.kl_coefficients(N_, M_, 1.0)
    abar = inputs.lognormal_cells(2, N_, 0.2)
    coef = unit.copy()
    coef[0] = abar
    coef[1:] *= SIG
    s = osg.build(N_, M_, P_, basis.LEGENDRE, coef)
    return abar, unit, oadj.solve_and_gradients(s, unit)


def test_autograd_gradients_match_oracle_adjoint():
    import torch
    from paper_1304_1755_gb300 import adjoint
    abar_np, unit, (J_ref, U_ref, L_ref, gab_ref, gs_ref) = _oracle()
    abar = torch.tensor(abar_np, dtype=torch.float64, device="cuda", requires_grad=True)
    sigma = torch.tensor(SIG, dtype=torch.float64, device="cuda", requires_grad=True)
    J = adjoint.objective(abar, sigma, N_, M_, P_, tol=1e-12)
    J.backward()
    assert abs(float(J.detach()) - J_ref) <= 1e-9 * abs(J_ref)
    g = abar.grad.cpu().numpy()
    assert np.linalg.norm(g - gab_ref) <= 1e-7 * np.linalg.norm(gab_ref)
    assert abs(float(sigma.grad) - gs_ref) <= 1e-7 * abs(gs_ref)


def test_autograd_gradients_match_finite_differences():
    import torch
    from paper_1304_1755_gb300 import adjoint
    abar_np = inputs.lognormal_cells(2, N_, 0.2)
    abar = torch.tensor(abar_np, dtype=torch.float64, device="cuda", requires_grad=True)
    sigma = torch.tensor(SIG, dtype=torch.float64, device="cuda", requires_grad=True)
    J = adjoint.objective(abar, sigma, N_, M_, P_, tol=1e-13)
    J.backward()
    eps = 1e-5
    with torch.no_grad():
        for seed in range(100, 104):
            d = torch.tensor(inputs.normal(seed, abar_np.shape), dtype=torch.float64, device="cuda")
            jp = float(adjoint.objective(abar + eps * d, sigma, N_, M_, P_, tol=1e-13))
            jm = float(adjoint.objective(abar - eps * d, sigma, N_, M_, P_, tol=1e-13))
            fd = (jp - jm) / (2 * eps)
            assert abs(fd - float(abar.grad @ d)) <= 1e-6 * abs(fd)
        jp = float(adjoint.objective(abar, sigma + eps, N_, M_, P_, tol=1e-13))
        jm = float(adjoint.objective(abar, sigma - eps, N_, M_, P_, tol=1e-13))
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - float(sigma.grad)) <= 1e-6 * abs(fd)
