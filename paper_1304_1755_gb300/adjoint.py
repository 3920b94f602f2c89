"""Adjoint gradients of J = E[int u dx] + Var[int u dx] / 2 behind a torch.autograd.Function.

The forward pass solves the SG system A(abar, sigma) U = F (Eq. tensor-product) with the
block-triangular preconditioned FGMRES of the C ABI and evaluates J with
``sg_objective``; the backward pass solves the adjoint system A^T Lam = dJ/dU with the
transposed (upper block-triangular) sweep and forms
  dJ/dabar_e = -sum_i Lam_i|e^T K_ref U_i|e,   dJ/dsigma = -(1/sigma) Lam^T (A - I (x) K_0) U
with ``sg_adjoint_gradients``.  Every step runs in the library's kernels; this module
only marshals tensors.  abar is the per-cell mean coefficient ((n-1)^2 values), sigma the
standard deviation that scales the unit-variance KL modes.
"""
import torch

from . import sg


class SGObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, abar, sigma, spec):
        n, M, p, family = spec["n"], spec["M"], spec["p"], spec["family"]
        # coefficients (sg_kl_coef: row 0 = abar, rows k >= 1 = sigma sqrt(lambda_k) b_k) and the load
        # vector (sg_rhs) come from the library; abar crosses to the host because sg_kl_coef is host code
        coef, _ = sg.sg_kl_coef(n, M, float(sigma), spec.get("corr_len", 1.0),
                                abar=abar.detach().to("cpu", torch.float64).numpy())
        stream = torch.cuda.current_stream()
        h = sg.Handle(n, M, p, family, coef, stream=stream)
        N = h.P * h.Nx
        F = torch.empty(N, dtype=torch.float64, device=abar.device)
        h.rhs(F, spec.get("f"))
        U = torch.zeros_like(F)
        opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=spec.get("restart", 30),
                    tol=spec.get("tol", 1e-10), pc_prec=spec.get("pc_prec", sg.F64), maxit=spec.get("maxit", 500))
        info = h.solve(F, U, **opts)
        G = torch.empty_like(U)
        J = h.objective(U, G)
        ctx.h, ctx.opts, ctx.sigma = h, opts, float(sigma)
        ctx.save_for_backward(U, G)
        ctx.info = info
        return torch.tensor(J, dtype=torch.float64, device=abar.device)

    @staticmethod
    def backward(ctx, gJ):
        U, G = ctx.saved_tensors
        h = ctx.h
        Lam = torch.zeros_like(U)
        h.solve(G, Lam, transpose=True, **ctx.opts)
        g_abar = torch.empty((h.n - 1) ** 2, dtype=torch.float64, device=U.device)
        g_sigma = h.adjoint_gradients(U, Lam, ctx.sigma, g_abar)
        h.close()
        return gJ * g_abar, gJ * torch.tensor(g_sigma, dtype=torch.float64, device=U.device), None


def objective(abar, sigma, n, M, p, family=sg.LEGENDRE, corr_len=1.0, **opts):
    """J(abar, sigma) as a differentiable scalar (abar: cuda float64 tensor of (n-1)^2 cells,
    sigma: 0-d float64 tensor).  opts: restart, tol, pc_prec, maxit, and f (device FP64 values of
    f at the (n-2)^2 interior nodes; f = 1 when absent)."""
    spec = dict(n=n, M=M, p=p, family=family, corr_len=corr_len, **opts)
    return SGObjective.apply(abar, sigma, spec)
