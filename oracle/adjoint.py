"""Adjoint gradients of statistics of int u dx (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Quantity of interest: Q = int u dx.  With u = sum_i u_i psi_i (Eq. PCE_u) and
orthonormal psi_i (psi_0 = 1), E[Q] = m^T U_0 and Var[Q] = sum_{i>=1} (m^T U_i)^2
with m_s = int phi_s dx.  Objective J = E[Q] + Var[Q] / 2.

The SG system A(theta) U = F (Eq. tensor-product) depends on the per-cell mean
coefficient abar_e (through K_0) and on sigma (through every K_k, k >= 1,
which is linear in sigma).  F does not depend on theta.  The adjoint
lambda solves A^T lambda = dJ/dU, and
  dJ/dtheta = - lambda^T (dA/dtheta) U,
  dA/dabar_e = I (x) K_ref^(e)   (cell e's element matrix scattered to its nodes),
  dA/dsigma  = sum_{k>=1} G_k (x) K_k / sigma.
Pins: central finite differences of J through the direct solver.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import fem, sg


def objective(sys, U):
    """J = m^T U_0 + 1/2 sum_{i>=1} (m^T U_i)^2 and its gradient dJ/dU."""
    m = fem.node_mass_weights(sys.n)
    Um = np.asarray(U).reshape(sys.P, sys.Nx)
    mu = Um @ m
    J = mu[0] + 0.5 * np.sum(mu[1:] ** 2)
    g = np.outer(np.concatenate([[1.0], mu[1:]]), m)
    return J, g.reshape(-1)


def cell_quadratic_forms(sys, Lam, U):
    """s_e = sum_i Lam_i|_e^T K_ref U_i|_e for every cell e."""
    Kref = fem.q1_reference_stiffness()
    corners = fem.cell_corner_nodes(sys.n)
    P, Nx = sys.P, sys.Nx
    Lp = np.concatenate([np.asarray(Lam).reshape(P, Nx), np.zeros((P, 1))], axis=1)
    Up = np.concatenate([np.asarray(U).reshape(P, Nx), np.zeros((P, 1))], axis=1)
    idx = np.where(corners >= 0, corners, Nx)
    Le, Ue = Lp[:, idx], Up[:, idx]                       # (P, Nc, 4)
    return np.einsum("pea,ab,peb->e", Le, Kref, Ue)


def gradients(sys, U, Lam, coef_unit):
    """(dJ/dabar per cell, dJ/dsigma) given the forward solution U and adjoint Lam.

    ``coef_unit`` are the KL coefficients at sigma = 1 (rows 1..M), so that
    dA/dsigma = sum_k G_k (x) K_k(coef_unit).
    """
    g_abar = -cell_quadratic_forms(sys, Lam, U)
    dsys = sg.build(sys.n, sys.M, sys.p, sys.family,
                    np.concatenate([np.zeros((1, coef_unit.shape[1])), coef_unit[1:]]))
    dAU = sg.apply(dsys, U)
    g_sigma = -float(np.dot(Lam, dAU))
    return g_abar, g_sigma


def solve_and_gradients(sys, coef_unit, f_nodes=None):
    """Forward direct solve, adjoint direct solve with A^T, and both gradients."""
    A = sg.assemble(sys)
    F = sg.rhs(sys, f_nodes)
    U = spla.spsolve(A.tocsc(), F)
    J, gU = objective(sys, U)
    Lam = spla.spsolve(A.T.tocsc(), gU)
    g_abar, g_sigma = gradients(sys, U, Lam, coef_unit)
    return J, U, Lam, g_abar, g_sigma
