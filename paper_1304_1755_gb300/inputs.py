"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds random draws and recipes for inputs only; it contains none
of the method's arithmetic (no KL, basis, stiffness, multigrid or Krylov code).
All generators use numpy's PCG64 with an explicit seed.

Recipes (the paper's own experiments use no external data set):
  * random operator inputs X ~ U(-1, 1), shape (P, N_x)
  * RHS perturbation: f_s = 1 + 0.1 z_s, z_s ~ N(0, 1) at interior nodes
  * lognormal mean coefficient: abar_e = exp(log_std * z_e), z_e ~ N(0, 1) per cell
  * finite-difference directions: N(0, 1) per cell
  * uneven batches: per system L ~ U{6..9} (n = 2^L + 1), M ~ U{2..6},
    p ~ U{2..4}, sigma ~ U[0.1, 0.5]
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(seed, shape, lo=-1.0, hi=1.0):
    return rng(seed).uniform(lo, hi, size=shape)


def normal(seed, shape):
    return rng(seed).standard_normal(size=shape)


def rhs_nodes(seed, n, amplitude=0.1):
    """f at the (n-2)^2 interior nodes: 1 + amplitude * N(0,1)."""
    return 1.0 + amplitude * normal(seed, (n - 2) ** 2)


def lognormal_cells(seed, n, log_std=0.2):
    """Per-cell mean coefficient exp(log_std * z) on the (n-1)^2 cells."""
    return np.exp(log_std * normal(seed, (n - 1) ** 2))


def random_cell_coefficients(seed, n, M, mean=1.0, spread=0.15):
    """Generic per-cell coefficient rows (M+1, (n-1)^2) for operator tests:
    row 0 = mean * (1 + U(-spread, spread)), rows k >= 1 = U(-spread, spread)."""
    g = rng(seed)
    c = g.uniform(-spread, spread, size=(M + 1, (n - 1) ** 2))
    c[0] = mean * (1.0 + c[0])
    return c


def batch_systems(seed, count):
    """Parameters of an uneven batch: list of dicts (n, M, p, sigma, seed)."""
    g = rng(seed)
    out = []
    for b in range(count):
        L = int(g.integers(6, 10))
        out.append(dict(n=2 ** L + 1, M=int(g.integers(2, 7)), p=int(g.integers(2, 5)),
                        sigma=float(g.uniform(0.1, 0.5)), seed=1000 + b))
    return out
