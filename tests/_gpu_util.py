"""Helpers shared by the GPU parity tests: one SG problem built twice from the same
seeded inputs -- once by the oracle (CPU, FP64) and once through the C ABI."""
import numpy as np

from oracle import basis, kl, mg, precond, sg as osg
from paper_1304_1755_gb300 import inputs


def coefficients(n, M, sigma=0.3, mean="one", seed=7):
    """KL coefficients (from the oracle's own KL) with a constant, lognormal or random mean row."""
    coef = kl.kl_coefficients(n, M, sigma)
    if mean == "lognormal":
        coef[0] = inputs.lognormal_cells(seed, n, 0.2)
    elif mean == "random":
        coef = inputs.random_cell_coefficients(seed, n, M, spread=0.2)
    return coef


class Pair:
    def __init__(self, n, M, p, family=basis.LEGENDRE, sigma=0.3, mean="one", nu=(1, 1), seed=7, coef=None):
        self.memo = {}                      # oracle results a test module may reuse across parameters
        import torch
        from paper_1304_1755_gb300 import sg
        self.coef = coefficients(n, M, sigma, mean, seed) if coef is None else coef
        self.sys = osg.build(n, M, p, family, self.coef)
        self.h = sg.Handle(n, M, p, family, self.coef, nu1=nu[0], nu2=nu[1],
                           stream=torch.cuda.current_stream())
        self.nu = nu
        assert self.h.P == self.sys.P and self.h.Nx == self.sys.Nx
        self._hier = None

    @property
    def hier(self):
        if self._hier is None:
            self._hier = mg.Hierarchy(self.sys.K[0], self.sys.n, nu1=self.nu[0], nu2=self.nu[1])
        return self._hier

    @property
    def N(self):
        return self.sys.P * self.sys.Nx

    def oracle_vsolver(self):
        return precond.DiagSolver(self.sys.K[0], self.hier)


def dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()


_PAIRS = {}


def pair(n, M, p, family=basis.LEGENDRE, sigma=0.3, mean="one", nu=(1, 1), seed=7):
    """A Pair shared by the tests of one process (the oracle set-up of the large grids is the slow
    part of these tests).  Users must not change the handle's state (stream, tuning)."""
    key = (n, M, p, family, sigma, mean, tuple(nu), seed)
    if key not in _PAIRS:
        _PAIRS[key] = Pair(n, M, p, family, sigma=sigma, mean=mean, nu=nu, seed=seed)
    return _PAIRS[key]


def residual_rounding(sys, U, F):
    """One rounding unit of the relative residual ||F - A U|| / ||F|| in FP64: eps ||(|F| + |A| |U|)|| /
    ||F||, |A| = sum_k |G_k| (x) |K_k|.  Each entry of a computed F - A U is off by a few eps times the
    entry of |F| + |A| |U| with signs that mostly cancel over the vector, so two evaluations that sum in
    different orders (the library's kernels, scipy) differ by a fraction of this unit; near the solve's
    attainable accuracy the residual itself is of that size."""
    import dataclasses
    absys = dataclasses.replace(sys, G=[np.abs(g) for g in sys.G], K=[abs(k) for k in sys.K])
    return np.finfo(float).eps * np.linalg.norm(np.abs(F) + osg.apply(absys, np.abs(U))) / np.linalg.norm(F)
