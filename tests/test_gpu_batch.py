"""Batched solves of uneven systems (sg_solve_batch): every system of a small uneven batch
against the oracle's direct solution, and against the same system solved alone through
sg_solve (the batch runs the same kernels on other streams, so the results agree to
rounding; they are in fact deterministic)."""
import numpy as np
import pytest

from oracle import basis, sg as osg
from paper_1304_1755_gb300 import sg
from _gpu_util import Pair, dev, host

pytestmark = pytest.mark.gpu

SHAPES = [(33, 2, 2, 0.3), (65, 3, 2, 0.2), (33, 3, 3, 0.4), (65, 2, 3, 0.3), (17, 2, 2, 0.1), (65, 4, 2, 0.25)]


@pytest.mark.parametrize("nstreams", [1, 3, 8])
def test_batch_matches_direct_and_single_solves(nstreams):
    import torch
    pairs = [Pair(n, M, p, basis.LEGENDRE, sigma=s) for n, M, p, s in SHAPES]
    Fs = [dev(osg.rhs(pr.sys)) for pr in pairs]
    Us = [torch.zeros_like(F) for F in Fs]
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=30, tol=1e-11, pc_prec=sg.F32, maxit=300)
    infos = sg.solve_batch([pr.h for pr in pairs], Fs, Us, nstreams=nstreams, **opts)
    torch.cuda.synchronize()
    for pr, F, U, info in zip(pairs, Fs, Us, infos):
        assert info.status == 0 and info.relres_true <= 1e-11
        Ustar = osg.solve_direct(osg.assemble(pr.sys), host(F))
        got = host(U)
        assert np.linalg.norm(got - Ustar) <= 1e-6 * np.linalg.norm(Ustar)
        U1 = torch.zeros_like(F)
        pr.h.solve(F, U1, **opts)
        torch.cuda.synchronize()
        assert np.abs(host(U1) - got).max() <= 1e-14 * np.abs(got).max()


def test_batch_rejects_bad_arguments():
    import ctypes
    pr = Pair(17, 2, 2)
    L = sg.lib()
    o = sg.SolveOpts(sg.FGMRES, sg.PC_BLOCKTRI, 30, 100, 1e-8, sg.F32, 0, 0, 0, 0)
    hs = (sg.VP * 1)(pr.h.h)
    null = (sg.VP * 1)(None)
    assert L.sg_solve_batch(hs, null, null, 1, ctypes.byref(o), None, 2) == -1
    assert L.sg_solve_batch(hs, null, null, 1, ctypes.byref(o), None, 0) == -1
    assert L.sg_solve_batch(hs, null, null, 0, ctypes.byref(o), None, 2) == 0


@pytest.mark.parametrize("n", [65, 129])
def test_autotuned_tile_gives_identical_operator(n):
    """The tile only changes which warp computes a node, not the arithmetic: the operator is
    bit-identical before and after tuning, in all three arithmetic forms."""
    import torch
    from paper_1304_1755_gb300 import inputs
    pr = Pair(n, 3, 3)
    X = dev(inputs.uniform(51, pr.N))
    outs = []
    for tuned in (False, True):
        if tuned:
            pr.h.autotune()
        Y64 = torch.empty_like(X)
        pr.h.apply(X, Y64, sg.F64)
        Xb = X.to(torch.bfloat16)
        Yb = torch.empty_like(Xb)
        pr.h.apply(Xb, Yb, sg.BF16)
        Xd = torch.cat([X.float(), (X - X.float().double()).float()])      # double-float hi, lo
        Yd = torch.empty_like(Xd)
        pr.h.apply(Xd, Yd, sg.DF64)
        torch.cuda.synchronize()
        outs.append((host(Y64), host(Yb), host(Yd)))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
