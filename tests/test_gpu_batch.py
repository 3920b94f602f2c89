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


GRAPH_CASES = [  # pc_prec, arith, precond, restart
    (sg.F64, sg.ARITH_F64, sg.PC_BLOCKTRI, 30),
    (sg.F32, sg.ARITH_F64_DFOP, sg.PC_BLOCKTRI, 30),
    (sg.BF16Z, sg.ARITH_F64_DFOP, sg.PC_BLOCKTRI, 30),
    (sg.F32, sg.ARITH_F64, sg.PC_BLOCKDIAG, 30),
    (sg.F32, sg.ARITH_F64_DFOP, sg.PC_BLOCKTRI, 4),       # several restart cycles: several graph launches
]


@pytest.mark.parametrize("case", GRAPH_CASES, ids=lambda c: f"p{c[0]}a{c[1]}pc{c[2]}m{c[3]}")
def test_batch_graph_matches_direct_and_single_solves(case):
    """sg_solve_batch_graph (the whole batch in one CUDA graph, Arnoldi scalars on the device) against
    the oracle's direct solutions and against sg_solve on each system alone: the same iterations
    (the scalar work is the host's, in the same order, on the device) and the same solution to
    rounding; a zero right-hand side in the batch gives U = 0."""
    import torch
    pcp, arith, pc, restart = case
    pairs = [Pair(n, M, p, basis.LEGENDRE, sigma=s) for n, M, p, s in SHAPES]
    Fs = [dev(osg.rhs(pr.sys)) for pr in pairs]
    Fs[4] = torch.zeros_like(Fs[4])
    Us = [torch.full_like(F, 7.0) for F in Fs]
    opts = dict(method=sg.FGMRES, precond=pc, restart=restart, tol=1e-11, pc_prec=pcp, maxit=400, arith=arith)
    infos = sg.solve_batch_graph([pr.h for pr in pairs], Fs, Us, **opts)
    torch.cuda.synchronize()
    bar = 1e-8 if pcp == sg.F64 else 1e-6
    for s, (pr, F, U, info) in enumerate(zip(pairs, Fs, Us, infos)):
        assert info.status == 0, (s, info.status)
        got = host(U)
        if s == 4:
            assert not got.any() and info.iters == 0
            continue
        assert info.relres_true <= 1e-11
        Ustar = osg.solve_direct(osg.assemble(pr.sys), host(F))
        assert np.linalg.norm(got - Ustar) <= bar * np.linalg.norm(Ustar)
        rr = np.linalg.norm(host(F) - osg.apply(pr.sys, got)) / np.linalg.norm(host(F))
        assert rr <= 2e-11 and abs(rr - info.relres_true) <= 1e-13
        U1 = torch.zeros_like(F)
        i1 = pr.h.solve(F, U1, **opts)
        torch.cuda.synchronize()
        assert abs(i1.iters - info.iters) <= 1
        assert np.linalg.norm(host(U1) - got) <= 1e-9 * np.linalg.norm(got)


def test_batch_graph_rejects_unsupported_options():
    import torch
    pr = Pair(17, 2, 2)
    F = dev(osg.rhs(pr.sys))
    U = torch.zeros_like(F)
    for bad in (dict(arith=sg.ARITH_DF64, pc_prec=sg.F32), dict(method=sg.GPCG), dict(restart=40),
                dict(arith=sg.ARITH_F64_DFOP, pc_prec=sg.F64)):
        o = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=30, tol=1e-8, pc_prec=sg.F32, maxit=100)
        o.update(bad)
        with pytest.raises(sg.SGError):
            sg.solve_batch_graph([pr.h], [F], [U], **o)


def test_batch_object_solves_repeatedly_and_guards_its_workspace():
    """sg_batch_create builds the graphs once; sg_batch_solve gives the same result on every call (the
    start graph resets U and the device state), and refuses to run after a handle's workspace grew."""
    import torch
    pairs = [Pair(n, M, p, basis.LEGENDRE, sigma=s) for n, M, p, s in SHAPES[:3]]
    Fs = [dev(osg.rhs(pr.sys)) for pr in pairs]
    Us = [torch.zeros_like(F) for F in Fs]
    b = sg.Batch([pr.h for pr in pairs], Fs, Us, restart=20, tol=1e-10, pc_prec=sg.F32, arith=sg.ARITH_F64_DFOP)
    first = b.solve()
    U1 = [U.clone() for U in Us]
    second = b.solve()
    torch.cuda.synchronize()
    assert [i.iters for i in first] == [i.iters for i in second]
    assert all(torch.equal(a, c) for a, c in zip(U1, Us))
    pairs[0].h.solve(Fs[0], torch.zeros_like(Fs[0]), restart=30, pc_prec=sg.F32)    # grows handle 0's basis
    with pytest.raises(sg.SGError):
        b.solve()
    b.close()
