"""GPU parity of the Krylov solves (Sec. 4.2, 6) against the oracle's exact solution.

Bar: relative L2 error of the coefficient vector <= 1e-8 for FP64 runs and <= 1e-6
for mixed-precision preconditioners, with the GPU solve run to a true relative
residual of 1e-12 (a residual alone bounds the error only up to the condition
number).  Also: the recomputed residual is checked by the oracle's own operator.
"""
import numpy as np
import pytest

from oracle import basis, krylov, precond, sg as osg
from paper_1304_1755_gb300 import inputs, sg
from _gpu_util import Pair, dev, host, residual_rounding

pytestmark = pytest.mark.gpu


def _direct(pr, F):
    """U* by sparse LU for small systems; above 1e5 unknowns by the oracle's BD-PCG with an exact
    LU of K_0 run to a relative residual of 1e-14 (A is SPD for these cases), with the assembled
    operator up to 1e6 unknowns and the oracle's matrix-free one above."""
    if pr.N <= 100_000:
        return osg.solve_direct(osg.assemble(pr.sys), F)
    if pr.N <= 1_000_000:
        A = osg.assemble(pr.sys)
        apply_A = lambda v: A @ v
    else:
        apply_A = lambda v: osg.apply(pr.sys, v)
    solver = precond.DiagSolver(pr.sys.K[0])
    # the attainable true residual of an FP64 solve grows with the system (rounding of the operator):
    # 1e-13 up to 1e6 unknowns, 5e-12 above
    tol = 1e-14 if pr.N <= 1_000_000 else 1e-12
    U, its, rr = krylov.pcg(apply_A, lambda r: precond.block_diag_inv(pr.sys, solver, r), F, tol=tol,
                            maxit=500)
    assert rr <= (1e-13 if pr.N <= 1_000_000 else 5e-12), rr
    return U


CASES = [  # method, precond, pc_prec, restart
    (sg.FGMRES, sg.PC_BLOCKTRI, sg.F64, 30),
    (sg.GMRES, sg.PC_BLOCKTRI, sg.F64, 30),
    (sg.FGMRES, sg.PC_BLOCKDIAG, sg.F64, 30),
    (sg.GPCG, sg.PC_BLOCKTRI, sg.F64, 0),
    (sg.PCG, sg.PC_BLOCKDIAG, sg.F64, 0),
    (sg.FGMRES, sg.PC_BLOCKTRI, sg.F32, 30),
    (sg.FGMRES, sg.PC_BLOCKTRI, sg.BF16, 30),
    (sg.FGMRES, sg.PC_BLOCKTRI, sg.BF16Z, 30),
    (sg.GPCG, sg.PC_BLOCKTRI, sg.BF16Z, 0),
    (sg.FGMRES, sg.PC_NONE, sg.F64, 30),
    (sg.PCG, sg.PC_BLOCKSYM, sg.F64, 0),
    (sg.FGMRES, sg.PC_BLOCKSYM, sg.F32, 30),
    (sg.BGS, sg.PC_BLOCKTRI, sg.F64, 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"m{c[0]}pc{c[1]}p{c[2]}")
def test_c1_solvers_match_direct(case):
    import torch
    method, pc, pcp, restart = case
    pr = Pair(33, 2, 2, sigma=0.3)               # C1: 33^2 Q1, M = 2 Legendre, p = 2, sigma = 0.3
    F = osg.rhs(pr.sys)
    Ustar = _direct(pr, F)
    U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(dev(F), U, method=method, precond=pc, pc_prec=pcp, restart=max(restart, 1),
                      tol=1e-12, maxit=3000 if pc == sg.PC_NONE else 300)
    assert info.status == 0
    got = host(U)
    err = np.linalg.norm(got - Ustar) / np.linalg.norm(Ustar)
    assert err <= (1e-8 if pcp == sg.F64 else 1e-6), err
    rr = np.linalg.norm(F - osg.apply(pr.sys, got)) / np.linalg.norm(F)
    assert rr <= 2e-12 and abs(rr - info.relres_true) <= 1e-13


def test_c1_iteration_counts_bt_below_bd():
    import torch
    pr = Pair(33, 2, 2, sigma=0.3)
    F = dev(osg.rhs(pr.sys))
    its = {}
    for pc in (sg.PC_BLOCKTRI, sg.PC_BLOCKDIAG):
        U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
        its[pc] = pr.h.solve(F, U, precond=pc, tol=1e-8).iters
    assert its[sg.PC_BLOCKTRI] < its[sg.PC_BLOCKDIAG]
    # same method and preconditioner in the oracle: counts agree within one step (rounding)
    s = pr.sys
    A = osg.assemble(s)
    solver = pr.oracle_vsolver()
    _, it_o, _ = krylov.gmres(lambda v: A @ v, lambda r: precond.block_tri_inv(s, solver, r), osg.rhs(s),
                              tol=1e-8, restart=30, flexible=True)
    assert abs(it_o - its[sg.PC_BLOCKTRI]) <= 1


@pytest.mark.parametrize("n,M,p,fam,mean", [(65, 3, 3, basis.HERMITE, "lognormal"), (129, 2, 2, basis.LEGENDRE, "one"),
                                              (17, 1, 0, basis.LEGENDRE, "one"), (5, 6, 4, basis.LEGENDRE, "one"),
                                              (33, 0, 3, basis.LEGENDRE, "lognormal")])
def test_solves_other_shapes(n, M, p, fam, mean):
    import torch
    pr = Pair(n, M, p, fam, sigma=0.2, mean=mean)
    F = osg.rhs(pr.sys, inputs.rhs_nodes(1, n))
    Ustar = _direct(pr, F)
    for pcp in (sg.F64, sg.F32):
        U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
        info = pr.h.solve(dev(F), U, pc_prec=pcp, tol=1e-12, restart=20)
        assert info.status == 0
        err = np.linalg.norm(host(U) - Ustar) / np.linalg.norm(Ustar)
        assert err <= (1e-8 if pcp == sg.F64 else 1e-6)


@pytest.mark.parametrize("n,M,p,fam,mean,pcp", [(33, 2, 2, basis.LEGENDRE, "one", sg.F32),
                                                 (33, 2, 2, basis.LEGENDRE, "one", sg.BF16),
                                                 (65, 3, 3, basis.HERMITE, "lognormal", sg.BF16),
                                                 (129, 2, 2, basis.LEGENDRE, "one", sg.F32),
                                                 (65, 3, 3, basis.HERMITE, "lognormal", sg.BF16Z),
                                                 (129, 2, 2, basis.LEGENDRE, "one", sg.BF16Z)])
def test_double_float_fgmres_matches_direct(n, M, p, fam, mean, pcp):
    """Double-float Arnoldi basis and operator (SG_ARITH_DF64): same bar as FP64 runs."""
    import torch
    pr = Pair(n, M, p, fam, sigma=0.3, mean=mean)
    F = osg.rhs(pr.sys, inputs.rhs_nodes(3, n))
    Ustar = _direct(pr, F)
    U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(dev(F), U, pc_prec=pcp, tol=1e-10, restart=30, arith=sg.ARITH_DF64)
    assert info.status == 0 and info.relres_true <= 1e-10
    err = np.linalg.norm(host(U) - Ustar) / np.linalg.norm(Ustar)
    assert err <= 1e-8, err


@pytest.mark.parametrize("n,M,p,fam,mean,pcp,method", [(33, 2, 2, basis.LEGENDRE, "one", sg.F32, sg.FGMRES),
                                                        (65, 3, 3, basis.HERMITE, "lognormal", sg.BF16Z, sg.FGMRES),
                                                        (129, 2, 2, basis.LEGENDRE, "one", sg.BF16Z, sg.FGMRES),
                                                        (65, 2, 3, basis.LEGENDRE, "one", sg.BF16, sg.FGMRES),
                                                        (65, 2, 3, basis.LEGENDRE, "one", sg.F32, sg.GMRES)])
def test_f64_basis_double_float_operator_matches_direct(n, M, p, fam, mean, pcp, method):
    """FP64 Arnoldi basis and Gram-Schmidt with the double-float outer operator
    (SG_ARITH_F64_DFOP), the configured arithmetic of the timed C3 solve: same bar as FP64 runs."""
    import torch
    pr = Pair(n, M, p, fam, sigma=0.3, mean=mean)
    F = osg.rhs(pr.sys, inputs.rhs_nodes(3, n))
    Ustar = _direct(pr, F)
    U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(dev(F), U, method=method, pc_prec=pcp, tol=1e-12, restart=30, arith=sg.ARITH_F64_DFOP)
    assert info.status == 0 and info.relres_true <= 1e-12
    got = host(U)
    err = np.linalg.norm(got - Ustar) / np.linalg.norm(Ustar)
    assert err <= 1e-8, err
    rr = np.linalg.norm(F - osg.apply(pr.sys, got)) / np.linalg.norm(F)
    assert rr <= 2e-12 and abs(rr - info.relres_true) <= residual_rounding(pr.sys, got, F)


def test_f64_dfop_mode_rejects_fp64_preconditioner_and_gpcg():
    import torch
    pr = Pair(9, 1, 1)
    F = dev(osg.rhs(pr.sys))
    U = torch.zeros_like(F)
    assert pr.h.solve(F, U, pc_prec=sg.F64, arith=sg.ARITH_F64_DFOP, check=False).status == -1
    assert pr.h.solve(F, U, method=sg.GPCG, pc_prec=sg.F32, arith=sg.ARITH_F64_DFOP, check=False).status == -1


def test_c2_configuration_solve_matches_oracle():
    """C2 as configured (257^2 Q1, M = 4 Legendre, p = 4: 4,551,750 unknowns, sigma = 0.3,
    f = 1 + 0.1 N(0,1) with seed 1; FP32 preconditioner inside FP64 flexible GMRES(30)), the load
    vector built by the library (sg_rhs) and checked against the oracle's, against the oracle's
    BD-PCG solution with exact K_0 solves (to the attainable 1e-12), and the oracle's residual of
    the GPU solution."""
    import torch
    n, M, p = 257, 4, 4
    pr = Pair(n, M, p, basis.LEGENDRE, sigma=0.3)
    f = inputs.rhs_nodes(1, n)
    F_or = osg.rhs(pr.sys, f)
    Fd = torch.empty(pr.N, dtype=torch.float64, device="cuda")
    pr.h.rhs(Fd, dev(f))
    torch.cuda.synchronize()
    assert np.allclose(host(Fd), F_or, rtol=2 ** -52, atol=0)
    Ustar = _direct(pr, F_or)
    for arith in (sg.ARITH_F64_DFOP, sg.ARITH_F64):
        U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
        info = pr.h.solve(Fd, U, method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=30, maxit=400, tol=5e-12,
                          pc_prec=sg.F32, arith=arith)
        assert info.status == 0 and info.relres_true <= 5e-12
        got = host(U)
        err = np.linalg.norm(got - Ustar) / np.linalg.norm(Ustar)
        assert err <= 1e-6, err                     # the mixed-precision bar (FP32 preconditioner)
        rr = np.linalg.norm(F_or - osg.apply(pr.sys, got)) / np.linalg.norm(F_or)
        assert rr <= 1e-11, rr                      # the oracle's own residual of the GPU solution


def test_repeated_solves_reuse_workspace_deterministically():
    """Workspace is reused across calls and modes (its padding must stay zero): a double-float
    solve, a strict FP64 GPCG solve that scribbles on the shared work vectors, then the
    double-float solve again must give bit-identical results."""
    import torch
    pr = Pair(33, 2, 3, sigma=0.3)
    F = dev(osg.rhs(pr.sys, inputs.rhs_nodes(4, 33)))
    U1 = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    U2, U3 = torch.zeros_like(U1), torch.zeros_like(U1)
    pr.h.solve(F, U1, pc_prec=sg.BF16, arith=sg.ARITH_DF64, tol=1e-10)
    pr.h.solve(F, U2, method=sg.GPCG, tol=1e-10)
    pr.h.solve(F, U3, pc_prec=sg.BF16, arith=sg.ARITH_DF64, tol=1e-10)
    assert torch.equal(U1, U3)
    assert float((U1 - U2).abs().max()) <= 1e-8 * float(U2.abs().max())


def test_transpose_solve_and_host_buffers():
    pr = Pair(33, 2, 3, sigma=0.35)
    F = osg.rhs(pr.sys, inputs.rhs_nodes(2, 33))
    A = osg.assemble(pr.sys)
    Ustar = osg.solve_direct(A.T.tocsr(), F)
    U = np.zeros(pr.N)
    info = pr.h.solve(F, U, transpose=True, tol=1e-12)      # host numpy buffers: staged inside the call
    assert info.status == 0
    assert np.linalg.norm(U - Ustar) / np.linalg.norm(Ustar) <= 1e-8


def test_zero_rhs_and_maxit_status():
    import torch
    pr = Pair(33, 2, 2)
    U = torch.ones(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(torch.zeros(pr.N, dtype=torch.float64, device="cuda"), U)
    assert info.status == 0 and float(U.abs().max()) == 0.0
    F = dev(osg.rhs(pr.sys))
    info = pr.h.solve(F, U, maxit=2, tol=1e-14, check=False)
    assert info.status == -4 and info.iters == 2


def test_nonfinite_rhs_reported():
    import torch
    pr = Pair(9, 1, 1)
    F = osg.rhs(pr.sys)
    F[3] = np.nan
    U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(dev(F), U, check=False)
    assert info.status == -6


def test_switching_krylov_arithmetic_on_one_handle():
    """Double-float and FP64 solves alternate on one handle (they share the Krylov workspace,
    whose padding each layout needs zeroed): every solve converges to the same solution."""
    import torch
    pr = Pair(65, 3, 3, sigma=0.3)
    F = dev(osg.rhs(pr.sys))
    Ustar = _direct(pr, host(F))
    df = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=20, tol=1e-10, pc_prec=sg.F32, arith=sg.ARITH_DF64)
    f64 = dict(df, pc_prec=sg.F64, arith=sg.ARITH_F64)
    for opts in (df, f64, df, f64, df):
        U = torch.zeros_like(F)
        info = pr.h.solve(F, U, **opts)
        torch.cuda.synchronize()
        assert info.status == 0 and info.relres_true <= 1e-10
        got = host(U)
        assert np.linalg.norm(got - Ustar) <= 1e-6 * np.linalg.norm(Ustar)


@pytest.mark.parametrize("case", ["df", "f64", "df_noconv", "f64_noconv", "df_x0"])
def test_pinned_host_buffers_solve(case):
    """Page-locked host F and U give the device solve's answer, bit for bit: converged (the
    iterate is copied out while its true residual is checked), stopped at maxit (the early
    copies of earlier restarts are superseded), and from a given initial guess."""
    import torch
    pr = Pair(65, 2, 3, sigma=0.3)
    F = osg.rhs(pr.sys)
    opts = dict(method=sg.FGMRES, precond=sg.PC_BLOCKTRI, restart=5, tol=1e-10, pc_prec=sg.F32, arith=sg.ARITH_DF64)
    if case.startswith("f64"):
        opts.update(pc_prec=sg.F64, arith=sg.ARITH_F64, method=sg.GMRES)
    if case.endswith("noconv"):
        opts.update(maxit=12)
    x0 = inputs.uniform(5, pr.N) if case == "df_x0" else None
    if x0 is not None:
        opts.update(x0_given=1)
    Ud = torch.zeros(pr.N, dtype=torch.float64, device="cuda") if x0 is None else dev(x0)
    opts.update(check=False)
    info_d = pr.h.solve(dev(F), Ud, **opts)
    Fh = torch.as_tensor(F).pin_memory()
    Uh = (torch.full((pr.N,), 7.0, dtype=torch.float64) if x0 is None else torch.as_tensor(x0.copy())).pin_memory()
    info = pr.h.solve(Fh, Uh, **opts)
    torch.cuda.synchronize()
    assert info.status == info_d.status and info.iters == info_d.iters
    if case.endswith("noconv"):
        assert info.status == -4                                  # SG_E_NOCONV
    else:
        assert info.status == 0 and info.relres_true <= 1e-10
    assert np.array_equal(Uh.numpy(), host(Ud))


def test_df_fgmres_long_arnoldi_cycles():
    """Double-float FGMRES(30) without a preconditioner: Arnoldi cycles of more than 16 steps (the
    multi-dot and multi-axpy kernels at large basis sizes).  The solve must converge (A is SPD, so
    restarted GMRES does) and match the direct solution to kappa(A) x tol."""
    import torch
    pr = Pair(33, 2, 2, sigma=0.3)
    F = dev(osg.rhs(pr.sys))
    Ustar = _direct(pr, host(F))
    U = torch.zeros_like(F)
    info = pr.h.solve(F, U, method=sg.FGMRES, precond=sg.PC_NONE, restart=30, maxit=5000, tol=1e-10,
                      pc_prec=sg.F32, arith=sg.ARITH_DF64)
    torch.cuda.synchronize()
    assert info.status == 0 and info.relres_true <= 1e-10
    assert info.iters > 16
    assert np.linalg.norm(host(U) - Ustar) <= 1e-6 * np.linalg.norm(Ustar)


def test_exact_lower_block_preconditioner_matches_oracle():
    """The 2 x 2 block-triangular preconditioner with the exact degree-(p-1) block (Sec. 4.2,
    Theorem 1's form) against the oracle's (both inner solves to 1e-13), its transpose by the
    duality <B^{-1} x, y> = <x, B^{-T} y>, and FGMRES with it against the direct solution."""
    import torch
    pr = Pair(33, 2, 3, basis.LEGENDRE, sigma=0.3)           # P = 10, A_hat: degree 2 (6 blocks)
    R = inputs.uniform(71, pr.N)
    ref = precond.block_tri_exact_inv(pr.sys, pr.oracle_vsolver(), R, inner_tol=1e-13)
    Z = torch.empty(pr.N, dtype=torch.float64, device="cuda")
    pr.h.precond_blocktri_exact(dev(R), Z, inner_tol=1e-13)
    torch.cuda.synchronize()
    got = host(Z)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    Y = inputs.uniform(72, pr.N)
    ZT = torch.empty_like(Z)
    pr.h.precond_blocktri_exact(dev(Y), ZT, transpose=True, inner_tol=1e-13)
    torch.cuda.synchronize()
    lhs, rhs = float(np.dot(got, Y)), float(np.dot(R, host(ZT)))
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), 1e-300)
    F = osg.rhs(pr.sys)
    Ustar = osg.solve_direct(osg.assemble(pr.sys), F)
    U = torch.zeros(pr.N, dtype=torch.float64, device="cuda")
    info = pr.h.solve(dev(F), U, method=sg.FGMRES, precond=sg.PC_BLOCKTRI_EXACT, pc_prec=sg.F64, tol=1e-12,
                      restart=30, inner_tol=1e-13)
    assert info.status == 0 and info.relres_true <= 1e-12
    assert np.linalg.norm(host(U) - Ustar) <= 1e-8 * np.linalg.norm(Ustar)
    A = osg.assemble(pr.sys)
    solver = pr.oracle_vsolver()
    _, its_o, _ = krylov.gmres(lambda v: A @ v,
                               lambda r: precond.block_tri_exact_inv(pr.sys, solver, r, inner_tol=1e-13), F,
                               tol=1e-12, restart=30, flexible=True)
    assert abs(info.iters - its_o) <= 1
    its_flat = pr.h.solve(dev(F), torch.zeros_like(U), method=sg.FGMRES, precond=sg.PC_BLOCKTRI, pc_prec=sg.F64,
                          tol=1e-12, restart=30).iters
    assert info.iters <= its_flat                          # the exact lower block is the stronger preconditioner
