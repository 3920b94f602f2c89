"""GPU parity: K1 (SG operator), the multigrid V-cycle and the block preconditioners
against the oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic):
  * FP64 operator: every output is a short sum of products of the coefficients
    and feature differences of X; the error is below ~50 ulp of the absolute
    sum, so |Y - Y*| <= 2e-13 (|A| |X|) elementwise.
  * FP32 arithmetic: the same bound with eps_32: 2e-5 (|A| |X|).
  * BF16 storage of the output: plus 2^-8 |Y*| (round to nearest of the store).
  * V-cycle / preconditioners (linear maps with O(1) amplification):
    FP64 1e-11, FP32 1e-4 relative to max |Z*|; BF16 storage 3e-2 in the norm.
"""
import numpy as np
import pytest

from oracle import basis, precond, sg as osg
from paper_1304_1755_gb300 import inputs
from _gpu_util import Pair, dev, host, pair

pytestmark = pytest.mark.gpu

SHAPES = [  # n, M, p, family, mean
    (3, 1, 1, basis.LEGENDRE, "one"),
    (5, 1, 0, basis.LEGENDRE, "one"),
    (9, 2, 3, basis.HERMITE, "random"),
    (33, 2, 2, basis.LEGENDRE, "one"),          # C1 shape
    (65, 3, 3, basis.HERMITE, "lognormal"),
    (129, 4, 2, basis.LEGENDRE, "one"),
]


def _abs_apply(pr, X):
    if "absA" not in pr.memo:
        pr.memo["absA"] = abs(osg.assemble(pr.sys))
    return pr.memo["absA"] @ np.abs(X)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[0]}M{s[1]}p{s[2]}f{s[3]}{s[4]}")
def test_apply_fp64(shape):
    import torch
    n, M, p, fam, mean = shape
    pr = pair(n, M, p, fam, mean=mean)
    X = inputs.uniform(11, pr.N)
    ref = osg.apply(pr.sys, X)
    Y = torch.empty(pr.N, dtype=torch.float64, device="cuda")
    pr.h.apply(dev(X), Y)
    torch.cuda.synchronize()
    bound = 2e-13 * _abs_apply(pr, X) + 1e-300
    assert np.all(np.abs(host(Y) - ref) <= bound)


# FP32 arithmetic runs two cells per lane in warps of 62-cell columns: 129 and 257 have several
# warp columns with seams and a ragged last one
@pytest.mark.parametrize("shape", SHAPES[2:] + [(257, 2, 1, basis.LEGENDRE, "lognormal")],
                         ids=lambda s: f"n{s[0]}M{s[1]}p{s[2]}")
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "bf16"])
def test_apply_low_precision(shape, prec):
    import torch
    n, M, p, fam, mean = shape
    pr = pair(n, M, p, fam, mean=mean)
    dt = torch.float32 if prec == 1 else torch.bfloat16
    Xd = dev(inputs.uniform(12, pr.N), dt)
    X = host(Xd)                          # the exactly representable input both sides use
    ref = osg.apply(pr.sys, X)
    Y = torch.empty(pr.N, dtype=dt, device="cuda")
    pr.h.apply(Xd, Y, prec)
    torch.cuda.synchronize()
    bound = 2e-5 * _abs_apply(pr, X) + (2.0 ** -8 * np.abs(ref) if prec == 2 else 0) + 1e-30
    assert np.all(np.abs(host(Y) - ref) <= bound)


def _to_df(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return np.concatenate([hi, lo]), hi.astype(np.float64) + lo.astype(np.float64)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s[0]}M{s[1]}p{s[2]}f{s[3]}{s[4]}")
def test_apply_double_float(shape):
    """Double-float operator (FP32 pairs): the input is the df split of an FP64 vector; the result
    hi + lo must match the FP64 oracle to 2e-13 (|A| |X|) (the df significand is 48 bits)."""
    import torch
    n, M, p, fam, mean = shape
    pr = pair(n, M, p, fam, mean=mean)
    xdf, X = _to_df(inputs.uniform(14, pr.N))
    ref = osg.apply(pr.sys, X)
    Y = torch.empty(2 * pr.N, dtype=torch.float32, device="cuda")
    pr.h.apply(dev(xdf), Y, 3)
    torch.cuda.synchronize()
    y = Y.cpu().numpy().astype(np.float64)
    got = y[:pr.N] + y[pr.N:]
    assert np.all(np.abs(got - ref) <= 2e-13 * _abs_apply(pr, X) + 1e-300)


def test_residual_fp64():
    import torch
    pr = Pair(33, 2, 2)
    U = inputs.uniform(13, pr.N)
    F = osg.rhs(pr.sys)
    R = torch.empty(pr.N, dtype=torch.float64, device="cuda")
    pr.h.residual(dev(F), dev(U), R)
    torch.cuda.synchronize()
    ref = F - osg.apply(pr.sys, U)
    assert np.all(np.abs(host(R) - ref) <= 2e-13 * (_abs_apply(pr, U) + np.abs(F)))


# (257 | 513, "one", (1, 1)): the constant-mean V(1,1) tile kernels with several tiles per level row
# (x seams at 64 coarse / 128 fine columns and ragged last tiles), the path of every large solve
MG_SHAPES = [(3, "one", (1, 1)), (5, "one", (1, 1)), (9, "random", (1, 1)), (33, "one", (1, 1)),
             (65, "lognormal", (1, 1)), (129, "one", (1, 1)), (129, "lognormal", (2, 2)), (257, "one", (2, 1)),
             (257, "one", (1, 1)), (513, "one", (1, 1)), (257, "lognormal", (1, 1))]


@pytest.mark.parametrize("n,mean,nu", MG_SHAPES, ids=lambda v: str(v))
@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "f32", "bf16"])
def test_vcycle(n, mean, nu, prec):
    import torch
    pr = pair(n, 1, 2, mean=mean, nu=nu)      # P = 3 blocks of workspace
    nb = 3
    B = inputs.uniform(21, (nb, pr.sys.Nx))
    if "vcycle" not in pr.memo:
        pr.memo["vcycle"] = pr.hier.vcycle(B.T).T
    ref = pr.memo["vcycle"]
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[prec]
    X = torch.empty(nb * pr.sys.Nx, dtype=dt, device="cuda")
    pr.h.vcycle(dev(B.reshape(-1)), X, nb, prec)
    torch.cuda.synchronize()
    got = host(X).reshape(nb, -1)
    scale = np.abs(ref).max()
    if prec == 0:
        assert np.abs(got - ref).max() <= 1e-11 * scale
    elif prec == 1:
        assert np.abs(got - ref).max() <= 1e-4 * scale
    else:
        assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [0, 2], ids=["f64", "bf16"])
def test_preconditioner_graph_replay_matches_direct(prec):
    """On a non-default stream each preconditioner application is captured once as a CUDA graph
    and replayed; results must be bit-identical to direct launches on the default stream."""
    import torch
    from paper_1304_1755_gb300 import sg
    pr = Pair(129, 3, 3, basis.LEGENDRE)
    R = dev(inputs.uniform(41, pr.N))
    dt = torch.float64 if prec == 0 else torch.bfloat16
    Z0 = torch.empty(pr.N, dtype=dt, device="cuda")
    pr.h.precond_blocktri(R, Z0, prec)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        h2 = sg.Handle(129, 3, 3, basis.LEGENDRE, pr.coef, stream=s)
        Z = torch.empty(pr.N, dtype=dt, device="cuda")
        for _ in range(3):                      # first call captures, the others replay
            Z.zero_()
            h2.precond_blocktri(R, Z, prec)
            s.synchronize()
            assert torch.equal(Z, Z0)
        Zd = torch.empty(pr.N, dtype=dt, device="cuda")
        h2.precond_blockdiag(R, Zd, prec)
    s.synchronize()
    Zd0 = torch.empty(pr.N, dtype=dt, device="cuda")
    pr.h.precond_blockdiag(R, Zd0, prec)
    torch.cuda.synchronize()
    assert torch.equal(Zd, Zd0)
    h2.close()


PC_SHAPES = [(9, 2, 3, basis.LEGENDRE, "one"), (33, 2, 2, basis.LEGENDRE, "one"),
             (65, 3, 2, basis.HERMITE, "lognormal"), (129, 2, 3, basis.LEGENDRE, "one"),
             (257, 2, 2, basis.LEGENDRE, "one"), (513, 1, 2, basis.HERMITE, "one")]


@pytest.mark.parametrize("shape", PC_SHAPES, ids=lambda s: f"n{s[0]}M{s[1]}p{s[2]}{s[4]}")
@pytest.mark.parametrize("kind", ["tri", "tri_T", "diag", "sym"])
@pytest.mark.parametrize("prec", [0, 1, 2, 4], ids=["f64", "f32", "bf16", "bf16z"])
def test_preconditioners(shape, kind, prec):
    import torch
    n, M, p, fam, mean = shape
    pr = pair(n, M, p, fam, mean=mean)
    R = inputs.uniform(31, pr.N)
    if ("pc", kind) not in pr.memo:
        solver = pr.oracle_vsolver()
        if kind == "diag":
            ref = precond.block_diag_inv(pr.sys, solver, R)
        elif kind == "sym":
            ref = precond.block_sym_inv(pr.sys, solver, R)
        else:
            ref = precond.block_tri_inv(pr.sys, solver, R, transpose=(kind == "tri_T"))
        pr.memo[("pc", kind)] = ref
    ref = pr.memo[("pc", kind)]
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16, 4: torch.float32}[prec]
    Z = torch.empty(pr.N, dtype=dt, device="cuda")
    if kind == "diag":
        pr.h.precond_blockdiag(dev(R), Z, prec)
    elif kind == "sym":
        pr.h.precond_blocksym(dev(R), Z, prec)
    else:
        pr.h.precond_blocktri(dev(R), Z, prec, transpose=(kind == "tri_T"))
    torch.cuda.synchronize()
    got = host(Z)
    scale = np.abs(ref).max()
    if prec == 0:
        assert np.abs(got - ref).max() <= 1e-11 * scale
    elif prec == 1:
        assert np.abs(got - ref).max() <= 1e-4 * scale
    else:
        assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref)
