"""sg_vcycle_static, the allocation-free V-cycle, against sg_vcycle and against the oracle.

Both entry points launch the same level kernels with the same arithmetic; only where the coarse
levels live differs (the handle's workspace or the library's static array), so the results
must be bit-identical.  They must also match the oracle's V-cycle within the storage
precision's tolerance (the bar of the V-cycle parity tests).  Two calls in a row with different
right-hand sides check that the shared array's leftover contents from the previous call do not
leak into the next one, and the device's free memory is unchanged across the second call (the
first call on a device may load the library's device code, which the runtime allocates
itself).  At 513^2 the tile kernels run with several tiles per level row."""
import ctypes

import numpy as np
import pytest

from paper_1304_1755_gb300 import inputs, sg
from _gpu_util import Pair, dev, host

pytestmark = pytest.mark.gpu

def _oracle_ok(got, ref, prec):
    """The V-cycle parity bar: FP64 1e-11 and FP32 1e-4 of max |ref| elementwise, BF16 3e-2 in norm."""
    if prec == 0:
        return np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    if prec == 1:
        return np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    return np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref)


def _call(fn, pr, B, X, nb, prec):
    import torch
    rc = fn(pr.h.h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), nb, prec)
    assert rc == 0, sg.lib().sg_last_error(pr.h.h)
    torch.cuda.synchronize()


def _out(pr, nb, prec):
    import torch
    dt = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[prec]
    return torch.full((nb * pr.sys.Nx,), float("nan"), dtype=dt, device="cuda")


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["f64", "f32", "bf16"])
@pytest.mark.parametrize("n,nb", [(129, 6), (33, 6), (513, 4)], ids=["n129", "n33", "n513"])
def test_static_vcycle_matches_vcycle_on_two_calls(n, nb, prec):
    import torch
    L = sg.lib()
    pr = Pair(n, 2, 2)                                 # P = 6 blocks of workspace
    B1h = inputs.uniform(41, (nb, pr.sys.Nx))
    B2h = inputs.uniform(42, (nb, pr.sys.Nx)) * 1e3
    B1, B2 = dev(B1h.reshape(-1)), dev(B2h.reshape(-1))
    X1, X2, R1, R2 = (_out(pr, nb, prec) for _ in range(4))
    _call(L.sg_vcycle_static, pr, B1, X1, nb, prec)
    free_before = torch.cuda.mem_get_info()[0]
    _call(L.sg_vcycle_static, pr, B2, X2, nb, prec)
    assert torch.cuda.mem_get_info()[0] == free_before
    _call(L.sg_vcycle, pr, B1, R1, nb, prec)
    _call(L.sg_vcycle, pr, B2, R2, nb, prec)
    assert torch.equal(X1, R1) and torch.equal(X2, R2)
    for X, Bh in ((X1, B1h), (X2, B2h)):
        got = host(X).reshape(nb, -1)
        assert np.isfinite(got).all()
        assert _oracle_ok(got, pr.hier.vcycle(Bh.T).T, prec)


def test_static_vcycle_rejects_oversize_request():
    import torch
    n, M, p = 513, 4, 3                                # P = 35; FP64 needs ~48 MB of level storage
    coef, _ = sg.sg_kl_coef(n, M, 0.3)
    h = sg.Handle(n, M, p, 0, coef, stream=torch.cuda.current_stream())
    N = h.P * h.Nx
    B = torch.zeros(N, dtype=torch.float64, device="cuda")
    X = torch.full((N,), 7.0, dtype=torch.float64, device="cuda")
    rc = sg.lib().sg_vcycle_static(h.h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()), h.P, 0)
    assert rc == -1
    msg = sg.lib().sg_last_error(h.h).decode()
    assert "bytes of scratch" in msg and "33554432" in msg
    torch.cuda.synchronize()
    assert bool((X == 7.0).all())                      # nothing was launched
    # BF16 storage fits: 35 blocks x ~86k level nodes x 2 bytes x 2 arrays
    Xb = torch.empty(N, dtype=torch.bfloat16, device="cuda")
    rc = sg.lib().sg_vcycle_static(h.h, ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(Xb.data_ptr()), h.P, 2)
    assert rc == 0
    torch.cuda.synchronize()
    assert bool((Xb == 0).all())                       # zero right-hand side gives zero
    h.close()
