"""sg_vcycle_static, the allocation-free V-cycle, against sg_vcycle on the same inputs.

Both entry points launch the same level kernels, so the results agree to rounding (the
test allows 1e-13 relative for FP64 and the storage precision's unit roundoff
otherwise).  Two calls in a row with different right-hand sides check that the shared
array's leftover contents from the previous call do not leak into the next one, and the
device's free memory is unchanged across the second call (the first call on a device may
load the library's device code, which the runtime allocates itself)."""
import ctypes

import numpy as np
import pytest

from paper_1304_1755_gb300 import inputs, sg
from _gpu_util import Pair, dev, host

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-6, 2: 1e-2}


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
@pytest.mark.parametrize("n", [129, 33], ids=["n129", "n33"])
def test_static_vcycle_matches_vcycle_on_two_calls(n, prec):
    import torch
    L = sg.lib()
    pr = Pair(n, 2, 2)                                 # P = 6 blocks
    nb = pr.sys.P
    B1 = dev(inputs.uniform(41, nb * pr.sys.Nx))
    B2 = dev(inputs.uniform(42, nb * pr.sys.Nx) * 1e3)
    X1, X2, R1, R2 = (_out(pr, nb, prec) for _ in range(4))
    _call(L.sg_vcycle_static, pr, B1, X1, nb, prec)
    free_before = torch.cuda.mem_get_info()[0]
    _call(L.sg_vcycle_static, pr, B2, X2, nb, prec)
    assert torch.cuda.mem_get_info()[0] == free_before
    _call(L.sg_vcycle, pr, B1, R1, nb, prec)
    _call(L.sg_vcycle, pr, B2, R2, nb, prec)
    got1, got2, ref1, ref2 = (host(t) for t in (X1, X2, R1, R2))
    for got, ref in ((got1, ref1), (got2, ref2)):
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


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
