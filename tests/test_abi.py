"""The C-ABI library loads, exports every function include/sg.h declares, and the
Python binding covers them (CPU only: no device calls).  Also checks the host KL
helper of the library against the oracle (pure host code)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sg.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1304_1755_gb300 import build, sg
    if not os.path.exists(sg.LIB_PATH):
        build.build()
    return sg.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sg_setup", "sg_apply", "sg_precond_blocktri", "sg_precond_blockdiag", "sg_solve"):
        assert required in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    from paper_1304_1755_gb300 import sg
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in sg.SIGNATURES, name


def test_null_arguments_rejected_without_device(lib):
    from paper_1304_1755_gb300 import sg
    import ctypes
    h = ctypes.c_void_p()
    assert lib.sg_setup(None, None, ctypes.byref(h)) == -1
    assert b"null" in lib.sg_last_error(None)
    coef = np.ones((1, 16))
    prob = sg.Problem(6, 0, 0, 0, coef.ctypes.data_as(sg.DP), 1, 1, 0.0)   # n = 6 is not 2^L + 1
    assert lib.sg_setup(ctypes.byref(prob), None, ctypes.byref(h)) == -1


def test_every_entry_point_rejects_a_null_handle_without_device(lib):
    """Every call that takes a handle returns SG_E_ARG for a null one (and sg_destroy ignores it),
    before touching the device."""
    from paper_1304_1755_gb300 import sg
    import ctypes
    D, I = ctypes.c_double(), ctypes.c_int()
    o = sg.SolveOpts(sg.FGMRES, sg.PC_BLOCKTRI, 30, 100, 1e-8, sg.F32, 0, 0, 0, 0)
    info = sg.SolveInfo()
    ms, ln = (ctypes.c_double * 4)(), (ctypes.c_long * 4)()
    calls = [
        lambda: lib.sg_set_stream(None, None),
        lambda: lib.sg_sizes(None, ctypes.byref(I), ctypes.byref(I), ctypes.byref(I)),
        lambda: lib.sg_basis(None, None),
        lambda: lib.sg_apply(None, None, None, 0),
        lambda: lib.sg_residual(None, None, None, None),
        lambda: lib.sg_precond_blocktri(None, None, None, 0, 0),
        lambda: lib.sg_precond_blockdiag(None, None, None, 0),
        lambda: lib.sg_precond_blocksym(None, None, None, 0),
        lambda: lib.sg_vcycle(None, None, None, 1, 0),
        lambda: lib.sg_vcycle_static(None, None, None, 1, 0),
        lambda: lib.sg_solve(None, None, None, ctypes.byref(o), ctypes.byref(info)),
        lambda: lib.sg_autotune(None, 0),
        lambda: lib.sg_objective(None, None, ctypes.byref(D), None),
        lambda: lib.sg_adjoint_gradients(None, None, None, 0.1, None, ctypes.byref(D)),
        lambda: lib.sg_timing_enable(None, 1),
        lambda: lib.sg_timing_read(None, ms, ln),
        lambda: lib.sg_rhs(None, None, None),
        lambda: lib.sg_precond_blocktri_exact(None, None, None, 0, 0.0),
        lambda: lib.sg_solve_batch_graph(None, None, None, 1, ctypes.byref(o), None),
        lambda: lib.sg_batch_create(None, None, None, 1, ctypes.byref(o), ctypes.byref(ctypes.c_void_p())),
        lambda: lib.sg_batch_solve(None, None),
    ]
    for call in calls:
        assert call() == -1
    lib.sg_destroy(None)
    lib.sg_batch_destroy(None)


def test_batch_rejects_a_repeated_handle_without_device(lib):
    """A handle listed twice is rejected before anything is read through it (the addresses below are
    never dereferenced)."""
    from paper_1304_1755_gb300 import sg
    import ctypes
    fake = ctypes.c_void_p(0x1000)
    hs = (sg.VP * 2)(fake, fake)
    vecs = (sg.VP * 2)(ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000))
    o = sg.SolveOpts(sg.FGMRES, sg.PC_BLOCKTRI, 30, 100, 1e-8, sg.F32, 0, 0, 0, 0)
    assert lib.sg_solve_batch(hs, vecs, vecs, 2, ctypes.byref(o), None, 2) == -1


@pytest.mark.parametrize("n,M,sigma", [(9, 2, 0.3), (33, 4, 0.5), (17, 6, 0.2)])
def test_library_kl_helper_matches_oracle(lib, n, M, sigma):
    from oracle import kl
    from paper_1304_1755_gb300 import sg
    coef, lam = sg.sg_kl_coef(n, M, sigma)
    ref = kl.kl_coefficients(n, M, sigma)
    assert np.allclose(coef, ref, rtol=0, atol=1e-13)
    assert np.allclose(lam, kl.kl_eigenvalues(M), rtol=1e-13)
    ab = np.linspace(0.5, 1.5, (n - 1) ** 2)
    coef2, _ = sg.sg_kl_coef(n, M, sigma, abar=ab)
    assert np.array_equal(coef2[0], ab)


@pytest.mark.parametrize("n,M,sigma", [(9, 2, 0.3), (33, 4, 0.5), (65, 6, 0.2), (5, 0, 0.1)])
def test_library_triangle_kl_helper_matches_oracle(lib, n, M, sigma):
    """sg_kl_coef_p1 (host): the per-triangle coefficients at the centroids, the oracle's."""
    from oracle import kl, p1
    from paper_1304_1755_gb300 import sg
    coef, lam = sg.sg_kl_coef_p1(n, M, sigma)
    assert coef.shape == (M + 1, 2 * (n - 1) ** 2)
    assert np.allclose(coef, p1.triangle_coefficients(n, M, sigma), rtol=0, atol=1e-14)
    assert np.allclose(lam, kl.kl_eigenvalues(M), rtol=1e-13)


@pytest.mark.parametrize("n,M,sigma,xi", [(9, 2, 0.3, 3 ** 0.5), (33, 4, 0.5, 3 ** 0.5), (17, 6, 0.2, 2.5)])
def test_library_coercivity_helper_matches_oracle(lib, n, M, sigma, xi):
    """sg_min_coef (host) against the oracle's corner minimum, itself pinned by enumeration."""
    from oracle import kl
    from paper_1304_1755_gb300 import sg
    coef = kl.kl_coefficients(n, M, sigma, abar=np.linspace(0.6, 1.4, (n - 1) ** 2))
    assert sg.sg_min_coef(coef, n, M, xi) == pytest.approx(kl.min_coefficient_at_corners(coef, xi), abs=1e-15)
