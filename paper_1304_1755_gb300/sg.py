"""Thin ctypes binding of ``libsg.so`` (declared in ``include/sg.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Functions take raw pointers (ints) or torch tensors (their
``data_ptr()``) and return the library's status codes as exceptions.  The
library must have been built (``paper_1304_1755_gb300.build``); a missing
library raises ``OSError`` -- there is no fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")

F64, F32, BF16, DF64, BF16Z = 0, 1, 2, 3, 4   # BF16Z: BF16 preconditioner storage, FP32 output
ARITH_F64, ARITH_DF64, ARITH_F64_DFOP = 0, 1, 2   # see sg_arith in include/sg.h
LEGENDRE, HERMITE = 0, 1
Q1, P1 = 0, 1                                   # sg_elements
GS_LEX, GS_RB = 0, 1                            # sg_gs_order (P1 smoother)
GMRES, FGMRES, GPCG, PCG, BGS = 0, 1, 2, 3, 4
PC_NONE, PC_BLOCKTRI, PC_BLOCKDIAG, PC_BLOCKSYM, PC_BLOCKTRI_EXACT, PC_BLOCKSYM_REC = 0, 1, 2, 3, 4, 5

STATUS = {0: "SG_OK", -1: "SG_E_ARG", -2: "SG_E_ALLOC", -3: "SG_E_CUDA", -4: "SG_E_NOCONV",
          -5: "SG_E_BREAKDOWN", -6: "SG_E_NONFINITE", -7: "SG_E_TIMEOUT", -8: "SG_E_STATE"}


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("M", ctypes.c_int), ("p", ctypes.c_int), ("family", ctypes.c_int),
                ("coef", ctypes.POINTER(ctypes.c_double)), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("elements", ctypes.c_int), ("gs_order", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("precond", ctypes.c_int), ("restart", ctypes.c_int),
                ("maxit", ctypes.c_int), ("tol", ctypes.c_double), ("pc_prec", ctypes.c_int),
                ("transpose", ctypes.c_int), ("x0_given", ctypes.c_int), ("reorth", ctypes.c_int),
                ("arith", ctypes.c_int), ("inner_tol", ctypes.c_double), ("inner_restart", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
                ("relres_est", ctypes.c_double), ("relres_true", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("n_apply", ctypes.c_int), ("n_precond", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
VP, DP, IP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
# exported name -> (restype, argtypes)
SIGNATURES = {
    "sg_kl_coef": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, VP, VP, VP]),
    "sg_kl_coef_p1": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, VP, VP]),
    "sg_min_coef": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, VP, ctypes.c_double, DP]),
    "sg_setup": (ctypes.c_int, [ctypes.POINTER(Problem), VP, ctypes.POINTER(VP)]),
    "sg_rhs": (ctypes.c_int, [VP, VP, VP]),
    "sg_destroy": (None, [VP]),
    "sg_set_stream": (ctypes.c_int, [VP, VP]),
    "sg_last_error": (ctypes.c_char_p, [VP]),
    "sg_sizes": (ctypes.c_int, [VP, IP, IP, IP]),
    "sg_basis": (ctypes.c_int, [VP, VP]),
    "sg_apply": (ctypes.c_int, [VP, VP, VP, ctypes.c_int]),
    "sg_residual": (ctypes.c_int, [VP, VP, VP, VP]),
    "sg_precond_blocktri": (ctypes.c_int, [VP, VP, VP, ctypes.c_int, ctypes.c_int]),
    "sg_precond_blockdiag": (ctypes.c_int, [VP, VP, VP, ctypes.c_int]),
    "sg_precond_blocksym": (ctypes.c_int, [VP, VP, VP, ctypes.c_int]),
    "sg_precond_blocksym_rec": (ctypes.c_int, [VP, VP, VP]),
    "sg_precond_blocktri_exact": (ctypes.c_int, [VP, VP, VP, ctypes.c_int, ctypes.c_double]),
    "sg_vcycle": (ctypes.c_int, [VP, VP, VP, ctypes.c_int, ctypes.c_int]),
    "sg_vcycle_static": (ctypes.c_int, [VP, VP, VP, ctypes.c_int, ctypes.c_int]),
    "sg_solve": (ctypes.c_int, [VP, VP, VP, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]),
    "sg_solve_batch": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.c_int,
                                      ctypes.POINTER(SolveOpts), VP, ctypes.c_int]),
    "sg_solve_batch_graph": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.c_int,
                                            ctypes.POINTER(SolveOpts), VP]),
    "sg_batch_create": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.c_int,
                                       ctypes.POINTER(SolveOpts), ctypes.POINTER(VP)]),
    "sg_batch_solve": (ctypes.c_int, [VP, VP]),
    "sg_batch_destroy": (None, [VP]),
    "sg_autotune": (ctypes.c_int, [VP, ctypes.c_int]),
    "sg_objective": (ctypes.c_int, [VP, VP, DP, VP]),
    "sg_adjoint_gradients": (ctypes.c_int, [VP, VP, VP, ctypes.c_double, VP, DP]),
    "sg_timing_enable": (ctypes.c_int, [VP, ctypes.c_int]),
    "sg_timing_read": (ctypes.c_int, [VP, DP, ctypes.POINTER(ctypes.c_longlong)]),
}


def lib():
    """Load libsg.so once (raises OSError when it has not been built)."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


def _check(rc, h=None):
    if rc != 0:
        msg = lib().sg_last_error(h)
        raise SGError(rc, msg.decode() if msg else "")
    return rc


def sg_kl_coef(n, M, sigma, corr_len=1.0, abar=None):
    """Host KL helper: returns ((M+1, (n-1)^2) coefficients, lambda[M]) as numpy arrays."""
    import numpy as np
    coef = np.zeros((M + 1, (n - 1) ** 2))
    lam = np.zeros(max(M, 1))
    ab = None if abar is None else np.ascontiguousarray(abar, dtype=np.float64)
    _check(lib().sg_kl_coef(n, M, sigma, corr_len, _ptr(ab), _ptr(coef), _ptr(lam)))
    return coef, lam[:M]


def sg_kl_coef_p1(n, M, sigma, corr_len=1.0):
    """Host KL helper for P1 elements: ((M+1, 2 (n-1)^2) per-triangle coefficients, lambda[M])."""
    import numpy as np
    coef = np.zeros((M + 1, 2 * (n - 1) ** 2))
    lam = np.zeros(max(M, 1))
    _check(lib().sg_kl_coef_p1(n, M, sigma, corr_len, _ptr(coef), _ptr(lam)))
    return coef, lam[:M]


def sg_min_coef(coef, n, M, xi_max=3.0 ** 0.5):
    """Host coercivity check: min over cells and over the box |xi_k| <= xi_max of a(x_e, xi)."""
    import numpy as np
    c = np.ascontiguousarray(coef, dtype=np.float64)
    assert c.shape == (M + 1, (n - 1) ** 2)
    out = ctypes.c_double()
    _check(lib().sg_min_coef(n, M, _ptr(c), xi_max, ctypes.byref(out)))
    return out.value


class Handle:
    """Owns one sg_handle.  Pointer arguments: torch tensors, numpy arrays or ints."""

    def __init__(self, n, M, p, family, coef, nu1=1, nu2=1, omega=0.0, stream=None, elements=0, gs_order=0):
        import numpy as np
        self._coef = np.ascontiguousarray(coef, dtype=np.float64)
        assert self._coef.shape == (M + 1, (2 if elements == P1 else 1) * (n - 1) ** 2)
        prob = Problem(n, M, p, family, self._coef.ctypes.data_as(DP), nu1, nu2, omega, elements, gs_order)
        h = VP()
        s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib().sg_setup(ctypes.byref(prob), s, ctypes.byref(h)))
        self.h = h
        Nx, P, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().sg_sizes(h, ctypes.byref(Nx), ctypes.byref(P), ctypes.byref(nl)), h)
        self.n, self.M, self.p, self.family = n, M, p, family
        self.Nx, self.P, self.nlevels = Nx.value, P.value, nl.value

    def close(self):
        if getattr(self, "h", None):
            lib().sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib().sg_set_stream(self.h, s), self.h)

    def basis(self):
        import numpy as np
        a = np.zeros((self.P, max(self.M, 1)), dtype=np.int32)
        _check(lib().sg_basis(self.h, _ptr(a)), self.h)
        return a[:, :self.M]

    def rhs(self, F, f_nodes=None):
        """sg_rhs: F = e_0 (x) h^2 f (device FP64; f_nodes device FP64 N_x values or None for f = 1)."""
        _check(lib().sg_rhs(self.h, _ptr(f_nodes), _ptr(F)), self.h)

    def apply(self, X, Y, prec=F64):
        _check(lib().sg_apply(self.h, _ptr(X), _ptr(Y), prec), self.h)

    def residual(self, F, U, R):
        _check(lib().sg_residual(self.h, _ptr(F), _ptr(U), _ptr(R)), self.h)

    def precond_blocktri(self, R, Z, prec=F64, transpose=False):
        _check(lib().sg_precond_blocktri(self.h, _ptr(R), _ptr(Z), prec, int(transpose)), self.h)

    def precond_blockdiag(self, R, Z, prec=F64):
        _check(lib().sg_precond_blockdiag(self.h, _ptr(R), _ptr(Z), prec), self.h)

    def precond_blocktri_exact(self, R, Z, transpose=False, inner_tol=1e-12, check=True):
        """sg_precond_blocktri_exact: the 2 x 2 form with the exact lower-degree block (FP64)."""
        rc = lib().sg_precond_blocktri_exact(self.h, _ptr(R), _ptr(Z), int(transpose), inner_tol)
        if check:
            _check(rc, self.h)
        return rc

    def precond_blocksym(self, R, Z, prec=F64):
        _check(lib().sg_precond_blocksym(self.h, _ptr(R), _ptr(Z), prec), self.h)

    def precond_blocksym_rec(self, R, Z):
        """sg_precond_blocksym_rec: the recursive 2 x 2 symmetric block preconditioner (FP64)."""
        _check(lib().sg_precond_blocksym_rec(self.h, _ptr(R), _ptr(Z)), self.h)

    def vcycle(self, B, X, nblocks, prec=F64):
        _check(lib().sg_vcycle(self.h, _ptr(B), _ptr(X), nblocks, prec), self.h)

    def vcycle_static(self, B, X, nblocks, prec=F64):
        """sg_vcycle_static: the same cycle with no device allocation (coarse levels in a
        fixed 32 MiB array shared by every caller in the process; calls must not overlap)."""
        _check(lib().sg_vcycle_static(self.h, _ptr(B), _ptr(X), nblocks, prec), self.h)

    def solve(self, F, U, method=FGMRES, precond=PC_BLOCKTRI, restart=30, maxit=500, tol=1e-8, pc_prec=F64,
              transpose=False, x0_given=False, reorth=0, arith=ARITH_F64, check=True, inner_tol=0.0, inner_restart=0):
        o = SolveOpts(method, precond, restart, maxit, tol, pc_prec, int(transpose), int(x0_given), reorth, arith,
                      inner_tol, inner_restart)
        info = SolveInfo()
        rc = lib().sg_solve(self.h, _ptr(F), _ptr(U), ctypes.byref(o), ctypes.byref(info))
        if check and rc not in (0,):
            _check(rc, self.h)
        return info

    def autotune(self, which=0):
        """sg_autotune: time the operator kernel's tile candidates for this problem and keep the best."""
        _check(lib().sg_autotune(self.h, which), self.h)

    def objective(self, U, G=None):
        J = ctypes.c_double()
        _check(lib().sg_objective(self.h, _ptr(U), ctypes.byref(J), _ptr(G)), self.h)
        return J.value

    def timing_enable(self, on=True):
        _check(lib().sg_timing_enable(self.h, int(on)), self.h)

    def timing_read(self):
        """(ms[4], launches[4]) per phase: operator, preconditioner, Gram-Schmidt, other."""
        ms = (ctypes.c_double * 4)()
        ln = (ctypes.c_longlong * 4)()
        _check(lib().sg_timing_read(self.h, ms, ln), self.h)
        return list(ms), list(ln)

    def adjoint_gradients(self, U, Lam, sigma, g_abar):
        gs = ctypes.c_double()
        _check(lib().sg_adjoint_gradients(self.h, _ptr(U), _ptr(Lam), sigma, _ptr(g_abar), ctypes.byref(gs)), self.h)
        return gs.value


def solve_batch(handles, Fs, Us, nstreams=8, method=FGMRES, precond=PC_BLOCKTRI, restart=30, maxit=500, tol=1e-8,
                pc_prec=F64, transpose=False, reorth=0, arith=ARITH_F64, check=True):
    """sg_solve_batch: solve independent systems (one Handle each) concurrently on nstreams
    streams; returns one SolveInfo per system (status = that system's sg_solve result)."""
    n = len(handles)
    if len(Fs) != n or len(Us) != n:
        raise ValueError("handles, Fs and Us must have the same length")
    o = SolveOpts(method, precond, restart, maxit, tol, pc_prec, int(transpose), 0, reorth, arith, 0.0, 0)
    hs = (VP * n)(*[h.h for h in handles])
    fp = (VP * n)(*[_ptr(F) for F in Fs])
    up = (VP * n)(*[_ptr(U) for U in Us])
    infos = (SolveInfo * n)()
    rc = lib().sg_solve_batch(hs, fp, up, n, ctypes.byref(o), ctypes.cast(infos, VP), nstreams)
    if check and rc != 0:
        bad = [i for i in range(n) if infos[i].status != 0]
        raise SGError(rc, f"sg_solve_batch: systems {bad} failed" + (
            f": {lib().sg_last_error(handles[bad[0]].h).decode()}" if bad else ""))
    return list(infos)


def solve_batch_graph(handles, Fs, Us, method=FGMRES, precond=PC_BLOCKTRI, restart=30, maxit=500, tol=1e-8,
                      pc_prec=F64, transpose=False, arith=ARITH_F64, reorth=0, check=True):
    """sg_solve_batch_graph: the batch solved in one CUDA graph (device-side Arnoldi control, one launch
    per restart cycle of all systems); returns one SolveInfo per system."""
    n = len(handles)
    if len(Fs) != n or len(Us) != n:
        raise ValueError("handles, Fs and Us must have the same length")
    o = SolveOpts(method, precond, restart, maxit, tol, pc_prec, int(transpose), 0, reorth, arith, 0.0, 0)
    hs = (VP * n)(*[h.h for h in handles])
    fp = (VP * n)(*[_ptr(F) for F in Fs])
    up = (VP * n)(*[_ptr(U) for U in Us])
    infos = (SolveInfo * n)()
    rc = lib().sg_solve_batch_graph(hs, fp, up, n, ctypes.byref(o), ctypes.cast(infos, VP))
    if check and rc != 0:
        bad = [i for i in range(n) if infos[i].status != 0]
        raise SGError(rc, f"sg_solve_batch_graph: systems {bad} failed" + (
            f": {lib().sg_last_error(handles[bad[0] if bad else 0].h).decode()}"))
    return list(infos)


class Batch:
    """sg_batch_create / sg_batch_solve / sg_batch_destroy: a batch whose CUDA graphs are built once and
    launched for every solve (the handles, F and U fixed at creation)."""

    def __init__(self, handles, Fs, Us, method=FGMRES, precond=PC_BLOCKTRI, restart=30, maxit=500, tol=1e-8,
                 pc_prec=F64, transpose=False, arith=ARITH_F64, reorth=0):
        n = len(handles)
        if len(Fs) != n or len(Us) != n:
            raise ValueError("handles, Fs and Us must have the same length")
        self.handles, self.n = handles, n
        self._keep = (Fs, Us)
        o = SolveOpts(method, precond, restart, maxit, tol, pc_prec, int(transpose), 0, reorth, arith, 0.0, 0)
        hs = (VP * n)(*[h.h for h in handles])
        fp = (VP * n)(*[_ptr(F) for F in Fs])
        up = (VP * n)(*[_ptr(U) for U in Us])
        b = VP()
        _check(lib().sg_batch_create(hs, fp, up, n, ctypes.byref(o), ctypes.byref(b)), handles[0].h)
        self.b = b

    def solve(self, check=True):
        infos = (SolveInfo * self.n)()
        rc = lib().sg_batch_solve(self.b, ctypes.cast(infos, VP))
        if check and rc != 0:
            raise SGError(rc, lib().sg_last_error(self.handles[0].h).decode())
        return list(infos)

    def close(self):
        if getattr(self, "b", None):
            lib().sg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
