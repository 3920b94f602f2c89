"""The oracle's block-triangular flexible GMRES in plain C with OpenMP (``csolve.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Used by the tests and by the CPU-baseline
leg of ``bench.py``; the CUDA library never loads it.

The C code runs the steps of ``krylov.gmres(flexible=True)`` with ``precond.block_tri_inv`` and
``mg.Hierarchy.vcycle`` (Sec. 4.1, 4.2, 6) on every host core.  Its matrices are the Python
oracle's own: the stiffness matrices K_k of ``sg.build``, the level operators, prolongations and
coarsest inverse of ``mg.Hierarchy``, and the coupling terms read off the G_k.  This module only
hands those arrays to C.

Pins (tests/test_oracle_csolver.py): the solution against the sparse direct solve; the operator,
the V-cycle and B_T^{-1} against the Python oracle's on the same inputs; the iteration count
against the Python oracle's FGMRES.

    python -m oracle.cbuild          # compiles libsgo.so next to this file
"""
import ctypes
import os
import time

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgo.so")

_lib = None


class _Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int), ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


class _Problem(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("Nx", ctypes.c_int), ("M", ctypes.c_int),
                ("K", ctypes.POINTER(_Csr)),
                ("t_ptr", ctypes.c_void_p), ("t_j", ctypes.c_void_p), ("t_k", ctypes.c_void_p),
                ("t_g", ctypes.c_void_p),
                ("l_ptr", ctypes.c_void_p), ("l_j", ctypes.c_void_p), ("l_k", ctypes.c_void_p),
                ("l_g", ctypes.c_void_p),
                ("u_ptr", ctypes.c_void_p), ("u_j", ctypes.c_void_p), ("u_k", ctypes.c_void_p),
                ("u_g", ctypes.c_void_p),
                ("nlev", ctypes.c_int), ("A", ctypes.POINTER(_Csr)), ("Dinv", ctypes.POINTER(ctypes.c_void_p)),
                ("Pr", ctypes.POINTER(_Csr)), ("Rs", ctypes.POINTER(_Csr)), ("coarse_inv", ctypes.c_void_p),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double)]


def lib():
    """Load libsgo.so, compiling it first when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import cbuild
            cbuild.build()
        L = ctypes.CDLL(LIB_PATH)
        VP = ctypes.c_void_p
        L.sgo_threads.restype = ctypes.c_int
        L.sgo_apply.argtypes = [VP, VP, VP]
        L.sgo_vcycles.argtypes = [VP, ctypes.c_int, VP, VP]
        L.sgo_precond_bt.argtypes = [VP, VP, VP, ctypes.c_int]
        L.sgo_bt_fgmres.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.sgo_bt_fgmres.restype = ctypes.c_int
        _lib = L
    return _lib


def threads():
    """Number of OpenMP threads the C oracle runs with (all host cores unless OMP_NUM_THREADS)."""
    return int(lib().sgo_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class CSolver:
    """C copy of one SG system and its V-cycle hierarchy; keeps every array it hands to C alive."""

    def __init__(self, sysm, hier):
        self._keep = []
        self.P, self.Nx = sysm.P, sysm.Nx
        K = (_Csr * (sysm.M + 1))(*[self._csr(Kk) for Kk in sysm.K])
        # terms of A = sum_k G_k (x) K_k per PC row (G_0 = I), the strictly lower ones (j < i), and
        # the strictly upper ones of A^T = sum_k G_k^T (x) K_k^T (row i: (j, k, G_k(j, i)), j > i)
        rows_all = [[] for _ in range(sysm.P)]
        rows_low = [[] for _ in range(sysm.P)]
        rows_upT = [[] for _ in range(sysm.P)]
        for k, G in enumerate(sysm.G):
            ii, jj = np.nonzero(G)
            for i, j in zip(ii, jj):
                rows_all[i].append((j, k, G[i, j]))
                if j < i:
                    rows_low[i].append((j, k, G[i, j]))
            GT = G.T
            for i in range(sysm.P):
                for j in range(i + 1, sysm.P):
                    if GT[i, j] != 0.0:
                        rows_upT[i].append((j, k, GT[i, j]))
        assert all(abs(Kk - Kk.T).max() == 0.0 for Kk in sysm.K), "the transposed sweep relies on symmetric K_k"
        t = self._terms(rows_all)
        lo = self._terms(rows_low)
        up = self._terms(rows_upT)
        nlev = len(hier.A)
        A = (_Csr * nlev)(*[self._csr(a) for a in hier.A])
        dinv = [np.ascontiguousarray(d, dtype=np.float64) for d in hier.Dinv]
        self._keep += dinv
        Dinv = (ctypes.c_void_p * nlev)(*[d.ctypes.data for d in dinv])
        Pr = (_Csr * max(nlev - 1, 1))(*[self._csr(p) for p in hier.P])
        Rs = (_Csr * max(nlev - 1, 1))(*[self._csr(p.T) for p in hier.P])
        cinv = np.ascontiguousarray(hier.coarse_inv, dtype=np.float64)
        self._keep += [K, A, Dinv, Pr, Rs, cinv]
        self.pb = _Problem(sysm.P, sysm.Nx, sysm.M, K, *t, *lo, *up, nlev, A, Dinv, Pr, Rs, _ptr(cinv),
                           hier.nu1, hier.nu2, hier.omega)

    def _csr(self, m):
        m = sp.csr_matrix(m)
        ptr = np.ascontiguousarray(m.indptr, dtype=np.int32)
        idx = np.ascontiguousarray(m.indices, dtype=np.int32)
        val = np.ascontiguousarray(m.data, dtype=np.float64)
        self._keep += [ptr, idx, val]
        return _Csr(m.shape[0], ptr.ctypes.data, idx.ctypes.data, val.ctypes.data)

    def _terms(self, rows):
        ptr = np.zeros(len(rows) + 1, dtype=np.int32)
        js, ks, gs = [], [], []
        for i, r in enumerate(rows):
            ptr[i + 1] = ptr[i] + len(r)
            for j, k, g in r:
                js.append(j), ks.append(k), gs.append(g)
        arrs = [ptr, np.array(js + [0], dtype=np.int32), np.array(ks + [0], dtype=np.int32),
                np.array(gs + [0.0], dtype=np.float64)]
        self._keep += arrs
        return [a.ctypes.data for a in arrs]

    def apply(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1)
        Y = np.empty_like(X)
        lib().sgo_apply(ctypes.byref(self.pb), _ptr(X), _ptr(Y))
        return Y

    def vcycles(self, B, nb):
        B = np.ascontiguousarray(B, dtype=np.float64).reshape(-1)
        X = np.empty_like(B)
        lib().sgo_vcycles(ctypes.byref(self.pb), nb, _ptr(B), _ptr(X))
        return X

    def precond_bt(self, R, transpose=False):
        R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
        Z = np.empty_like(R)
        lib().sgo_precond_bt(ctypes.byref(self.pb), _ptr(R), _ptr(Z), int(transpose))
        return Z

    def fgmres(self, F, restart=30, maxit=400, tol=1e-8, transpose=False):
        """(U, iterations, true relative residual, status, seconds) of BT-FGMRES(restart) from 0
        (transpose: the adjoint system with the transposed sweep)."""
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
        U = np.empty_like(F)
        its, rr = ctypes.c_int(), ctypes.c_double()
        t0 = time.perf_counter()
        rc = lib().sgo_bt_fgmres(ctypes.byref(self.pb), _ptr(F), _ptr(U), restart, maxit, tol, int(transpose),
                                 ctypes.byref(its), ctypes.byref(rr))
        dt = time.perf_counter() - t0
        return U, its.value, rr.value, rc, dt
