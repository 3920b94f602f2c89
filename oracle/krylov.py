"""Krylov solvers used with the block preconditioners (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.2: B_T is nonsymmetric, so it is used with GMRES (Saad-Schultz) or
GPCG (Blaheta); B_D (and the symmetric B_S) with standard PCG.  Sec. 6: zero
initial guess, stop on the relative Euclidean residual, GMRes(10) restarted,
GPCG[1].

* ``gmres``: restarted GMRES with right preconditioning.  ``flexible=True``
  stores the preconditioned vectors z_j = M^{-1} v_j and updates x += Z y
  (FGMRES); otherwise x += M^{-1}(V y).  Modified Gram-Schmidt, Givens
  rotations; the true residual is recomputed at every restart and at the end.
* ``gpcg1``: GPCG with one stored direction.  The paper cites the method
  without printing it; the reading used is: g = M^{-1} r; the new direction
  d = g - (<A g, d'> / <A d', d'>) d' is A-orthogonalised against the previous
  direction d'; alpha = <r, d> / <A d, d>; x += alpha d; r -= alpha A d.
* ``pcg``: standard preconditioned conjugate gradients.
* ``gmres_left``: restarted GMRES on M^{-1} A x = M^{-1} b, stopping on the preconditioned
  residual (a reading of the paper's Table 3 runs, see the function).

Each returns (x, iterations, true relative residual).  Iterations count
preconditioner applications.  Pins: the solutions against the direct solve;
the k-step iterates against their defining minimisation (GMRES: least
residual over x0 + M K_k; PCG: least energy error over K_k) by brute force on
a small system, GPCG[1] with an SPD preconditioner against PCG, FGMRES with a
fixed preconditioner against GMRES.  The paper's own iteration counts are for
another discretisation and smoother, so they are not a pin.
"""
import numpy as np


def gmres(apply_A, apply_M, b, x0=None, tol=1e-8, restart=30, maxit=1000, flexible=False):
    b = np.asarray(b, dtype=np.float64)
    Minv = (lambda v: v) if apply_M is None else apply_M
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    its = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or its >= maxit:
            return x, its, beta / bnorm
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            z = Minv(V[j])
            if flexible:
                Z.append(z)
            w = apply_A(z)
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        if flexible:
            for i in range(k):
                x = x + y[i] * Z[i]
        else:
            x = x + Minv(sum(y[i] * V[i] for i in range(k)))


def gmres_left(apply_A, apply_M, b, x0=None, tol=1e-8, restart=30, maxit=1000):
    """Restarted GMRES on the left-preconditioned system M^{-1} A x = M^{-1} b, stopping when the
    preconditioned residual ||M^{-1}(b - A x)|| <= tol ||M^{-1} b|| (the criterion of a left-
    preconditioned GMRES such as MATLAB's, which the paper's Table 3 runs were made with; the paper
    states only "relative residual").  Classical Gram-Schmidt run twice per step, Givens rotations.
    Returns (x, iterations, true relative residual ||b - A x|| / ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    pbnorm = np.linalg.norm(apply_M(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    its = 0
    while True:
        r = apply_M(b - apply_A(x))
        beta = np.linalg.norm(r)
        if beta <= tol * pbnorm or its >= maxit:
            return x, its, np.linalg.norm(b - apply_A(x)) / bnorm
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            w = apply_M(apply_A(V[j]))
            for _ in range(2):
                for i in range(j + 1):
                    c = np.dot(V[i], w)
                    H[i, j] += c
                    w = w - c * V[i]
            hnext = np.linalg.norm(w)
            H[j + 1, j] = hnext
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= tol * pbnorm or its >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + sum(y[i] * V[i] for i in range(k))


def gpcg1(apply_A, apply_M, b, x0=None, tol=1e-8, maxit=1000):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - apply_A(x)
    d_prev = Ad_prev = None
    its = 0
    while np.linalg.norm(r) > tol * bnorm and its < maxit:
        gv = apply_M(r)
        Ag = apply_A(gv)
        if d_prev is None:
            d, Ad = gv, Ag
        else:
            beta = np.dot(Ag, d_prev) / np.dot(Ad_prev, d_prev)
            d = gv - beta * d_prev
            Ad = Ag - beta * Ad_prev
        alpha = np.dot(r, d) / np.dot(Ad, d)
        x = x + alpha * d
        r = r - alpha * Ad
        d_prev, Ad_prev = d, Ad
        its += 1
    rt = b - apply_A(x)
    return x, its, np.linalg.norm(rt) / bnorm


def pcg(apply_A, apply_M, b, x0=None, tol=1e-8, maxit=1000):
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - apply_A(x)
    z = apply_M(r)
    d = z.copy()
    rz = np.dot(r, z)
    its = 0
    while np.linalg.norm(r) > tol * bnorm and its < maxit:
        Ad = apply_A(d)
        alpha = rz / np.dot(d, Ad)
        x = x + alpha * d
        r = r - alpha * Ad
        its += 1
        z = apply_M(r)
        rz_new = np.dot(r, z)
        d = z + (rz_new / rz) * d
        rz = rz_new
    rt = b - apply_A(x)
    return x, its, np.linalg.norm(rt) / bnorm


def block_gauss_seidel(apply_A, apply_BT, b, x0=None, tol=1e-8, maxit=1000):
    """Stationary block Gauss-Seidel iteration of Sec. 4.2 (the B-GS rows of Table 3):
    x_{k+1} = x_k + B_T^{-1} (b - A x_k), zero initial guess."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - apply_A(x)
    its = 0
    while np.linalg.norm(r) > tol * bnorm and its < maxit:
        x = x + apply_BT(r)
        r = b - apply_A(x)
        its += 1
    return x, its, np.linalg.norm(r) / bnorm
