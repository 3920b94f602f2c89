"""Reproduce the iteration counts of the paper's Tables 2 and 3 with the oracle's version of the
paper's own discretisation (``oracle.p1``), under each reading of B_T and B_S.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): it calls the oracle and nothing else, and prints
the counts beside the paper's (``tests/golden/paper_examples.json``).  A full run takes a few minutes
on one core:

    python -m oracle.reproduce_tables            # Table 3, all readings
    python -m oracle.reproduce_tables --table2   # Table 2 (sigma = 0.1, several h, p, m)
"""
import argparse
import json
import os

import numpy as np

from . import basis, krylov, p1, precond, sg

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                      "paper_examples.json")


def _setup(n, M, p, sigma):
    s = p1.build(n, M, p, basis.LEGENDRE, sigma)
    F = p1.rhs(s)
    solver = precond.DiagSolver(s.K[0], p1.GSHierarchy(s.K[0], n))
    return s, F, solver


def table3_counts(sigma, n=65, M=6, p=4):
    """Counts of the five methods at one sigma under the flat and the coupled readings of B_T (the
    coupled one with lexicographic and with four-colour Gauss-Seidel) and the flat and recursive B_S."""
    s, F, solver = _setup(n, M, p, sigma)
    Ax = lambda v: sg.apply(s, v)
    off = basis.degree_levels(s.alphas)
    low = np.arange(off[-2])
    flat = lambda r: precond.block_tri_inv(s, solver, r)
    lex = p1.CoupledGSHierarchy(s, low)
    mc = p1.MulticolourCoupledGSHierarchy(s, low)
    coupled = lambda r: p1.block_tri_2x2_inv(s, lex, solver, r)
    coupled4 = lambda r: p1.block_tri_2x2_inv(s, mc, solver, r)
    out = {}
    for tag, bt in (("flat", flat), ("coupled", coupled), ("coupled-4c", coupled4)):
        out["Block-GS " + tag] = krylov.block_gauss_seidel(Ax, bt, F, tol=1e-10, maxit=400)[1]
        out["BT-GPCG " + tag] = krylov.gpcg1(Ax, bt, F, tol=1e-10, maxit=400)[1]
        out["BT-GMRes " + tag] = krylov.gmres(Ax, bt, F, tol=1e-10, restart=10, maxit=400)[1]
        out["BT-GMRes-left " + tag] = krylov.gmres_left(Ax, bt, F, tol=1e-10, restart=10, maxit=400)[1]
    out["BD-PCG"] = krylov.pcg(Ax, lambda r: precond.block_diag_inv(s, solver, r), F, tol=1e-10, maxit=400)[1]
    out["BS-PCG flat"] = krylov.pcg(Ax, lambda r: precond.block_sym_inv(s, solver, r), F, tol=1e-10, maxit=400)[1]
    out["BS-PCG recursive"] = krylov.pcg(Ax, lambda r: precond.block_sym_recursive_inv(s, solver, r), F, tol=1e-10,
                                         maxit=400)[1]
    return out


def table2_counts(n, M, p, sigma=0.1):
    s, F, solver = _setup(n, M, p, sigma)
    Ax = lambda v: sg.apply(s, v)
    bt = lambda r: precond.block_tri_inv(s, solver, r)
    return {
        "BD-PCG": krylov.pcg(Ax, lambda r: precond.block_diag_inv(s, solver, r), F, tol=1e-10, maxit=400)[1],
        "BT-GPCG": krylov.gpcg1(Ax, bt, F, tol=1e-10, maxit=400)[1],
        "BS-PCG": krylov.pcg(Ax, lambda r: precond.block_sym_recursive_inv(s, solver, r), F, tol=1e-10,
                             maxit=400)[1],
        "BT-GMRes": krylov.gmres(Ax, bt, F, tol=1e-10, restart=10, maxit=400)[1],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--table2", action="store_true")
    args = ap.parse_args()
    golden = json.load(open(GOLDEN))
    if args.table2:
        paper = golden["table2"]
        print("Table 2 (sigma = 0.1): oracle counts, paper in brackets")
        for n, M, p in ((33, 4, 2), (33, 6, 2), (33, 4, 3), (65, 4, 2), (129, 4, 2)):
            c = table2_counts(n, M, p)
            print(f"h = 1/{n - 1}, m = {M}, p = {p}: " + ", ".join(f"{k} {v} ({paper[k]})" for k, v in c.items()),
                  flush=True)
        return
    t3 = golden["table3"]
    for j, sigma in enumerate(t3["sigma"]):
        c = table3_counts(sigma)
        print(f"sigma = {sigma}", flush=True)
        for k, v in c.items():
            method = k.split(" ")[0].replace("-left", "")
            print(f"  {k:22s} {v:4d}   paper {t3[method][j][0]}", flush=True)


if __name__ == "__main__":
    main()
