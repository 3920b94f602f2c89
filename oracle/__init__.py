"""Plain FP64 CPU oracle for the stochastic Galerkin (SG) block-triangular solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may.  The oracle shares no code with the CUDA path: the
only module both sides use is the seeded input generator
``paper_1304_1755_gb300.inputs``, which holds none of the method's arithmetic.

Source: Zheng, Lin and Xu, "Block Triangular Preconditioning for Stochastic
Galerkin Method" (arXiv 1304.1755).  Every function cites the section,
equation, theorem or table it follows.

Modules
  kl       truncated Karhunen-Loeve expansion of the exponential covariance
           (Sec. 2.1, Eqs. truncated-KLE and exponential-covariance)
  basis    total-degree gPC multi-indices and the stochastic matrices G_k
           (Sec. 2.2, Eq. def-stochastic, Sec. 3.2)
  fem      Q1 stiffness matrices K_k and load vector (Eq. def-stiffness)
  sg       global Galerkin matrix A = sum_k G_k (x) K_k (Eq. tensor-product),
           direct solve and unpreconditioned GMRES
  mg       geometric multigrid V-cycle on the mean operator (Sec. 4.1, 6)
  precond  block-diagonal B_D, block-triangular B_T and the symmetric B_S (flat
           and recursive 2 x 2 forms) (Sec. 4.1, 4.2)
  krylov   right-preconditioned (F)GMRES, GPCG[1], PCG, block Gauss-Seidel
           (Sec. 4.2, 6)
  adjoint  objective E[int u] + Var[int u]/2 and its adjoint gradient
  p1       the paper's own discretisation of its test problem: P1 triangles,
           point Gauss-Seidel V(2,2), and the coupled-cycle reading of B_T (Sec. 6)
  reproduce_tables  prints the counts of Tables 2 and 3 under each reading

Parity pins: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an independent quadrature, brute force, an invariant or a
theorem of the paper, except those whose header says "parity unpinned".
"""
