"""GB300-native stochastic Galerkin solver with block-triangular preconditioning.

Method: Zheng, Lin and Xu, "Block Triangular Preconditioning for Stochastic
Galerkin Method" (arXiv 1304.1755).  The compute path is the C-ABI library
``libsg.so`` (hand-written sm_103a CUDA, declared in ``include/sg.h``);
``paper_1304_1755_gb300.sg`` is a thin ctypes binding with the same names.
Importing this package loads nothing; the library is loaded on first use of
``paper_1304_1755_gb300.sg`` and a missing library is an error (there is no
CPU fallback).
"""
