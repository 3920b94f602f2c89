"""Host-side arithmetic of bench.py (no GPU): the couplings per row that enter the operator's
algorithmic flop count equal the nonzeros of sum_k G_k built by the oracle, and the
workload table matches the configuration sizes."""
import math
import os
import sys

import numpy as np

from oracle import basis

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_couplings_per_row_match_oracle_pattern():
    for name in ("c1", "c2", "c3", "c4"):
        wl = bench.WORKLOADS[name]
        al = basis.multi_indices(wl["M"], wl["p"])
        G = basis.g_matrices(al, basis.LEGENDRE if wl["family"] == 0 else basis.HERMITE)
        nnz = sum(int(np.count_nonzero(g)) for g in G)          # G_0 = I contributes the mean term
        assert abs(bench.terms_per_row(wl) * len(al) - nnz) < 1e-9


def test_workload_sizes():
    c3 = bench.WORKLOADS["c3"]
    assert math.comb(c3["M"] + c3["p"], c3["p"]) == 210
    assert (c3["n"] - 2) ** 2 * 210 == 219_771_090
    c2 = bench.WORKLOADS["c2"]
    assert (c2["n"] - 2) ** 2 * math.comb(c2["M"] + c2["p"], c2["p"]) == 4_551_750
    # FP64 flop count of the canonical operator at C3: 67.2 per unknown
    assert abs(bench.k1_method_flops(c3) / ((c3["n"] - 2) ** 2 * 210) - 67.2) < 1e-9


def test_gram_schmidt_fma_count():
    """Classical Gram-Schmidt costs 2 (j + 2) FP64 FMA per element at Arnoldi step j of a cycle; 15 steps
    of one FGMRES(20) cycle give 270 per element, and a restart starts the count again."""
    import bench
    assert bench.gs_fp64_fmas(1, 15, 20) == 270
    assert bench.gs_fp64_fmas(10, 1, 20) == 40
    assert bench.gs_fp64_fmas(1, 5, 3) == bench.gs_fp64_fmas(1, 3, 3) + bench.gs_fp64_fmas(1, 2, 3)
