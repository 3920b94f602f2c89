"""The seeded input recipes (``paper_1304_1755_gb300.inputs``) that both the CUDA path's tests and the
oracle draw from: deterministic per seed, the stated shapes, and the stated distributions."""
import math

import numpy as np

from paper_1304_1755_gb300 import inputs


def test_draws_are_deterministic_per_seed_and_differ_across_seeds():
    a, b, c = inputs.uniform(11, (3, 50)), inputs.uniform(11, (3, 50)), inputs.uniform(12, (3, 50))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(inputs.normal(100, 64), inputs.normal(100, 64))


def test_shapes_and_ranges():
    n = 33
    u = inputs.uniform(5, (4, (n - 2) ** 2))
    assert u.shape == (4, 961) and u.min() >= -1.0 and u.max() < 1.0
    assert inputs.rhs_nodes(1, n).shape == ((n - 2) ** 2,)
    assert inputs.lognormal_cells(2, n).shape == ((n - 1) ** 2,)
    c = inputs.random_cell_coefficients(7, n, 3, spread=0.2)
    assert c.shape == (4, (n - 1) ** 2)
    assert np.all(np.abs(c[1:]) <= 0.2) and np.all(np.abs(c[0] - 1.0) <= 0.2)


def test_distributions_match_the_recipes():
    """Sample moments within five standard errors: f = 1 + 0.1 z, abar = exp(0.2 z) (log-normal with
    mean exp(0.02)), FD directions N(0, 1)."""
    m = 200_000
    f = inputs.rhs_nodes(1, int(math.isqrt(m)) + 2)
    k = f.size
    assert abs(f.mean() - 1.0) <= 5 * 0.1 / math.sqrt(k) and abs(f.std() - 0.1) <= 5 * 0.1 / math.sqrt(2 * k)
    a = inputs.lognormal_cells(2, int(math.isqrt(m)) + 1, 0.2)
    la = np.log(a)
    assert abs(la.mean()) <= 5 * 0.2 / math.sqrt(a.size) and abs(la.std() - 0.2) <= 5 * 0.2 / math.sqrt(2 * a.size)
    assert abs(a.mean() - math.exp(0.02)) <= 5 * a.std() / math.sqrt(a.size)
    z = inputs.normal(100, m)
    assert abs(z.mean()) <= 5 / math.sqrt(m) and abs(z.std() - 1.0) <= 5 / math.sqrt(2 * m)


def test_uneven_batch_recipe():
    """Grids 65^2 .. 513^2 (n = 2^L + 1, L in 6..9), M in 2..6, p in 2..4, sigma in [0.1, 0.5], and the
    per-system seeds 1000 + b; every value of each range occurs in a batch of 64."""
    sysd = inputs.batch_systems(5, 64)
    assert len(sysd) == 64
    Ls = {int(round(math.log2(s["n"] - 1))) for s in sysd}
    assert all(s["n"] == 2 ** int(round(math.log2(s["n"] - 1))) + 1 for s in sysd)
    assert Ls == {6, 7, 8, 9}
    assert {s["M"] for s in sysd} == {2, 3, 4, 5, 6} and {s["p"] for s in sysd} == {2, 3, 4}
    assert all(0.1 <= s["sigma"] <= 0.5 for s in sysd)
    assert [s["seed"] for s in sysd] == list(range(1000, 1064))
    assert inputs.batch_systems(5, 64) == sysd
