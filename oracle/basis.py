"""Total-degree gPC basis and stochastic matrices G_k (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.2: Xi_p = span of the orthonormal polynomials of total degree <= p in m
variables, dimension N_xi = (m+p)!/(m! p!).  Sec. 3.3: the basis is
hierarchical, degree by degree, which gives the 2x2 split of Eq.
(hierarchical_structure).  Ordering used here: by total degree, then
descending lexicographic order of the multi-index within one degree (the paper
only requires the degree grading).

Eq. (def-stochastic): G_0(i,j) = E[psi_i psi_j] = delta_ij (orthonormality,
Sec. 3.2), G_k(i,j) = E[xi_k psi_i psi_j].  With product bases this factors
into 1-D integrals; the three-term recurrence of the orthonormal 1-D family,
  xi q_n(xi) = gamma(n) q_{n+1}(xi) + gamma(n-1) q_{n-1}(xi),
gives G_k(i,j) = gamma(min(a_k, b_k)) when the multi-indices differ by one in
component k only, else 0.
  Legendre on U(-sqrt3, sqrt3):  gamma(n) = sqrt3 (n+1) / sqrt((2n+1)(2n+3))
  Hermite on N(0,1):             gamma(n) = sqrt(n+1)

Pins: Gauss quadrature of the triple products with independently built
orthonormal polynomials; N_xi formula and the m=6, p=4 -> 210 example (Sec.
2.2); Table 1 block counts.
"""
import math
from itertools import product

import numpy as np

LEGENDRE, HERMITE = 0, 1


def n_basis(M, p):
    """N_xi = (M+p)! / (M! p!)  (Sec. 2.2)."""
    return math.comb(M + p, p)


def multi_indices(M, p):
    """All alpha in N^M with |alpha| <= p: by degree, descending lex within a degree."""
    out = []
    for q in range(p + 1):
        level = [a for a in product(range(q + 1), repeat=M) if sum(a) == q]
        level.sort(reverse=True)
        out.extend(level)
    if M == 0:
        out = [()]
    return out


def degree_levels(alphas):
    """Start offsets of each total-degree level: rows [off[q], off[q+1]) have degree q."""
    degs = [sum(a) for a in alphas]
    p = max(degs)
    off = [0]
    for q in range(p + 1):
        off.append(off[-1] + degs.count(q))
    return off


def gamma(family, n):
    """Off-diagonal entry of the Jacobi matrix of the orthonormal 1-D family."""
    if family == LEGENDRE:
        return math.sqrt(3.0) * (n + 1) / math.sqrt((2 * n + 1) * (2 * n + 3))
    if family == HERMITE:
        return math.sqrt(n + 1.0)
    raise ValueError("family")


def g_matrices(alphas, family):
    """Dense G_0..G_M (list of P x P arrays), Eq. (def-stochastic)."""
    P = len(alphas)
    M = len(alphas[0]) if P else 0
    index = {a: i for i, a in enumerate(alphas)}
    G = [np.eye(P)]
    for k in range(M):
        Gk = np.zeros((P, P))
        for i, a in enumerate(alphas):
            up = list(a)
            up[k] += 1
            j = index.get(tuple(up))
            if j is not None:
                v = gamma(family, a[k])
                Gk[i, j] = v
                Gk[j, i] = v
        G.append(Gk)
    return G
