"""Exact optimum of the (unregularised) POT linear programme for tiny inputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/pot.py``).

``pot_lp`` writes the slack LP form of the appendix ("Linear Programming Form
of POT"): x = (vec X, p, q) >= 0, minimise <C, X> subject to
X 1 + p = r, X^T 1 + q = c and 1^T X 1 = s, and hands it to scipy's HiGHS
solver (a library primitive).  ``kmatching_bruteforce`` computes the same
optimum by enumeration for uniform marginals, where the optimum is attained at
a partial matching (vertices of the bipartite k-cardinality matching polytope
are integral), so the two pin each other.
"""
from __future__ import annotations

import itertools

import numpy as np


def pot_lp(C, r, c, s) -> float:
    from scipy.optimize import linprog

    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    nx = n * m
    nv = nx + n + m
    cost = np.concatenate([C.reshape(-1), np.zeros(n + m)])
    A = np.zeros((n + m + 1, nv))
    for i in range(n):
        A[i, i * m:(i + 1) * m] = 1.0          # row sums of X
        A[i, nx + i] = 1.0                    # + p_i
    for j in range(m):
        A[n + j, j:nx:m] = 1.0                # column sums of X
        A[n + j, nx + n + j] = 1.0            # + q_j
    A[n + m, :nx] = 1.0                       # total mass
    b = np.concatenate([np.asarray(r, float), np.asarray(c, float), [s]])
    res = linprog(cost, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    return float(res.fun)


def kmatching_bruteforce(C, k: int) -> float:
    """Minimum total cost of a matching with exactly k edges between the rows
    and columns of C (exhaustive search over row subsets and injective column
    assignments)."""
    C = np.asarray(C, dtype=np.float64)
    n, m = C.shape
    best = np.inf
    for rows in itertools.combinations(range(n), k):
        for cols in itertools.permutations(range(m), k):
            v = sum(C[i, j] for i, j in zip(rows, cols))
            if v < best:
                best = v
    return float(best)
