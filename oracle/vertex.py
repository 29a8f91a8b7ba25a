"""Brute-force LP solution by vertex enumeration (ground truth for tiny LPs).

For min c'x, Ax = b, x >= 0 with A of full row rank m, every basic feasible
solution is x_B = A_B^{-1} b >= 0 for a set B of m linearly independent
columns, and a bounded LP attains its optimum at one of them (fundamental
theorem of linear programming).  Enumerating all C(n, m) bases is
exponential, so this is only for m <= 6, n <= 12.
"""
from __future__ import annotations

import itertools

import numpy as np


def enumerate_vertices(A: np.ndarray, b: np.ndarray, feas_tol: float = 1e-10):
    """All basic feasible solutions as (x, basis) pairs."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    out = []
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if np.linalg.matrix_rank(AB) < m:
            continue
        xB = np.linalg.solve(AB, b)
        if np.all(xB >= -feas_tol):
            x = np.zeros(n)
            x[list(B)] = np.maximum(xB, 0.0)
            out.append((x, B))
    return out


def solve_lp(A, b, c, feas_tol: float = 1e-10):
    """(x*, c'x*, bases attaining it) over all vertices; raises if none is feasible."""
    verts = enumerate_vertices(A, b, feas_tol)
    if not verts:
        raise ValueError("no feasible vertex")
    objs = np.array([c @ x for x, _ in verts])
    best = objs.min()
    tol = 1e-9 * (1.0 + abs(best))
    winners = [(x, B) for (x, B), o in zip(verts, objs) if o <= best + tol]
    return winners[0][0], float(best), [B for _, B in winners]
