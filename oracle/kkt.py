"""KKT residuals of a primal/dual pair (Lemma 2, Eqs. 19a-19c).

The optimality system for min c'x, Ax = b, x in K and its dual
max b'y, A'y + z = c, z in K is
    c - z - A'y = 0,   Ax = b,   x'z = 0,  x in K,  z in K.
The paper stops against another solver's accuracy (Eq. 15); here the
stopping test is a relative KKT residual (reading), every term <= tol:
    r_p    = ||Ax - b|| / (1 + ||b||)
    r_d    = ||A'y + z - c|| / (1 + ||c||)
    r_gap  = |c'x - b'y| / (1 + |c'x| + |b'y|)
    r_cone = max(dist(x, K), dist(z, K)) / (1 + max(||x||, ||z||))
All norms are Euclidean.  The y-free gap of Eq. (15b),
|(A^dagger b)'(c - z) - c'x|, is available separately.

Pinned by: all residuals vanish (to rounding) at a planted optimum and are
positive at perturbed points; the y-free gap equals |b'y - c'x| for every
dual pair z = c - A'y and sees only the row-space part of z
(tests/test_oracle_kkt.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import cones as C

KEYS = ("r_p", "r_d", "r_gap", "r_cone", "obj_p", "obj_d")


def residuals(A, b, c, x, y, z, n_orth: int, soc_dims=()) -> dict:
    """r_p, r_d, r_gap, r_cone of the optimality system (Lemma 2, Eqs. 19a-19c)
    as defined above, plus the two objectives c'x and b'y."""
    A = sp.csr_matrix(A)
    obj_p = float(c @ x)
    obj_d = float(b @ y)
    r_p = np.linalg.norm(A @ x - b) / (1.0 + np.linalg.norm(b))
    r_d = np.linalg.norm(A.T @ y + z - c) / (1.0 + np.linalg.norm(c))
    r_gap = abs(obj_p - obj_d) / (1.0 + abs(obj_p) + abs(obj_d))
    r_cone = max(C.dist_K(x, n_orth, soc_dims), C.dist_K(z, n_orth, soc_dims)) / \
        (1.0 + max(np.linalg.norm(x), np.linalg.norm(z)))
    return dict(r_p=float(r_p), r_d=float(r_d), r_gap=float(r_gap), r_cone=float(r_cone),
                obj_p=obj_p, obj_d=obj_d)


def max_residual(res: dict) -> float:
    """The stopping quantity: the largest of the four relative residuals."""
    return max(res["r_p"], res["r_d"], res["r_gap"], res["r_cone"])


def yfree_gap(A, b, c, x, z) -> float:
    """|(A^dagger b)'(c - z) - c'x| of Eq. (15b), A^dagger b = A'(AA')^{-1} b."""
    A = sp.csr_matrix(A)
    M = (A @ A.T).toarray()
    adb = A.T @ np.linalg.solve(M, b)
    return float(abs(adb @ (c - z) - c @ x))
