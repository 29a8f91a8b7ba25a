"""LP crossover polish in FP64 -- test infrastructure, not a product path.

The paper stops Algorithm 2 on its KKT test and polishes nothing (other
solvers' polishing is only mentioned); this is the active-set polish of an
approximate LP solution (K = R+^n) built as an alternative to running
Algorithm 2 on to a tighter tolerance:

  B  = {j : x_j > z_j}                       (support guess: x_j > 0 = z_j at a
                                              strictly complementary optimum)
  x~ = the orthogonal projection of x onto {u : u_j = 0 (j not in B), A u = b}
     = x_B + A_B' (A_B A_B')^+ (b - A_B x_B)  on B, 0 elsewhere;
  y~ = the projection of y onto {v : A_B' v = c_B} in the metric of
       J = diag(A_B A_B') (J_ii = 1 where the row has no entry in B):
       y + J^{-1/2} (A_B' J^{-1/2})^+ (c_B - A_B' y);
  z~ = c - A' y~.

At a nondegenerate vertex (|B| = m, A_B nonsingular) x~ and y~ are the
vertex and its unique dual, whatever x and y were.  The metric of y~
matters only where A_B' v = c_B leaves v free (|B| < m); it is the one a
Jacobi-preconditioned CG started from zero works in.  The polished point is
taken only if its largest relative KKT residual is below the iterate's.

The pseudoinverse solves are numpy's least-squares routine on dense
matrices (small problems only).

Pinned by: the worked example's vertex and dual recovered from a rough
iterate, random nondegenerate LPs against vertex enumeration, the
projection property (x~ is feasible and x - x~ is orthogonal to the
affine set's directions), and the degenerate case's J-metric minimality
(tests/test_oracle_crossover.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import kkt


def support(x, z):
    return np.asarray(x) > np.asarray(z)


def polish(A, b, c, x, y, z):
    """(x~, y~, z~, B) as defined above (dense algebra)."""
    A = sp.csr_matrix(A, dtype=np.float64).toarray()
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    B = support(x, z)
    AB = A[:, B]
    xt = np.zeros_like(x)
    if B.any():
        corr = np.linalg.lstsq(AB, b - AB @ x[B], rcond=None)[0]
        xt[B] = x[B] + corr
    diag = (AB * AB).sum(axis=1)
    jh = np.where(diag > 0.0, np.sqrt(np.where(diag > 0.0, diag, 1.0)), 1.0)
    rc = c[B] - AB.T @ y
    d = np.linalg.lstsq(AB.T / jh[None, :], rc, rcond=None)[0] / jh if B.any() else np.zeros_like(y)
    yt = y + d
    zt = c - A.T @ yt
    return xt, yt, zt, B


def polish_if_better(A, b, c, x, y, z, n_orth=None):
    """The polished point if its largest KKT residual is smaller, else the
    iterate; returns (x, y, z, accepted, residuals before, after)."""
    n = len(x)
    n_orth = n if n_orth is None else n_orth
    before = kkt.residuals(sp.csr_matrix(A), b, c, x, y, z, n_orth, [])
    xt, yt, zt, _ = polish(A, b, c, x, y, z)
    after = kkt.residuals(sp.csr_matrix(A), b, c, xt, yt, zt, n_orth, [])
    if kkt.max_residual(after) < kkt.max_residual(before):
        return xt, yt, zt, True, before, after
    return np.asarray(x), np.asarray(y), np.asarray(z), False, before, after
