"""The comparison iterations of Section III-B (Douglas-Rachford splitting and
ADMM) for the conic program of Eq. (1), in FP64 -- test infrastructure: they
run the convergence comparison of Section III-A (the worked example, with
no preconditioning, the printed Sinkhorn-Knopp scalings and the printed
adaptive-conditioning scaling), not a product path.

Splitting (Section III-B): f = indicator of K, g(x) = c'x + indicator{Ax = b}.
    prox_{mu f}(v) = proj_K(v)
    prox_{mu g}(v) = argmin_x c'x + ||x - v||^2 / (2 mu) s.t. Ax = b
                   = P_aff(v - mu c),  P_aff(u) = u - A'(AA')^{-1}(Au - b)
DR (the section's two steps, prox taken with parameter mu):
    x <- prox_{mu f}(z);   z <- z + prox_{mu g}(2x - z) - x
ADMM (the section's three steps):
    x1 <- prox_{f/mu}(x2 - z/mu);  x2 <- prox_{g/mu}(x1 + z/mu);  z <- z + mu (x1 - x2)
with prox_{g/mu}(v) = P_aff(v - c/mu).

Preconditioning by positive diagonals D (rows) and E (columns): the
iteration runs on min (Ec)'u s.t. (DAE)u = Db, u in K (E keeps K = R+^n
invariant) and its point is mapped back by x = E u.

ADMM is Douglas-Rachford with the two proximal steps swapped, on the
variable zeta = x1 + z_prev/mu: zeta <- zeta + proj_K(2 prox_g(zeta) - zeta)
- prox_g(zeta), with x2 = prox_g(zeta) (the textbook identity, used as a pin).

Ruiz equilibration (a standard equilibrating preconditioner that the code
computes itself, beside the printed Sinkhorn-Knopp scalings): row and column
infinity norms of DAE driven to 1 by repeated square-root scalings.

Pinned by: DR's z reproduces Algorithm 1's s (Section III-B's splitting is
the one Algorithm 1 runs), ADMM's x2 reproduces the swapped DR, both reach
the worked example's vertex optimum, Ruiz's scaled matrix has unit row and
column maxima (tests/test_oracle_baselines.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import cones as C


class _Affine:
    """Projection onto {u : Au = b} for a dense A of full row rank:
    u - A'(AA')^{-1}(Au - b) = u - Q R'^{-1}(Au - b) with A' = QR (thin QR,
    so the projection does not square A's condition number)."""

    def __init__(self, A, b):
        self.A = np.asarray(A, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.Q, self.R = np.linalg.qr(self.A.T)

    def __call__(self, u):
        r = self.A @ u - self.b
        return u - self.Q @ sla.solve_triangular(self.R, r, trans="T")


def _scaled(A, b, c, D, E):
    A = np.asarray(A, dtype=np.float64)
    D = np.ones(A.shape[0]) if D is None else np.asarray(D, dtype=np.float64)
    E = np.ones(A.shape[1]) if E is None else np.asarray(E, dtype=np.float64)
    return (D[:, None] * A) * E[None, :], D * np.asarray(b, float), E * np.asarray(c, float), E


def douglas_rachford(A, b, c, n_orth, soc_dims=(), mu=1.0, D=None, E=None, iters=1000, z0=None):
    """x = E u after each DR iteration (list) and the last z, on the problem
    scaled by D, E."""
    As, bs, cs, E = _scaled(A, b, c, D, E)
    aff = _Affine(As, bs)
    z = np.zeros(As.shape[1]) if z0 is None else np.asarray(z0, float).copy()
    out = []
    for _ in range(iters):
        x = C.proj_K(z, n_orth, soc_dims)
        z = z + aff(2.0 * x - z - mu * cs) - x
        out.append(E * x)
    return out, z


def admm(A, b, c, n_orth, soc_dims=(), mu=1.0, D=None, E=None, iters=1000, x2_0=None, z_0=None):
    """x = E x1 after each ADMM iteration (list), on the problem scaled by D,
    E, from x2 = x2_0 and z = z_0 (default 0)."""
    As, bs, cs, E = _scaled(A, b, c, D, E)
    aff = _Affine(As, bs)
    n = As.shape[1]
    x2 = np.zeros(n) if x2_0 is None else np.asarray(x2_0, float).copy()
    z = np.zeros(n) if z_0 is None else np.asarray(z_0, float).copy()
    out = []
    for _ in range(iters):
        x1 = C.proj_K(x2 - z / mu, n_orth, soc_dims)
        x2 = aff(x1 + z / mu - cs / mu)
        z = z + mu * (x1 - x2)
        out.append(E * x1)
    return out


def ruiz(A, iters=20):
    """Ruiz equilibration (infinity norms): D <- D / sqrt(row max |DAE|),
    E <- E / sqrt(column max |DAE|), repeated; returns (D, E)."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    D, E = np.ones(A.shape[0]), np.ones(A.shape[1])
    for _ in range(iters):
        S = D[:, None] * A * E[None, :]
        D = D / np.sqrt(S.max(axis=1))
        E = E / np.sqrt(S.max(axis=0))
    return D, E


def iterations_to(xs, x_star, rtol):
    """First iteration (1-based) from which ||x - x*|| <= rtol ||x*|| holds for
    good, or None."""
    ok = [np.linalg.norm(x - x_star) <= rtol * np.linalg.norm(x_star) for x in xs]
    for k in range(len(ok)):
        if all(ok[k:]):
            return k + 1
    return None
