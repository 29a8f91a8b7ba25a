"""The subspace range(A_hat') and its reflection (Algorithm 1 step 5, Algorithm 2 steps 12-13).

For A_hat = A diag(O) (Algorithm 2 step 12; O = I in Algorithm 1) the
subspace is A_hat_cal = range(A_hat').  Reading of the paper's dagger
(its notation section says "pseudoinverse of transpose", while every use --
Algorithm 1 step 2, the stopping test Eq. (15b), Lemma 2 -- needs an n x m
matrix with dagger(A) A = projector onto range(A')): the Moore-Penrose
pseudoinverse A_hat^dagger = A_hat' (A_hat A_hat')^{-1}, which requires full
row rank.  With M = A_hat A_hat':
    proj(v)   = A_hat' M^{-1} A_hat v          (orthogonal projector onto range(A_hat'))
    abs(v)    = 2 proj(v) - v                  (Definition 1 applied to the subspace)
    pinv_t(b) = A_hat' M^{-1} b                (A_hat^dagger b)
The linear solve with M is a library step: a dense Cholesky factorisation
(scipy.linalg.cho_factor) when m <= 4000, otherwise plain Jacobi-
preconditioned conjugate gradients written out below, run to a relative
residual of 1e-13.  A failed factorisation (M not positive definite: rank-
deficient A or an empty row) raises FactorError.

Pinned by: abs is an involution and preserves norms (Lemma 1), A_hat proj(v)
= A_hat v, and proj is idempotent (tests/test_oracle_subspace.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class FactorError(RuntimeError):
    """M = A_hat A_hat' is not positive definite."""


def jacobi_pcg(matvec, rhs: np.ndarray, diag: np.ndarray, tol: float = 1e-13,
               max_iter: int | None = None, x0: np.ndarray | None = None):
    """Textbook preconditioned conjugate gradients (Hestenes-Stiefel) with the
    Jacobi preconditioner diag(M); stops when ||r|| <= tol ||rhs||.
    Returns (x, iterations)."""
    n = rhs.size
    if max_iter is None:
        max_iter = max(10 * n, 1000)
    x = np.zeros(n) if x0 is None else x0.copy()
    r = rhs - matvec(x) if x0 is not None else rhs.copy()
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0.0:
        return np.zeros(n), 0
    zv = r / diag
    pdir = zv.copy()
    rho = r @ zv
    for k in range(1, max_iter + 1):
        q = matvec(pdir)
        pq = pdir @ q
        if not pq > 0.0:
            raise FactorError("CG breakdown: M is not positive definite")
        alpha = rho / pq
        x += alpha * pdir
        r -= alpha * q
        if np.linalg.norm(r) <= tol * bnorm:
            return x, k
        zv = r / diag
        rho_new = r @ zv
        pdir = zv + (rho_new / rho) * pdir
        rho = rho_new
    return x, max_iter


class Subspace:
    """Operators of the subspace range(A_hat'), A_hat = A diag(O)."""

    def __init__(self, A, O: np.ndarray, solver: str = "auto", cg_tol: float = 1e-13):
        A = sp.csr_matrix(A, dtype=np.float64)
        self.m, self.n = A.shape
        self.Ah = (A @ sp.diags(np.asarray(O, dtype=np.float64))).tocsr()
        self.AhT = self.Ah.T.tocsr()
        if solver == "auto":
            solver = "chol" if self.m <= 4000 else "cg"
        self.solver = solver
        self.cg_tol = cg_tol
        self.cg_iters = 0
        if solver == "chol":
            M = (self.Ah @ self.AhT).toarray()
            try:
                self._chol = sla.cho_factor(M, lower=True, check_finite=True)
            except (sla.LinAlgError, ValueError) as e:
                raise FactorError(str(e)) from e
            # a numerically singular M passes cho_factor with a tiny pivot: reject it
            piv = np.abs(np.diag(self._chol[0]))
            if piv.min() <= 1e-12 * piv.max():
                raise FactorError("M = A_hat A_hat' is numerically singular")
        elif solver == "cg":
            self._diag = np.asarray(self.Ah.multiply(self.Ah).sum(axis=1)).ravel()
            if np.any(self._diag <= 0.0):
                raise FactorError("empty row in A_hat")
        else:
            raise ValueError(solver)

    def matvec_M(self, v: np.ndarray) -> np.ndarray:
        return self.Ah @ (self.AhT @ v)

    def solve_M(self, rhs: np.ndarray) -> np.ndarray:
        """M^{-1} rhs."""
        if self.solver == "chol":
            return sla.cho_solve(self._chol, rhs)
        w, k = jacobi_pcg(self.matvec_M, rhs, self._diag, tol=self.cg_tol)
        self.cg_iters += k
        return w

    def pinv_t(self, b: np.ndarray) -> np.ndarray:
        """A_hat^dagger b = A_hat' M^{-1} b."""
        return self.AhT @ self.solve_M(b)

    def proj(self, v: np.ndarray) -> np.ndarray:
        """Orthogonal projection onto range(A_hat')."""
        return self.AhT @ self.solve_M(self.Ah @ v)

    def abs(self, v: np.ndarray) -> np.ndarray:
        """abs_{A_hat_cal}(v) = 2 proj(v) - v."""
        return 2.0 * self.proj(v) - v
