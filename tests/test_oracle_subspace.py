"""Pins for the oracle's subspace operators (Algorithm 1 steps 1-2, 5).

abs over range(A') is a reflection: an involution that preserves norms
(Lemma 1); proj is idempotent, symmetric, and leaves A v unchanged; the
pseudoinverse reading gives A (A^dagger b) = b.  The CG solver must agree
with the Cholesky solver.  Rank deficiency is reported, not hidden.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.subspace import Subspace, FactorError, jacobi_pcg


def _rand_A(rng, m, n, dens=0.3):
    while True:
        A = sp.random(m, n, density=dens, random_state=rng, data_rvs=rng.standard_normal).tocsr()
        if np.linalg.matrix_rank(A.toarray()) == m:
            return A


@pytest.mark.parametrize("solver", ["chol", "cg"])
def test_reflection_properties(solver):
    rng = np.random.default_rng(5)
    A = _rand_A(rng, 7, 15)
    O = rng.uniform(0.1, 10.0, 15)
    S = Subspace(A, O, solver=solver)
    Ah = (A @ sp.diags(O)).toarray()
    for _ in range(20):
        v = rng.standard_normal(15)
        pv = S.proj(v)
        np.testing.assert_allclose(S.proj(pv), pv, atol=1e-10)
        np.testing.assert_allclose(Ah @ pv, Ah @ v, atol=1e-10)
        av = S.abs(v)
        assert abs(np.linalg.norm(av) - np.linalg.norm(v)) < 1e-10
        np.testing.assert_allclose(S.abs(av), v, atol=1e-10)
        u = rng.standard_normal(15)
        assert abs(u @ S.proj(v) - v @ S.proj(u)) < 1e-10
    b = rng.standard_normal(7)
    np.testing.assert_allclose(Ah @ S.pinv_t(b), b, atol=1e-10)
    # dagger(A) b is the minimum-norm solution: orthogonal to the null space of A_hat
    np.testing.assert_allclose(S.pinv_t(b), np.linalg.pinv(Ah) @ b, atol=1e-10)


def test_cg_matches_cholesky():
    rng = np.random.default_rng(6)
    A = _rand_A(rng, 30, 70, 0.2)
    O = np.exp(rng.uniform(-2, 2, 70))
    a = Subspace(A, O, solver="chol")
    b = Subspace(A, O, solver="cg")
    r = rng.standard_normal(30)
    np.testing.assert_allclose(a.solve_M(r), b.solve_M(r), rtol=1e-9, atol=1e-12)


def test_pcg_textbook_spd():
    rng = np.random.default_rng(7)
    Q = rng.standard_normal((40, 40))
    M = Q @ Q.T + 40 * np.eye(40)
    rhs = rng.standard_normal(40)
    x, k = jacobi_pcg(lambda v: M @ v, rhs, np.diag(M).copy(), tol=1e-14)
    np.testing.assert_allclose(x, np.linalg.solve(M, rhs), rtol=1e-10)
    assert k <= 40 + 5


def test_rank_deficient_raises():
    A = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 0.0]]))
    with pytest.raises(FactorError):
        Subspace(A, np.ones(3), solver="chol")
    A2 = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [0.0, 0.0, 0.0]]))
    with pytest.raises(FactorError):
        Subspace(A2, np.ones(3), solver="cg")
