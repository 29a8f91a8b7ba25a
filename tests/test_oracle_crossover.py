"""The LP crossover polish of the oracle (oracle/crossover.py), pinned
against vertex enumeration, LP duality and the projection definitions
(CPU only)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import alg, crossover as X, kkt, vertex

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))


def _rough(A, b, c, tol):
    r = alg.algorithm2(sp.csr_matrix(A), b, c, A.shape[1], [], L=alg.LP_SCHEDULE, max_iter=20000, tol=tol,
                       check_every=1)
    return r.x, r.y, r.z


def test_worked_example_vertex_from_a_rough_iterate():
    A, b, c = np.array(GOLD["A"]), np.array(GOLD["b"]), np.array(GOLD["c"])
    x, y, z = _rough(A, b, c, 1e-3)
    before = kkt.max_residual(kkt.residuals(sp.csr_matrix(A), b, c, x, y, z, 5, []))
    assert before > 1e-5
    xt, yt, zt, ok, _, after = X.polish_if_better(A, b, c, x, y, z)
    assert ok
    xs, obj = vertex.solve_lp(A, b, c)[:2]
    np.testing.assert_allclose(xt, xs, atol=1e-11)
    # the dual of the optimal basis: reduced costs >= 0 and complementary, strong duality
    assert (zt >= -1e-12).all() and np.abs(zt[xs > 0]).max() <= 1e-12
    assert abs(b @ yt - obj) <= 1e-11 * abs(obj)
    assert kkt.max_residual(after) <= 1e-12


def _random_vertex_lp(rng, m, n):
    """A random LP with a unique nondegenerate optimal vertex: basis of m
    columns, x_B > 0, reduced costs > 0 off the basis."""
    A = rng.standard_normal((m, n))
    basis = rng.choice(n, m, replace=False)
    xs = np.zeros(n)
    xs[basis] = rng.uniform(0.5, 2.0, m)
    y = rng.standard_normal(m)
    zs = np.zeros(n)
    off = np.setdiff1d(np.arange(n), basis)
    zs[off] = rng.uniform(0.5, 2.0, off.size)
    return A, A @ xs, A.T @ y + zs, xs, y, zs


@pytest.mark.parametrize("seed", range(6))
def test_random_vertices_recovered(seed):
    rng = np.random.default_rng(100 + seed)
    A, b, c, xs, ys, zs = _random_vertex_lp(rng, 4, 9)
    # enumeration agrees that xs is the optimum
    xe = vertex.solve_lp(A, b, c)[0]
    np.testing.assert_allclose(xe, xs, atol=1e-9)
    noise = 1e-3
    x = xs + noise * rng.standard_normal(9)
    y = ys + noise * rng.standard_normal(4)
    z = zs + noise * rng.standard_normal(9)
    xt, yt, zt, B = X.polish(A, b, c, x, y, z)
    assert (B == (xs > 0)).all()
    np.testing.assert_allclose(xt, xs, atol=1e-11)
    np.testing.assert_allclose(yt, ys, atol=1e-10)
    np.testing.assert_allclose(zt, zs, atol=1e-10)


def test_x_polish_is_the_orthogonal_projection():
    """|B| > m: x~ satisfies A x~ = b with x~ = 0 off B, and x_B - x~_B lies in
    range(A_B') (orthogonal to the affine set's directions)."""
    rng = np.random.default_rng(7)
    m, n = 5, 14
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    c = rng.standard_normal(n)
    x = rng.uniform(0.0, 1.0, n)
    z = rng.uniform(0.0, 1.0, n)
    z[:9] = 0.0                                        # B has at least 9 > m columns
    y = rng.standard_normal(m)
    xt, _, _, B = X.polish(A, b, c, x, y, z)
    assert B.sum() > m
    np.testing.assert_allclose(A @ xt, b, atol=1e-12)
    assert (xt[~B] == 0).all()
    AB = A[:, B]
    v, *_ = np.linalg.lstsq(AB.T, x[B] - xt[B], rcond=None)
    np.testing.assert_allclose(AB.T @ v, x[B] - xt[B], atol=1e-12)


def test_y_polish_is_the_j_metric_projection():
    """|B| < m leaves y free along null(A_B'): y~ minimises ||J^{1/2}(y~ - y)||
    subject to A_B' y~ = c_B, J = diag(A_B A_B') (1 on rows without an entry
    in B); checked against the KKT block system of that problem."""
    rng = np.random.default_rng(8)
    m, n = 6, 10
    A = rng.standard_normal((m, n))
    A[5, :3] = 0.0                                     # row 5 has no entry in B below
    x = np.zeros(n)
    x[:3] = 1.0
    z = np.full(n, 0.5)
    z[:3] = 0.0
    b, c, y = rng.standard_normal(m), rng.standard_normal(n), rng.standard_normal(m)
    _, yt, zt, B = X.polish(A, b, c, x, y, z)
    assert B.sum() == 3
    AB = A[:, B]
    J = (AB * AB).sum(axis=1)
    J[J == 0] = 1.0
    K = np.block([[np.diag(J), AB], [AB.T, np.zeros((3, 3))]])
    rhs = np.concatenate([np.zeros(m), c[B] - AB.T @ y])
    d = np.linalg.solve(K, rhs)[:m]
    np.testing.assert_allclose(yt, y + d, atol=1e-12)
    np.testing.assert_allclose(zt, c - A.T @ yt, atol=1e-12)
    assert yt[5] == pytest.approx(y[5], abs=1e-14)     # untouched: row 5 carries no constraint


def test_a_worse_polish_is_rejected():
    """A basic coordinate planted to look nonbasic (x_j halved, z_j = x*_j):
    the support guess misses it; on this seed the polished point is worse and
    the iterate is kept unchanged."""
    rng = np.random.default_rng(202)
    A, b, c, xs, ys, zs = _random_vertex_lp(rng, 4, 9)
    x, y, z = xs.copy(), ys.copy(), zs.copy()
    j = np.flatnonzero(xs > 0)[0]
    x[j], z[j] = 0.5 * xs[j], xs[j]
    xk, yk, zk, ok, before, after = X.polish_if_better(A, b, c, x, y, z)
    assert not ok and kkt.max_residual(after) > kkt.max_residual(before)
    assert (xk == x).all() and (yk == y).all() and (zk == z).all()


def test_empty_support_and_ties():
    """B = {x > z} is strict: ties x_j = z_j stay out, and with B empty the
    affine set {u = 0, A u = b} leaves x~ = 0, y~ = y (no constraint
    A_B' v = c_B to meet) and z~ = c - A'y."""
    rng = np.random.default_rng(9)
    m, n = 3, 6
    A = rng.standard_normal((m, n))
    b, c, y = rng.standard_normal(m), rng.standard_normal(n), rng.standard_normal(m)
    x = rng.uniform(0.0, 1.0, n)
    assert not X.support(x, x).any()
    xt, yt, zt, B = X.polish(A, b, c, x, y, x.copy())
    assert not B.any()
    assert (xt == 0.0).all()
    np.testing.assert_array_equal(yt, y)
    np.testing.assert_allclose(zt, c - A.T @ y, atol=1e-14)
    # one tie broken the other way enters B alone: x~ is then b's least-squares
    # multiple of that column
    z = x.copy()
    z[2] = x[2] - 0.1
    xt, _, _, B = X.polish(A, b, c, x, y, z)
    assert np.flatnonzero(B).tolist() == [2]
    a = A[:, 2]
    assert xt[2] == pytest.approx(a @ b / (a @ a), rel=1e-12)
    assert (xt[np.arange(n) != 2] == 0.0).all()
