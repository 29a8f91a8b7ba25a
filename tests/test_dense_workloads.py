"""The paper's dense workloads (Sections V-A and V-C) on the host: the
generators follow the printed recipes, and the oracle solves small instances
(the LP against HiGHS, the SOCP by its KKT certificate)."""
import numpy as np
import pytest

from oracle import alg, cones as C, kkt
from paper_2103_00736_gb300 import instances as I


@pytest.mark.parametrize("n", [100, 250])
def test_dense_lp_recipe(n):
    x = I.dense_lp(n)
    m = int(np.floor(0.8 * n))
    assert (x.m, x.n, x.nnz, x.n_orth, len(x.soc_dims)) == (m, n, m * n, n, 0)
    A = x.to_scipy().toarray()
    assert A.min() >= -1.0 and A.max() <= 1.0 and np.all(A != 0)
    rng = np.random.default_rng(I.seed_for(I.K_DENSE, n))      # the draws, in the printed order
    A2 = rng.uniform(-1.0, 1.0, size=(m, n))
    xdot = rng.standard_normal(n)
    c = rng.standard_normal(n)
    assert np.array_equal(A, A2) and np.array_equal(x.c, c)
    np.testing.assert_allclose(x.b, A2 @ np.abs(xdot), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("h", [4, 10])
def test_dense_socp_recipe(h):
    n = 20 * h
    x = I.dense_socp(n, h)
    assert (x.m, x.n_orth) == ((4 * n) // 5, 0) and np.all(x.soc_dims == h) and x.soc_dims.sum() == n
    A = x.to_scipy().toarray()
    assert A.min() >= -1.0 and A.max() <= 1.0
    assert x.c.min() >= 0.0 and x.c.max() <= 1.0
    # the reflection used for b is the oracle's abs_K (Definition 1)
    v = np.random.default_rng(5).uniform(-1.0, 1.0, size=n)
    np.testing.assert_allclose(I._lorentz_reflection(v, h), C.abs_K(v, 0, x.soc_dims), rtol=1e-14, atol=1e-15)


def test_dense_lp_oracle_matches_highs():
    from scipy.optimize import linprog
    x = I.dense_lp(100)
    A = x.to_scipy()
    r = alg.algorithm2(A, x.b, x.c, x.n, [], L=alg.LP_SCHEDULE, max_iter=20000, tol=1e-8, check_every=10)
    hi = linprog(x.c, A_eq=A, b_eq=x.b, bounds=(0, None), method="highs")
    assert r.status == "solved" and hi.status == 0
    assert abs(r.res["obj_p"] - hi.fun) <= 1e-6 * (1 + abs(hi.fun))


@pytest.mark.parametrize("h", [4, 10])
def test_dense_socp_oracle_certificate(h):
    x = I.dense_socp(100, h)
    A = x.to_scipy()
    r = alg.algorithm2(A, x.b, x.c, 0, x.soc_dims, t=1.7, L=alg.SOCP_SCHEDULE, max_iter=20000, tol=1e-7,
                       check_every=10)
    assert r.status == "solved"
    res = kkt.residuals(A, x.b, x.c, r.x, r.y, r.z, 0, x.soc_dims)
    assert kkt.max_residual(res) <= 1e-7
