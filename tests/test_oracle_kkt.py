"""Pins for the oracle's KKT residuals (Eqs. 19a-19c) against planted optima."""
import numpy as np
import pytest

from oracle import kkt
from paper_2103_00736_gb300 import instances as I


def _planted():
    yield I.small_lp()
    yield I.large_lp(scale=0.002)
    yield I.socp(scale=0.002)
    yield I.bernoulli_lp(I.seed_for(I.K_BATCH, 7), 60, 150)
    yield I.serve_request(3, mmax=300)


@pytest.mark.parametrize("idx", range(5))
def test_planted_optimum_has_zero_residual(idx):
    inst = list(_planted())[idx]
    A = inst.to_scipy()
    res = kkt.residuals(A, inst.b, inst.c, inst.x_star, inst.y_star, inst.s_star,
                        inst.n_orth, inst.soc_dims)
    assert kkt.max_residual(res) < 1e-13
    assert abs(res["obj_p"] - res["obj_d"]) <= 1e-10 * (1 + abs(res["obj_p"]))


def test_perturbations_are_detected():
    inst = I.socp(scale=0.002)
    A = inst.to_scipy()
    rng = np.random.default_rng(0)
    base = (inst.x_star, inst.y_star, inst.s_star)
    for which, key in [(0, "r_p"), (1, "r_d"), (2, "r_d")]:
        args = [v.copy() for v in base]
        args[which] += 1e-3 * rng.standard_normal(args[which].size)
        res = kkt.residuals(A, inst.b, inst.c, *args, inst.n_orth, inst.soc_dims)
        assert res[key] > 1e-6
    # leaving the cone is seen by r_cone
    x = inst.x_star.copy()
    x[0] = -1.0
    res = kkt.residuals(A, inst.b, inst.c, x, inst.y_star, inst.s_star, inst.n_orth, inst.soc_dims)
    assert res["r_cone"] > 1e-3
    # scaling x and s together breaks the gap but not membership
    res = kkt.residuals(A, inst.b, inst.c, 1.1 * inst.x_star, inst.y_star, inst.s_star,
                        inst.n_orth, inst.soc_dims)
    assert res["r_gap"] > 1e-3 and res["r_cone"] < 1e-14


def test_yfree_gap_is_the_duality_gap_of_any_dual_pair():
    """Eq. (15b) without y: for z = c - A'y and Ax = b, (A^dagger b)'(c - z)
    = b'(AA')^{-1} A A' y = b'y, so the y-free gap is |b'y - c'x| for every
    y, and zero at the planted optimum."""
    rng = np.random.default_rng(3)
    for inst in (I.small_lp(), I.socp(scale=0.002)):
        A = inst.to_scipy()
        assert kkt.yfree_gap(A, inst.b, inst.c, inst.x_star, inst.s_star) <= \
            1e-9 * (1 + abs(inst.obj_star))
        for _ in range(3):
            y = inst.y_star + rng.standard_normal(inst.m)
            z = inst.c - A.T @ y
            g = kkt.yfree_gap(A, inst.b, inst.c, inst.x_star, z)
            assert abs(g - abs(inst.b @ y - inst.c @ inst.x_star)) <= 1e-8 * (1 + abs(g))
    # with a z that is not of the form c - A'y only the row-space part counts
    inst = I.small_lp()
    A = inst.to_scipy()
    u = rng.standard_normal(inst.n)
    P = A.T @ np.linalg.lstsq(A.toarray().T, u, rcond=None)[0]     # row-space part of u
    g1 = kkt.yfree_gap(A, inst.b, inst.c, inst.x_star, inst.s_star + u)
    g2 = kkt.yfree_gap(A, inst.b, inst.c, inst.x_star, inst.s_star + P)
    assert abs(g1 - g2) <= 1e-9 * (1 + g1) and g1 > 1e-3
