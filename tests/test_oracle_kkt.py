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
