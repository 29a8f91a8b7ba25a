"""GPU parity of the column-blocked FP32 passes and of the FP32 outer passes
(precision ACS_PREC_FP32), through the C ABI, against the FP64 CPU oracle.

Tolerances (the stated requirement of the method's hot path):
  * FP32 iterates (FP32 CG passes, and with ACS_PREC_FP32 also the outer
    iteration's two products in FP32): ||x_gpu - x_oracle|| / ||x_oracle||
    <= 1e-4 over the first 50 iterations under the paper's LP schedule;
  * end results: every relative KKT residual <= 1e-6 re-evaluated by the
    oracle's FP64 residual function; the objective within 1e-6 (relative)
    of the planted optimum, solving to 2e-7 (a residual of 1e-6 alone does
    not bound the objective error by 1e-6).
Block widths of 64 columns cut the small instances into many blocks with a
ragged last block, which the default width (49152 columns) reaches only at
full size (the full-size parity tests run with the default).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import alg, kkt  # noqa: E402

LP_SCHED = dict(cond_first=300, cond_period=100)
SOCP_SCHED = dict(t=1.7, cond_first=200, cond_period=100)


def _kkt_of(inst, x, y, z):
    return kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)


def _solve(inst, tol, max_iter, **kw):
    with capi.Solver(inst, **kw) as s:
        st = s.solve(tol=tol, max_iter=max_iter)
        rc, x, y, z, iters, res = s.get()
        lay = capi.acs_debug_layout(s.h)
        cnt = capi.acs_debug_pass_counts(s.h)
    return st, x, y, z, iters, res, lay, cnt


@pytest.mark.parametrize("col_block", [0, 64, 4])
@pytest.mark.parametrize("precision", [capi.PREC_MIXED, capi.PREC_FP32])
def test_first_50_iterates(precision, col_block):
    inst = I.small_lp()
    ref = alg.algorithm2(inst.to_scipy(), inst.b, inst.c, inst.n, [], L=alg.LP_SCHEDULE,
                         max_iter=50, tol=0.0, keep_x=50)
    worst = 0.0
    for k in (1, 2, 5, 20, 50):
        st, x, y, z, iters, res, lay, cnt = _solve(inst, 0.0, k, precision=precision, projection=capi.PROJ_CG,
                                                   col_block=col_block, cg_eta=1e-9, cg_tol=0.0, **LP_SCHED)
        assert st == capi.MAX_ITER and iters == k
        assert lay["col_blocked"] == 1
        if col_block:
            assert lay["A_blocks"] == -(-inst.n // lay["A_width"]) and lay["A_width"] <= col_block
            assert lay["At_blocks"] == -(-inst.m // lay["At_width"])
        if precision == capi.PREC_FP32:
            # every outer product of these iterations ran in FP32: the FP64
            # passes over A are b_tilde at the rescaling of l = 1 and the KKT checks
            assert cnt["fp32_outer_A"] == k and cnt["fp32_outer_At"] == k
            assert cnt["fp64_A"] == cnt["rescalings"] + cnt["checks"]
        xr = ref.x_history[k - 1]
        err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
        worst = max(worst, err)
        assert err <= 1e-4, (k, err)
    print("worst relative iterate error", worst)


@pytest.mark.parametrize("col_block", [0, 64])
@pytest.mark.parametrize("precision", [capi.PREC_MIXED, capi.PREC_FP32])
def test_small_lp_end_result(precision, col_block):
    inst = I.small_lp()
    st, x, y, z, iters, res, lay, cnt = _solve(inst, 2e-7, 20000, precision=precision, projection=capi.PROJ_CG,
                                               col_block=col_block, **LP_SCHED)
    assert st == capi.SOLVED, capi.acs_status_string(st)
    ours = _kkt_of(inst, x, y, z)
    assert kkt.max_residual(ours) <= 1e-6, ours
    assert abs(ours["obj_p"] - inst.obj_star) <= 1e-6 * abs(inst.obj_star)
    if precision == capi.PREC_FP32:
        assert cnt["fp32_outer_At"] > 0
        # the FP64 products finished the solve
        assert cnt["outer32_end"] > 0 and cnt["fp64_At"] > 0


@pytest.mark.parametrize("precision", [capi.PREC_MIXED, capi.PREC_FP32])
def test_small_socp_end_result(precision):
    """Orthant and Lorentz cones of sizes 3..64 (scaled SOCP recipe), many blocks."""
    inst = I.socp(scale=0.002)
    st, x, y, z, iters, res, lay, cnt = _solve(inst, 2e-7, 20000, precision=precision, col_block=128,
                                               projection=capi.PROJ_CG, **SOCP_SCHED)
    assert st == capi.SOLVED, capi.acs_status_string(st)
    assert lay["col_blocked"] == 1 and lay["A_blocks"] > 1 and lay["At_blocks"] > 1
    ours = _kkt_of(inst, x, y, z)
    assert kkt.max_residual(ours) <= 1e-6, ours
    assert abs(ours["obj_p"] - inst.obj_star) <= 1e-6 * (1 + abs(inst.obj_star))


def test_medium_socp_iterates_default_width():
    """A tenth of the SOCP recipe (n ~ 77000 > 49152 columns): two blocks at
    the default width on A, the first 20 iterates against the oracle's
    (Jacobi CG to 1e-13 in FP64)."""
    inst = I.socp(scale=0.1)
    ref = alg.algorithm2(inst.to_scipy(), inst.b, inst.c, inst.n_orth, inst.soc_dims, t=1.7,
                         L=alg.SOCP_SCHEDULE, max_iter=20, tol=0.0, keep_x=20, solver="cg")
    for precision in (capi.PREC_MIXED, capi.PREC_FP32):
        for k in (1, 20):
            st, x, y, z, iters, res, lay, cnt = _solve(inst, 0.0, k, precision=precision, cg_eta=1e-9,
                                                       cg_tol=0.0, col_block=0, **SOCP_SCHED)
            assert lay["col_blocked"] == 1 and lay["A_blocks"] == 2
            xr = ref.x_history[k - 1]
            err = np.linalg.norm(x - xr) / np.linalg.norm(xr)
            assert err <= 1e-4, (precision, k, err)


def test_layout_switches():
    """The column-blocked image is built when asked for, unless A is stored
    in BF16 or the cached operator runs from the first iteration."""
    inst = I.small_lp()
    for kw, want in ((dict(projection=capi.PROJ_CG, col_block=0), 1), (dict(projection=capi.PROJ_CG, col_block=-1), 0),
                     (dict(projection=capi.PROJ_CG, col_block=0, a_storage=capi.STORE_BF16), 0),
                     (dict(col_block=0), 0)):
        with capi.Solver(inst, **kw) as s:
            assert capi.acs_debug_layout(s.h)["col_blocked"] == want, kw


def test_blocked_and_l2_layouts_agree():
    """The same solve (CG projection) with the column-blocked passes and with
    the L2-gather passes ends at the same point (to the tolerance of the
    stopping test)."""
    inst = I.socp(scale=0.002)
    out = []
    for cb in (-1, 0, 32):
        st, x, y, z, iters, res, lay, cnt = _solve(inst, 2e-7, 20000, col_block=cb, projection=capi.PROJ_CG,
                                                   **SOCP_SCHED)
        assert st == capi.SOLVED
        assert lay["col_blocked"] == (cb >= 0)
        out.append(_kkt_of(inst, x, y, z)["obj_p"])
    assert max(out) - min(out) <= 1e-6 * (1 + abs(inst.obj_star))
