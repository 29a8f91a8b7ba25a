"""GPU parity on the paper's dense workloads (Section V-A LPs, Section V-C
SOCPs with Lorentz cones of size 4 and 10), through the C ABI, against the
FP64 CPU oracle.  These instances have no planted optimum: the objective is
compared with the oracle's own solution, both solved to 2e-7 (a residual of
1e-6 alone does not bound the objective error by 1e-6); the GPU's point is
re-evaluated by the oracle's residual function (every residual <= 1e-6).
First iterates: FP64 with the cached operator (exact projections, like the
oracle's) within 1e-9; the FP32 correction CG within 1e-4."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import alg, kkt  # noqa: E402

LP = dict(t=9.2, cond_first=300, cond_period=100)
SOCP = dict(t=1.7, cond_first=200, cond_period=100)


def _solve(x, tol, max_iter, **kw):
    with capi.Solver(x, **kw) as s:
        st = s.solve(tol=tol, max_iter=max_iter)
        rc, xs, ys, zs, iters, res = s.get()
    return st, xs, ys, zs, iters


def _case(kind, n, h=None):
    if kind == "lp":
        x = I.dense_lp(n)
        return x, LP, alg.LP_SCHEDULE, 9.2
    x = I.dense_socp(n, h)
    return x, SOCP, alg.SOCP_SCHEDULE, 1.7


@pytest.mark.parametrize("kind,n,h", [("lp", 100, None), ("lp", 400, None), ("socp", 100, 4),
                                      ("socp", 400, 10), ("socp", 800, 4)])
@pytest.mark.parametrize("projection", [capi.PROJ_AUTO, capi.PROJ_CG])
def test_dense_end_result(kind, n, h, projection):
    x, sched, L, t = _case(kind, n, h)
    A = x.to_scipy()
    ref = alg.algorithm2(A, x.b, x.c, x.n_orth, x.soc_dims, t=t, L=L, max_iter=20000, tol=2e-7, check_every=10)
    assert ref.status == "solved"
    st, xs, ys, zs, iters = _solve(x, 2e-7, 20000, projection=projection, **sched)
    assert st == capi.SOLVED, capi.acs_status_string(st)
    ours = kkt.residuals(A, x.b, x.c, xs, ys, zs, x.n_orth, x.soc_dims)
    assert kkt.max_residual(ours) <= 1e-6, ours
    assert abs(ours["obj_p"] - ref.res["obj_p"]) <= 1e-6 * (1 + abs(ref.res["obj_p"])), (ours, ref.res)


@pytest.mark.parametrize("kind,n,h", [("lp", 200, None), ("socp", 200, 10)])
def test_dense_first_iterates(kind, n, h):
    x, sched, L, t = _case(kind, n, h)
    A = x.to_scipy()
    ref = alg.algorithm2(A, x.b, x.c, x.n_orth, x.soc_dims, t=t, L=L, max_iter=30, tol=0.0, keep_x=30)
    for prec, proj, rtol in ((capi.PREC_FP64, capi.PROJ_DENSE, 1e-9), (capi.PREC_MIXED, capi.PROJ_CG, 1e-4)):
        for k in (1, 10, 30):
            st, xs, ys, zs, iters = _solve(x, 0.0, k, precision=prec, projection=proj, cg_eta=1e-9, cg_tol=0.0,
                                           **sched)
            xr = ref.x_history[k - 1]
            err = np.linalg.norm(xs - xr) / np.linalg.norm(xr)
            assert err <= rtol, (prec, k, err)


def test_dense_lp_with_full_rows_above_the_sparse_limit():
    """m = 1200 > dense_switch_max_m: with full rows the solve may switch to
    the cached operator (its M assembled by the tiled FP64 product) when CG
    stalls; end result against the oracle's objective, and, with the cached
    operator from the first iteration, the oracle's exact first iterates."""
    x, sched, L, t = _case("lp", 1500)
    A = x.to_scipy()
    ref = alg.algorithm2(A, x.b, x.c, x.n_orth, x.soc_dims, t=t, L=L, max_iter=20000, tol=2e-7, check_every=10,
                         keep_x=10)
    assert ref.status == "solved"
    with capi.Solver(x, **sched) as s:
        st = s.solve(tol=2e-7, max_iter=20000)
        _, xs, ys, zs, iters, res = s.get()
        pc = capi.acs_debug_pass_counts(s.h)
    assert st == capi.SOLVED
    ours = kkt.residuals(A, x.b, x.c, xs, ys, zs, x.n_orth, x.soc_dims)
    assert kkt.max_residual(ours) <= 1e-6, ours
    assert abs(ours["obj_p"] - ref.res["obj_p"]) <= 1e-6 * (1 + abs(ref.res["obj_p"]))
    st, xs, _, _, _ = _solve(x, 0.0, 10, precision=capi.PREC_FP64, projection=capi.PROJ_DENSE, **sched)
    assert np.linalg.norm(xs - ref.x_history[9]) <= 1e-9 * np.linalg.norm(ref.x_history[9])
