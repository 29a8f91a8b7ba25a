"""GPU: the LP crossover polish (acs_polish) through the C ABI against the
oracle's polish (oracle/crossover.py) applied to the same iterate.

Tolerances: the oracle solves the two projections with dense least squares,
the device with FP64 Jacobi-PCG refinement rounds; both are accurate to a
few ulps times cond(A_B A_B') of the support's columns, so x~, y~, z~ are
compared at 1e-9 relative (1e-8 on the row-scaled planted LP, whose rows
span four decades) and the residuals of an accepted polish at 1e-11.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I, studies  # noqa: E402
from oracle import crossover as X, kkt, vertex  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))


def _solve_then_polish(inst, tol, rounds=3, **kw):
    with capi.Solver(inst, **kw) as s:
        st = s.solve(tol=tol, max_iter=20000)
        _, x, y, z, iters, res = s.get()
        pst, info = s.polish(rounds)
        _, xp, yp, zp, iters2, res2 = s.get()
    assert iters2 == iters
    return (st, x, y, z, res), (pst, info, xp, yp, zp, res2)


def _close(a, b, rtol):
    assert np.linalg.norm(a - b) <= rtol * (1.0 + np.linalg.norm(b)), np.abs(a - b).max()


def _dense_inst(A, b, c):
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    csr = sp.csr_matrix(A)
    nan_n, nan_m = np.full(n, np.nan), np.full(m, np.nan)
    return I.Instance(m=m, n=n, row_ptr=csr.indptr.astype(np.int64), col=csr.indices.astype(np.int32),
                      val=csr.data.astype(np.float64), b=np.asarray(b, float), c=np.asarray(c, float),
                      n_orth=n, soc_dims=np.zeros(0, np.int32), x_star=nan_n, y_star=nan_m, s_star=nan_n,
                      name="dense")


def test_worked_example_vertex():
    """From a 1e-3 iterate the polish lands on the enumerated vertex and the
    dual of its basis; the oracle's polish of the same iterate agrees."""
    A, b, c = np.array(GOLD["A"]), np.array(GOLD["b"]), np.array(GOLD["c"])
    inst = _dense_inst(A, b, c)
    (st, x, y, z, res), (pst, info, xp, yp, zp, res2) = _solve_then_polish(inst, 1e-3)
    assert pst == capi.SOLVED and info[5] == 1.0 and info[0] == 3
    xs = vertex.solve_lp(A, b, c)[0]
    _close(xp, xs, 1e-10)
    xo, yo, zo, _ = X.polish(A, b, c, x, y, z)
    _close(xp, xo, 1e-9)
    _close(yp, yo, 1e-9)
    _close(zp, zo, 1e-9)
    assert max(res2[:4]) <= 1e-11
    ours = kkt.residuals(sp.csr_matrix(A), b, c, xp, yp, zp, 5, [])
    assert kkt.max_residual(ours) <= 1e-11


@pytest.mark.parametrize("k", range(3))
def test_section_iv_a_lps(k):
    """Dense 80 x 100 LPs of Section IV-A's recipe (nondegenerate vertices)."""
    rp, col, val, b, c = studies.e2_instance(k)
    A = sp.csr_matrix((val, col, rp), shape=(80, 100)).toarray()
    inst = _dense_inst(A, b, c)
    (st, x, y, z, res), (pst, info, xp, yp, zp, res2) = _solve_then_polish(inst, 1e-4)
    xo, yo, zo, accept_o, before, after = X.polish_if_better(A, b, c, x, y, z)
    assert (pst == capi.SOLVED) == accept_o
    assert pst == capi.SOLVED
    _close(xp, xo, 1e-9)
    _close(yp, yo, 1e-9)
    _close(zp, zo, 1e-9)
    assert max(res2[:4]) <= 1e-11 and abs(max(res2[:4]) - kkt.max_residual(after)) <= 1e-11


def test_degenerate_planted_lp():
    """The small planted LP (|supp x*| = 150 < m = 200): x~ is unique; y~ only
    up to null(A_B'), where the oracle takes the J-metric least change and the
    device's factored M (m <= 4096) the solution with no component along the
    dropped pivots -- both solve A_B' y = c_B, which is what is compared."""
    inst = I.small_lp()
    A = inst.to_scipy()
    (st, x, y, z, res), (pst, info, xp, yp, zp, res2) = _solve_then_polish(
        inst, 1e-6, cond_first=300, cond_period=100)
    xo, yo, zo, accept_o, before, after = X.polish_if_better(A, inst.b, inst.c, x, y, z)
    assert info[0] == 150 and info[6] == 1.0
    assert pst == capi.SOLVED and accept_o
    _close(xp, xo, 1e-9)
    B = x > z
    Ad = A.toarray()
    assert np.abs(Ad[:, B].T @ yp - inst.c[B]).max() <= 1e-11
    _close(zp, inst.c - Ad.T @ yp, 1e-12)
    ours = kkt.residuals(A, inst.b, inst.c, xp, yp, zp, inst.n, [])
    assert kkt.max_residual(ours) <= 1e-12, ours
    assert abs(inst.c @ xp - inst.obj_star) <= 1e-10 * abs(inst.obj_star)


def test_planted_sparse_lp_with_row_scaling():
    """large_lp's recipe at 1 % (m = 2000, n = 10000, rows over four decades,
    |supp x*| = 3000 > m: y* unique, x~ the projection onto the face)."""
    inst = I.large_lp(scale=0.01)
    A = inst.to_scipy()
    (st, x, y, z, res), (pst, info, xp, yp, zp, res2) = _solve_then_polish(inst, 1e-4)
    xo, yo, zo, accept_o, before, after = X.polish_if_better(A, inst.b, inst.c, x, y, z)
    assert pst == capi.SOLVED and accept_o
    _close(xp, xo, 1e-8)
    _close(yp, yo, 1e-8)
    _close(zp, zo, 1e-8)
    assert max(res2[:4]) <= 1e-10
    assert abs(inst.c @ xp - inst.obj_star) <= 1e-9 * abs(inst.obj_star)


def test_large_lp_full_size():
    """m = 2e5, n = 1e6, nnz = 1e7 from a 1e-4 iterate: the polished point's
    residuals, re-evaluated by the oracle's FP64 residual function, and the
    planted objective."""
    inst = I.large_lp()
    A = inst.to_scipy()
    (st, x, y, z, res), (pst, info, xp, yp, zp, res2) = _solve_then_polish(inst, 1e-4)
    print("polish", info, res2[:4])
    assert pst == capi.SOLVED
    ours = kkt.residuals(A, inst.b, inst.c, xp, yp, zp, inst.n, [])
    assert kkt.max_residual(ours) <= 1e-9, ours
    assert abs(ours["obj_p"] - inst.obj_star) <= 1e-9 * abs(inst.obj_star)


def test_worse_polish_keeps_the_iterate():
    """Six iterations of the worked example: the support guess holds column 1,
    which is not in the optimal basis; the polished point is worse (the
    oracle's: 0.327 against 0.069) and the iterate stays as it was."""
    A, b, c = np.array(GOLD["A"]), np.array(GOLD["b"]), np.array(GOLD["c"])
    inst = _dense_inst(A, b, c)
    with capi.Solver(inst) as s:
        s.solve(tol=0.0, max_iter=6)
        _, x, y, z, _, res = s.get()
        pst, info = s.polish()
        _, x2, y2, z2, _, res2 = s.get()
        with pytest.raises(capi.AcsError):                      # state used as scratch
            capi.acs_get_state(s.h, 3, 5)
    _, _, _, accept_o, before, after = X.polish_if_better(A, b, c, x, y, z)
    assert pst == capi.POLISH_KEPT and not accept_o
    assert (x2 == x).all() and (y2 == y).all() and (z2 == z).all() and (res2 == res).all()


def test_polish_arguments_and_a_later_solve():
    inst = I.socp(scale=0.001)
    with capi.Solver(inst) as s:
        with pytest.raises(capi.AcsError):                      # before any solve; and not an LP
            s.polish()
    lp = I.small_lp()
    with capi.Solver(lp, cond_first=300, cond_period=100) as s:
        with pytest.raises(capi.AcsError):
            s.polish()                                          # no solve yet
        s.solve(tol=1e-6, max_iter=20000)
        _, x1, *_ = s.get()
        with pytest.raises(capi.AcsError):
            s.polish(rounds=9)
        s.polish()
        s.solve(tol=1e-6, max_iter=20000)                       # starts from x = z = e again
        _, x2, *_ = s.get()
        capi.acs_get_state(s.h, lp.m, lp.n)                     # the state is valid again
    np.testing.assert_array_equal(x1, x2)


def test_polished_solve_of_the_large_lp():
    """polish_tol = 1e-2: the solve stops after the first polish (taken, its
    solves stopped at 1e-7 of their first residual), well before the plain
    iteration would; the oracle's FP64 residual function and the planted
    objective agree, with a tenfold margin on the 1e-6 bar."""
    inst = I.large_lp()
    with capi.Solver(inst, polish_tol=1e-2) as s:
        st = s.solve(tol=1e-6, max_iter=20000)
        _, x, y, z, iters, res = s.get()
        pc = capi.acs_debug_pass_counts(s.h)
    assert st == capi.SOLVED
    assert pc["polish_attempts"] == 1 and pc["polish_taken"] == 1 and iters < 390
    ours = kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n, [])
    assert kkt.max_residual(ours) <= 1e-7, ours
    assert abs(ours["obj_p"] - inst.obj_star) <= 1e-7 * abs(inst.obj_star)


def test_polished_solve_resumes_the_iteration():
    """A dense LP of the Section V-A recipe (n = 400, m = 320, cached
    operator): the polishes at 1e-2 and 1e-3 do not reach tol (the support is
    not yet that of the vertex; the second is better than its iterate and
    still resumed from the iterate's state), the iteration resumes each time
    as if uninterrupted, and the polish at 1e-4 lands on the vertex.  The
    iteration count equals that of a plain solve to 1e-4; a polished solve
    whose only polish fails ends exactly like the plain solve."""
    inst = I.dense_lp(400)
    with capi.Solver(inst) as s:
        s.solve(tol=1e-4, max_iter=20000)
        _, x4, _, _, it4, _ = s.get()
        s.solve(tol=1e-3, max_iter=20000)
        _, x3, _, _, it3, _ = s.get()
    with capi.Solver(inst, polish_tol=1e-2) as s:
        st = s.solve(tol=1e-6, max_iter=20000)
        _, x, y, z, iters, res = s.get()
        pc = capi.acs_debug_pass_counts(s.h)
        st2 = s.solve(tol=1e-3, max_iter=20000)                  # the 1e-2 polish fails; the rest iterates
        _, x2, _, _, it2, _ = s.get()
    assert st == capi.SOLVED and pc["polish_taken"] >= 1 and pc["polish_attempts"] == 3
    assert pc["polish_factored"] == 3 and iters == it4
    ours = kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n, [])
    assert kkt.max_residual(ours) <= 1e-9, ours
    assert st2 == capi.SOLVED and it2 == it3
    np.testing.assert_allclose(x2, x3, rtol=0, atol=1e-12)


def test_empty_support():
    """b = 0, c > 0: the optimum is x* = 0, and after 7 iterations x < z on
    every column (in the oracle's iterate by at least 0.04), so the support B
    is empty: both projections start on a zero residual, x~ = 0, y~ = y (no
    constraint A_B' v = c_B to meet) and z~ = c - A'y, a point whose
    residuals are at rounding level, so the polish is taken."""
    rng = np.random.default_rng(31)
    m, n = 20, 60
    A = rng.standard_normal((m, n)) * (rng.uniform(size=(m, n)) < 0.3)
    b, c = np.zeros(m), rng.uniform(0.5, 1.5, n)
    inst = _dense_inst(A, b, c)
    with capi.Solver(inst) as s:
        s.solve(tol=0.0, max_iter=7)
        _, x, y, z, _, res = s.get()
        pst, info = s.polish()
        _, xp, yp, zp, _, res2 = s.get()
    assert not X.support(x, z).any() and (z - x).min() > 0.01
    assert pst == capi.SOLVED and info[0] == 0 and info[5] == 1.0
    assert (xp == 0.0).all()
    np.testing.assert_array_equal(yp, y)
    xo, yo, zo, B = X.polish(A, b, c, x, y, z)
    assert not B.any()
    _close(zp, zo, 1e-12)
    assert max(res2[:4]) <= 1e-13 < max(res[:4])
