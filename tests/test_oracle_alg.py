"""Pins for the oracle's Algorithms 1 and 2 against ground truth the paper and
mathematics fix: the paper's worked example (Section III-A) solved by vertex
enumeration, random tiny LPs by vertex enumeration, an independent LP solver
(HiGHS via scipy), planted optima, a closed-form SOCP, the textbook
Douglas-Rachford step, Lemma 2's fixed point and Lemma 3's monotonicity.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import alg, cones as C, kkt, vertex
from oracle.subspace import Subspace
from paper_2103_00736_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")
SCHEDS = {
    "none": alg.NO_SCHEDULE,
    "lp": alg.LP_SCHEDULE,
    "first50": alg.Schedule(explicit=tuple(range(1, 51))),
}


def _worked():
    g = json.load(open(GOLDEN))
    return g, np.array(g["A"]), np.array(g["b"]), np.array(g["c"])


def test_worked_example_fixture_matches_printed_condition_numbers():
    g, A, b, c = _worked()
    assert abs(np.linalg.cond(A) - g["cond_A"]) < 0.05
    assert abs(np.linalg.cond(A @ np.diag(g["E_AC"])) - g["cond_AC"]) < 0.1
    # D^SK, E^SK are printed to 4 digits, so only 0.1% agreement is possible
    sk = np.linalg.cond(np.diag(g["D_SK"]) @ A @ np.diag(g["E_SK"]))
    assert abs(sk - g["cond_SK"]) / g["cond_SK"] < 1e-3


@pytest.mark.parametrize("sched", list(SCHEDS))
def test_worked_example_reaches_vertex_optimum(sched):
    g, A, b, c = _worked()
    x_ref, obj_ref, bases = vertex.solve_lp(A, b, c)
    assert bases == [(2, 3, 4)]      # unique optimal basis: columns 3, 4, 5
    r = alg.algorithm2(A, b, c, 5, [], mu=g["mu"], t=9.2, L=SCHEDS[sched], max_iter=20000, tol=1e-8)
    assert r.status == "solved"
    assert abs(r.res["obj_p"] - obj_ref) <= 1e-6 * abs(obj_ref) + 1e-8
    np.testing.assert_allclose(r.x, x_ref, atol=1e-6)


def test_worked_example_conditioning_fewer_iterations():
    g, A, b, c = _worked()
    it = {k: alg.algorithm2(A, b, c, 5, [], L=v, max_iter=20000, tol=1e-6).iters
          for k, v in SCHEDS.items()}
    assert it["first50"] < it["none"]


def _tiny_lp(rng, m, n):
    A = rng.standard_normal((m, n))
    x0 = rng.uniform(0.0, 1.0, n) * (rng.random(n) < 0.7)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.1, 1.0, n)
    return A, A @ x0, A.T @ y0 + s0


@pytest.mark.parametrize("seed", range(8))
def test_tiny_lp_matches_vertex_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(2, 7)), int(rng.integers(7, 13))
    A, b, c = _tiny_lp(rng, m, n)
    x_ref, obj_ref, bases = vertex.solve_lp(A, b, c)
    r = alg.algorithm2(A, b, c, n, [], L=SCHEDS["first50"], max_iter=50000, tol=1e-9)
    assert r.status == "solved"
    assert abs(r.res["obj_p"] - obj_ref) <= 1e-6 * (1 + abs(obj_ref))
    if len(bases) == 1:
        np.testing.assert_allclose(r.x, x_ref, atol=1e-5)


def test_small_lp_matches_planted_optimum_and_highs():
    from scipy.optimize import linprog
    inst = I.small_lp()
    A = inst.to_scipy()
    hi = linprog(inst.c, A_eq=A, b_eq=inst.b, bounds=(0, None), method="highs")
    assert hi.status == 0
    assert abs(hi.fun - inst.obj_star) <= 1e-8 * abs(inst.obj_star)
    for sched in ("lp", "first50"):
        r = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=SCHEDS[sched], max_iter=5000, tol=1e-6)
        assert r.status == "solved"
        assert abs(r.res["obj_p"] - inst.obj_star) <= 1e-6 * abs(inst.obj_star)
        # |supp x*| = 150 < m: x* is unique
        assert np.linalg.norm(r.x - inst.x_star) <= 1e-4 * np.linalg.norm(inst.x_star)


def test_socp_closed_form():
    # min x1 s.t. x2 = 1, x3 = 1, x in K_3: optimum x = (sqrt 2, 1, 1), y = (1, 1)/sqrt 2
    A = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    b = np.array([1.0, 1.0])
    c = np.array([1.0, 0.0, 0.0])
    r = alg.algorithm2(A, b, c, 0, [3], t=1.7, L=alg.SOCP_SCHEDULE, max_iter=20000, tol=1e-9)
    assert r.status == "solved"
    np.testing.assert_allclose(r.x, [math.sqrt(2), 1, 1], atol=1e-7)
    np.testing.assert_allclose(r.y, [1 / math.sqrt(2)] * 2, atol=1e-7)


def test_small_socp_planted():
    inst = I.socp(scale=0.002)
    A = inst.to_scipy()
    r = alg.algorithm2(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, t=1.7,
                       L=alg.SOCP_SCHEDULE, max_iter=20000, tol=1e-7, check_every=10)
    assert r.status == "solved"
    assert abs(r.res["obj_p"] - inst.obj_star) <= 1e-6 * (1 + abs(inst.obj_star))


def _dr_textbook_step(A, b, c, s, mu, n_orth, dims):
    """z <- z + prox_{mu g}(2 prox_f(z) - z) - prox_f(z) (Section III-A), with
    prox_{mu g}(v) = argmin mu c'x + |x - v|^2/2 s.t. Ax = b from its KKT block system."""
    m, n = A.shape
    pk = C.proj_K(s, n_orth, dims)
    v = 2 * pk - s
    K = np.block([[np.eye(n), A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([v - mu * c, b]))
    return s + sol[:n] - pk


@pytest.mark.parametrize("mu", [1.0, 0.3])
def test_algorithm1_step_is_douglas_rachford(mu):
    rng = np.random.default_rng(11)
    inst = I.socp(scale=0.0005)
    A = inst.to_scipy().toarray()
    s = rng.standard_normal(inst.n)
    _, _, s1, _, _ = alg.algorithm1(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=mu, s0=s, iters=1)
    ref = _dr_textbook_step(A, inst.b, inst.c, s, mu, inst.n_orth, inst.soc_dims)
    np.testing.assert_allclose(s1, ref, atol=1e-10 * (1 + np.abs(ref).max()))


def _star(u, sub, n_orth, dims):
    return sub.abs(C.abs_K(u, n_orth, dims))


def test_lemma1_star_operator():
    inst = I.socp(scale=0.0005)
    sub = Subspace(inst.to_scipy(), np.ones(inst.n))
    rng = np.random.default_rng(12)
    for _ in range(20):
        u, v = rng.standard_normal(inst.n), rng.standard_normal(inst.n)
        su, sv = _star(u, sub, inst.n_orth, inst.soc_dims), _star(v, sub, inst.n_orth, inst.soc_dims)
        assert abs(np.linalg.norm(su) - np.linalg.norm(u)) < 1e-10 * np.linalg.norm(u)
        assert su @ sv >= u @ v - 1e-10 * np.linalg.norm(u) * np.linalg.norm(v)


@pytest.mark.parametrize("mu", [1.0, 2.0])
def test_lemma2_fixed_point(mu):
    inst = I.socp(scale=0.0005)
    A = inst.to_scipy()
    s_opt = inst.x_star - mu * inst.s_star
    x, z, s, p, d = alg.algorithm1(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=mu, s0=s_opt, iters=3)
    np.testing.assert_allclose(s, s_opt, atol=1e-10)
    np.testing.assert_allclose(x, inst.x_star, atol=1e-10)
    np.testing.assert_allclose(z, inst.s_star, atol=1e-10)
    sub = Subspace(A, np.ones(inst.n))
    np.testing.assert_allclose(d, 0.5 * (s_opt + _star(s_opt, sub, inst.n_orth, inst.soc_dims)), atol=1e-10)


def test_lemma3_fejer_monotone_between_conditionings():
    inst = I.small_lp()
    A = inst.to_scipy()
    mu = 1.0
    L = alg.Schedule(explicit=(1, 40, 80))
    dist, steps = [], []
    prev = {}

    def hook(l, s, p, O, d):
        s_opt = inst.x_star / O - mu * O * inst.s_star
        dist.append((l, np.linalg.norm(s - s_opt), O.copy()))

    alg.algorithm2(A, inst.b, inst.c, inst.n, [], mu=mu, L=L, max_iter=120, tol=0.0, on_iter=hook)
    # the distance settles at a positive constant (z* is not unique here), where
    # successive changes reach the rounding level of the solve with M (cond ~1e8
    # once O spreads over e^9.2): allow 1e-8 relative slack
    n_checked = 0
    for (l0, d0, O0), (l1, d1, O1) in zip(dist[:-1], dist[1:]):
        if np.array_equal(O0, O1):
            assert d1 <= d0 * (1 + 1e-8), (l0, d0, d1)
            n_checked += 1
    assert n_checked > 100


def test_lemma3_summable_steps():
    inst = I.small_lp()
    A = inst.to_scipy()
    s_opt = inst.x_star - inst.s_star
    sub = Subspace(A, np.ones(inst.n))
    d = sub.pinv_t(inst.b) + 0.5 * (sub.abs(inst.c) - inst.c)
    s = np.zeros(inst.n)
    total = 0.0
    for _ in range(300):
        p = C.abs_K(s, inst.n, [])
        s_new = 0.5 * s - 0.5 * sub.abs(p) + d
        total += np.sum((s_new - s) ** 2)
        s = s_new
    assert total <= np.sum(s_opt ** 2) * (1 + 1e-10)


def test_conditioning_rule():
    rng = np.random.default_rng(13)
    n_orth, dims = 4, [3, 5]
    x = np.abs(rng.standard_normal(12)) + 0.1
    z = np.abs(rng.standard_normal(12)) + 0.1
    o = alg.conditioning_vector(x, z, n_orth, dims)
    # constant on each cone, equal to |x1 - |xbar|| / |z1|
    off = C.soc_offsets(n_orth, dims)
    for a, e in zip(off[:-1], off[1:]):
        assert np.all(o[a:e] == o[a])
        np.testing.assert_allclose(o[a], abs(x[a] - np.linalg.norm(x[a + 1:e])) / abs(z[a]))
    np.testing.assert_allclose(o[:4], x[:4] / z[:4])
    # spread of O is capped at e^t; exponent 1 when already within the cap
    for t in (0.5, 1.7, 9.2):
        O, a = alg.conditioning_matrix(x * np.exp(rng.uniform(-20, 20, 12)), z, n_orth, dims, t)
        assert math.log(O.max() / O.min()) <= t * (1 + 1e-12)
    O, a = alg.conditioning_matrix(x, z, n_orth, dims, 100.0)
    assert a == 1.0
    np.testing.assert_allclose(O, o)
    # o in {0, inf, nan} carries no scale: the exponent comes from the finite o,
    # and o = inf / 0 / nan take the largest / smallest / middle scale under the cap
    z0 = z.copy(); z0[0] = 0.0                      # o_0 = inf
    x0 = x.copy(); x0[1] = 0.0                      # o_1 = 0
    x0[2] = 0.0; z0[2] = 0.0                        # o_2 = nan
    O, a = alg.conditioning_matrix(x0, z0, n_orth, dims, 9.2)
    fin = alg.conditioning_vector(x, z, n_orth, dims)[3:]
    assert a == alg.conditioning_exponent(fin, 9.2) and 0.0 < a <= 1.0
    assert O[0] == O[3:].max() and O[1] == O[3:].min()
    np.testing.assert_allclose(O[2], np.sqrt(O[3:].max() * O[3:].min()))
    assert np.all(np.isfinite(O)) and math.log(O.max() / O.min()) <= 9.2 * (1 + 1e-12)
    # nothing finite at all: O = I
    O, a = alg.conditioning_matrix(np.zeros(12), np.zeros(12), n_orth, dims, 9.2)
    assert np.all(O == 1.0)
    # all equal: exponent 1
    assert alg.conditioning_exponent(np.full(5, 3.0), 9.2) == 1.0


def test_literal_step11_switches_rescaling_off():
    """Step 11 evaluated as printed: an o of 0 or inf makes the log spread
    infinite, the exponent 0 and O = I (0^0 = inf^0 = 1); with nan as the
    only non-finite entry the exponent stays positive and O gets a nan.  On
    an instance with an empty column (x_j -> 0, z_j -> c_j > 0, so o_j = 0 from
    the second rescaling on) the literal rule therefore reproduces the run
    with no rescaling at all, iterate for iterate, while the oracle's rule
    keeps rescaling."""
    rng = np.random.default_rng(21)
    x = np.abs(rng.standard_normal(6)) + 0.1
    z = np.abs(rng.standard_normal(6)) + 0.1
    for bad_x, bad_z in ((0.0, 1.0), (1.0, 0.0)):            # o = 0, o = inf
        x0, z0 = x.copy(), z.copy()
        x0[2], z0[2] = bad_x, bad_z
        O, a = alg.conditioning_matrix_literal(x0, z0, 6, [], 9.2)
        assert a == 0.0 and np.all(O == 1.0)
    x0, z0 = x.copy(), z.copy()
    x0[2] = z0[2] = 0.0                                       # o = nan only
    O, a = alg.conditioning_matrix_literal(x0, z0, 6, [], 9.2)
    assert a > 0.0 and np.isnan(O[2]) and np.all(np.isfinite(np.delete(O, 2)))
    # without non-finite o both rules agree
    O1, a1 = alg.conditioning_matrix_literal(x, z, 6, [], 1.0)
    O2, a2 = alg.conditioning_matrix(x, z, 6, [], 1.0)
    assert a1 == a2 and np.allclose(O1, O2, rtol=1e-14)
    # an empty column with c_j = 0.7
    inst = I.small_lp()
    n = inst.n + 1
    A = sp.hstack([inst.to_scipy(), sp.csr_matrix((inst.m, 1))]).tocsr()
    c = np.concatenate([inst.c, [0.7]])
    lit = alg.algorithm2(A, inst.b, c, n, [], L=alg.LP_SCHEDULE, max_iter=420, tol=0.0, keep_x=420,
                         rule="literal")
    off = alg.algorithm2(A, inst.b, c, n, [], L=alg.NO_SCHEDULE, max_iter=420, tol=0.0, keep_x=420)
    ours = alg.algorithm2(A, inst.b, c, n, [], L=alg.LP_SCHEDULE, max_iter=420, tol=0.0)
    assert [a for _, _, a in lit.O_history] == [1.0, 0.0, 0.0]
    for k in (299, 300, 301, 420):
        np.testing.assert_allclose(lit.x_history[k - 1], off.x_history[k - 1], rtol=0, atol=1e-12)
    assert [l for l, _, _ in ours.O_history] == [1, 300, 400]
    assert all(0.0 < a < 1.0 for _, _, a in ours.O_history[1:])


def test_schedule_sets_of_the_paper():
    """The periodic part of L as the paper states it: {300, 400, ...} for its
    LPs (Section V-A), {200, 300, ...} for its SOCPs (Section V-C), plus
    l = 1 (step 4).  The sets are written out here for l <= 1000 and compared
    with Schedule's membership test and with the iterations at which
    algorithm2 actually rescales."""
    lp = {1, 300, 400, 500, 600, 700, 800, 900, 1000}
    socp = {1, 200, 300, 400, 500, 600, 700, 800, 900, 1000}
    assert {l for l in range(1, 1001) if l in alg.LP_SCHEDULE} | {1} == lp
    assert {l for l in range(1, 1001) if l in alg.SOCP_SCHEDULE} | {1} == socp
    assert 1 not in alg.LP_SCHEDULE and 299 not in alg.LP_SCHEDULE and 301 not in alg.LP_SCHEDULE
    assert [l for l in range(1, 60) if l in alg.Schedule(first=5, period=7)] == [5, 12, 19, 26, 33, 40, 47, 54]
    assert [l for l in range(1, 60) if l in alg.Schedule(first=5)] == [5]
    assert [l for l in range(1, 60) if l in alg.Schedule(explicit=(3, 9), first=50, period=4)] == [3, 9, 50, 54, 58]
    # the iterations at which Algorithm 2 rescales, on a tiny LP run to l = 1000
    rng = np.random.default_rng(3)
    A = sp.csr_matrix(rng.standard_normal((3, 6)))
    xs = np.abs(rng.standard_normal(6))
    b = A @ xs
    c = np.abs(rng.standard_normal(6)) + 0.5
    for L, want in ((alg.LP_SCHEDULE, lp), (alg.SOCP_SCHEDULE, socp)):
        r = alg.algorithm2(A, b, c, 6, [], L=L, max_iter=1000, tol=0.0, check_every=10 ** 9)
        assert {l for l, _, _ in r.O_history} == want


def test_recast_is_identity_when_O_unchanged():
    # step 14 applied with the O that produced x, z (steps 20-21) returns the same s
    inst = I.small_lp()
    A = inst.to_scipy()
    seen = {}

    def hook(l, s, p, O, d):
        seen["s"], seen["p"], seen["O"] = s.copy(), p.copy(), O.copy()

    alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=SCHEDS["first50"], max_iter=7, tol=0.0, on_iter=hook)
    s, p, O = seen["s"], seen["p"], seen["O"]
    x = O * (p + s) / 2
    z = (p - s) / (O * 2)
    np.testing.assert_allclose(x / O - O * z, s, atol=1e-12)


def test_row_scaling_invariance():
    """range((RA)') = range(A') and (RA)^dagger (Rb) = A^dagger b: the iterates do
    not depend on a row scaling R.  Checked to rounding while O = I; once O
    follows x/z the rounding differences are amplified, so there only the
    converged objective is compared."""
    inst = I.small_lp()
    A = inst.to_scipy()
    R = 10.0 ** np.random.default_rng(14).uniform(-2, 2, inst.m)
    RA = sp.diags(R) @ A
    r1 = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=SCHEDS["lp"], max_iter=40, tol=0.0)
    r2 = alg.algorithm2(RA, R * inst.b, inst.c, inst.n, [], L=SCHEDS["lp"], max_iter=40, tol=0.0)
    np.testing.assert_allclose(r1.x, r2.x, atol=1e-12 * np.abs(r1.x).max())
    r1 = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=SCHEDS["first50"], max_iter=500, tol=1e-8)
    r2 = alg.algorithm2(RA, R * inst.b, inst.c, inst.n, [], L=SCHEDS["first50"], max_iter=500, tol=1e-8)
    assert abs(r1.res["obj_p"] - r2.res["obj_p"]) <= 1e-7 * abs(r1.res["obj_p"])


@pytest.mark.slow
def test_conditioning_schedule_ordering():
    """Section IV-A: ten dense 80 x 100 LPs (A, c ~ N(0,1), b = A xdot, xdot ~
    U[0,1]), t = 9.2.  Conditioning at the first 50 iterations beats one
    conditioning at l = 300, which beats none.  Compared on the median
    iteration count to KKT <= 1e-6 over six seeded instances (an instance that
    does not converge within 6000 iterations counts as 6001)."""
    from scipy.optimize import linprog
    cap = 6000
    its = {"first50": [], "one300": [], "none": []}
    for seed in range(6):
        rp, col, val, b, c = I.paper_e2_lp(I.seed_for(I.K_SMALL_LP, 50 + seed))
        A = sp.csr_matrix((val, col, rp), shape=(80, 100))
        hi = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
        assert hi.status == 0
        for k, L in [("first50", SCHEDS["first50"]), ("one300", alg.Schedule(explicit=(300,))),
                     ("none", alg.NO_SCHEDULE)]:
            r = alg.algorithm2(A, b, c, 100, [], L=L, max_iter=cap, tol=1e-6, check_every=5)
            its[k].append(r.iters if r.status == "solved" else cap + 1)
            if r.status == "solved":
                assert abs(r.res["obj_p"] - hi.fun) <= 1e-4 * abs(hi.fun)
    med = {k: float(np.median(v)) for k, v in its.items()}
    assert med["first50"] < med["one300"] < med["none"], its


def test_iterate_history_and_y():
    inst = I.small_lp()
    A = inst.to_scipy()
    r = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=alg.LP_SCHEDULE, max_iter=400, tol=1e-7,
                       keep_x=5)
    assert len(r.x_history) == 5
    # y = w / mu is the multiplier: dual residual vanishes at convergence
    assert np.linalg.norm(A.T @ r.y + r.z - inst.c) <= 1e-6 * (1 + np.linalg.norm(inst.c))


@pytest.mark.parametrize("seed", range(6))
def test_vertex_enumeration_matches_highs(seed):
    """The brute-force ground truth itself agrees with a simplex/IPM code."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(500 + seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(6, 11))
    A, b, c = _tiny_lp(rng, m, n)
    x_ref, obj_ref, bases = vertex.solve_lp(A, b, c)
    hi = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert hi.status == 0
    assert abs(hi.fun - obj_ref) <= 1e-9 * (1 + abs(obj_ref))
    assert np.abs(A @ x_ref - b).max() <= 1e-9 * (1 + np.abs(b).max()) and x_ref.min() >= 0


def test_y_is_the_weighted_least_squares_multiplier():
    """y is not formed by the paper; the oracle takes the multiplier of the
    projection solve, (g - v)/mu.  At a solution it must agree with the plain
    definition: the least-squares y of A_hat'y = c_hat - z_hat in the scaled
    space (z_hat = O z, since O(A'y + z - c) = 0), y = M^-1 A_hat (c_hat - z_hat)."""
    inst = I.small_lp()
    A = inst.to_scipy()
    r = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=SCHEDS["lp"], max_iter=6000, tol=1e-10)
    assert r.status == "solved"
    Ah = (A @ sp.diags(r.O)).toarray()
    y_ls = np.linalg.solve(Ah @ Ah.T, Ah @ (r.O * inst.c - r.O * r.z))
    assert np.linalg.norm(r.y - y_ls) <= 1e-7 * (1 + np.linalg.norm(r.y))
    # and the wrong sign or a missing O would not agree
    y_bad = np.linalg.solve(Ah @ Ah.T, Ah @ (inst.c - r.z))
    assert np.linalg.norm(r.y - y_bad) > 1e-3 * np.linalg.norm(r.y)


def test_iterates_follow_a_reordering_of_coordinates_and_cones():
    """K is a product: reordering the orthant coordinates and the order of the
    Lorentz cones (moving whole blocks), with the matching columns of A and
    entries of c, reorders Algorithm 2's iterates the same way (through two
    rescalings), up to rounding."""
    inst = I.socp(scale=0.001)
    A = inst.to_scipy().tocsc()
    n_orth, dims = inst.n_orth, np.asarray(inst.soc_dims)
    rng = np.random.default_rng(4)
    off = C.soc_offsets(n_orth, dims)
    order = rng.permutation(len(dims))
    perm = np.concatenate([rng.permutation(n_orth)] +
                          [np.arange(off[k], off[k + 1]) for k in order]).astype(int)
    L = alg.Schedule(first=1, period=7)
    kw = dict(t=1.7, L=L, max_iter=20, tol=0.0, keep_x=20)
    r0 = alg.algorithm2(A, inst.b, inst.c, n_orth, dims, **kw)
    r1 = alg.algorithm2(A[:, perm], inst.b, inst.c[perm], n_orth, dims[order], **kw)
    scale = np.abs(r0.x).max()
    np.testing.assert_allclose(r1.x, r0.x[perm], atol=1e-9 * scale)
    np.testing.assert_allclose(r1.z, r0.z[perm], atol=1e-9 * np.abs(r0.z).max())
    np.testing.assert_allclose(r1.O, r0.O[perm], rtol=1e-9)
    np.testing.assert_allclose(r1.y, r0.y, atol=1e-9 * np.abs(r0.y).max())
    # a cone reordered without its coordinates is a different problem
    r2 = alg.algorithm2(A[:, perm], inst.b, inst.c[perm], n_orth, dims, **kw)
    if not np.array_equal(dims[order], dims):
        assert np.abs(r2.x - r0.x[perm]).max() > 1e-6 * scale


@pytest.mark.parametrize("mu", [1.0, 0.6])
def test_algorithm2_without_rescaling_is_algorithm1(mu):
    """With no rescaling after l = 1 (where x = z = e gives o = 1, O = I),
    Algorithm 2 (one-solve form of d, steps 17-21) is Algorithm 1 (steps 2-6)
    started from s = x/O - mu O z = (1 - mu) e."""
    inst = I.socp(scale=0.001)
    A = inst.to_scipy()
    for k in (1, 7, 40):
        r = alg.algorithm2(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=mu, L=alg.NO_SCHEDULE,
                           max_iter=k, tol=0.0)
        assert np.all(r.O == 1.0)
        e = C.cone_identity(inst.n, inst.n_orth, inst.soc_dims)
        x, z, s, p, d = alg.algorithm1(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=mu,
                                       s0=(1.0 - mu) * e, iters=k)
        np.testing.assert_allclose(r.s, s, atol=1e-10 * (1 + np.abs(s).max()))
        np.testing.assert_allclose(r.x, x, atol=1e-10 * (1 + np.abs(x).max()))
        np.testing.assert_allclose(r.z, z, atol=1e-10 * (1 + np.abs(z).max()))
