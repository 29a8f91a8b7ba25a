"""GPU: the comparison iterations of Section III (Douglas-Rachford, which is
the iteration of Algorithm 1, and ADMM) through the C ABI against the FP64
oracle, and the Section III-A comparison on the worked example.

Tolerances: the worked example runs on the cached FP64 operator (m = 3), whose
solve of M w = r carries a relative error of about cond(M) eps: cond(M) =
cond(DAE)^2 is 4.2e6 for the unscaled, SK and Ruiz data (error ~5e-10) and
5.2e9 for E^AC (~6e-7); the iterates are checked at 1e-8 and 1e-5 of ||x||
respectively.  End results: every relative KKT residual <= 1e-6 as the
oracle's FP64 residual function evaluates the returned (x, y, z).
"""
import json
import os

import numpy as np
import pytest

pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I, studies  # noqa: E402
from oracle import alg, baselines as B, kkt, vertex  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
A = np.array(GOLD["A"])
b = np.array(GOLD["b"])
c = np.array(GOLD["c"])
KS = (1, 2, 3, 5, 10, 20, 40)


def _scaling(name):
    if name == "ruiz":
        return B.ruiz(A)
    if name == "sk":
        return np.array(GOLD["D_SK"]), np.array(GOLD["E_SK"])
    if name == "ac":
        return np.ones(3), np.array(GOLD["E_AC"])
    return np.ones(3), np.ones(5)


def _alg1_iterates(D, E, ks):
    As, bs, cs = (D[:, None] * A) * E[None, :], D * b, E * c
    out, s, done = {}, np.zeros(5), 0
    for k in sorted(ks):
        x, _, s, _, _ = alg.algorithm1(As, bs, cs, 5, s0=s, iters=k - done)
        done = k
        out[k] = E * x
    return [out[k] for k in ks]


@pytest.mark.parametrize("scaling", ["none", "sk", "ruiz", "ac"])
def test_dr_iterates_match_algorithm1(scaling):
    """splitting = DR: x after k iterations equals Algorithm 1's x on the
    scaled data (the oracle's Algorithm 1; DR's z = Algorithm 1's s is pinned
    on the CPU)."""
    D, E = _scaling(scaling)
    got = studies.scaled_iterates(D, E, capi.SPLIT_DR, KS)
    ref = _alg1_iterates(D, E, KS)
    tol = 1e-5 if scaling == "ac" else 1e-8
    for k, xg, xr in zip(KS, got, ref):
        assert np.linalg.norm(xg - xr) <= tol * np.linalg.norm(xr), (k, xg, xr)


@pytest.mark.parametrize("scaling", ["none", "sk", "ruiz", "ac"])
def test_admm_iterates_match_oracle(scaling):
    """splitting = ADMM: zeta starts at x - mu z = 0 (x = z = e, mu = 1), the
    oracle's ADMM from x2 = z = 0, whose first x1 is 0; the GPU's x after k
    iterations is the oracle's (k+1)-th x1."""
    D, E = _scaling(scaling)
    got = studies.scaled_iterates(D, E, capi.SPLIT_ADMM, KS)
    ref = B.admm(A, b, c, 5, D=D, E=E, iters=max(KS) + 1)
    tol = 1e-5 if scaling == "ac" else 1e-8
    for k, xg in zip(KS, got):
        xr = ref[k]
        assert np.linalg.norm(xg - xr) <= tol * np.linalg.norm(xr), (k, xg, xr)


def test_admm_on_a_lorentz_cone():
    """The ADMM cone phase: min x1 s.t. x2 = 1, x3 = 1, x in L^3 (x* = (sqrt 2, 1, 1)),
    iterates against the oracle's ADMM from x2 = z = 0, and the optimum."""
    As = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    bs, cs = np.array([1.0, 1.0]), np.array([1.0, 0.0, 0.0])
    ref = B.admm(As, bs, cs, 0, [3], iters=60)
    for k in (1, 2, 5, 20, 59):
        st, x, _, _, _ = studies.solve_dense(As, bs, cs, 0.0, k, n_orth=0, soc_dims=[3], cond_first=0,
                                             splitting=capi.SPLIT_ADMM, precision=capi.PREC_FP64)
        assert st == capi.MAX_ITER
        np.testing.assert_allclose(x, ref[k], rtol=1e-9, atol=1e-12)
    st, x, y, z, _ = studies.solve_dense(As, bs, cs, 1e-10, 5000, n_orth=0, soc_dims=[3], cond_first=0,
                                         splitting=capi.SPLIT_ADMM, precision=capi.PREC_FP64)
    assert st == capi.SOLVED
    np.testing.assert_allclose(x, [np.sqrt(2.0), 1.0, 1.0], atol=1e-8)


@pytest.mark.parametrize("projection", [capi.PROJ_AUTO, capi.PROJ_CG])
def test_admm_solves_the_small_lp(projection):
    """ADMM (L empty) to an end result, cached operator and CG projection."""
    inst = I.small_lp()
    s = capi.acs_settings_default(splitting=capi.SPLIT_ADMM, projection=projection, cond_first=0)
    with capi.Solver(inst, settings=s) as sv:
        st = sv.solve(tol=1e-7, max_iter=20000)
        rc, x, y, z, iters, res = sv.get()
    assert st == capi.SOLVED, capi.acs_status_string(st)
    r = kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)
    assert kkt.max_residual(r) <= 1e-6, r
    assert abs(r["obj_p"] - inst.obj_star) <= 1e-6 * abs(inst.obj_star)


def test_admm_solves_the_small_socp():
    inst = I.socp(scale=0.002)
    s = capi.acs_settings_default(splitting=capi.SPLIT_ADMM, cond_first=0)
    with capi.Solver(inst, settings=s) as sv:
        st = sv.solve(tol=1e-7, max_iter=20000)
        rc, x, y, z, iters, res = sv.get()
    assert st == capi.SOLVED, capi.acs_status_string(st)
    r = kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)
    assert kkt.max_residual(r) <= 1e-6, r


def test_section_iii_a_study_on_the_gpu():
    """The study's iteration counts (to ||x - x*|| <= 1e-6 ||x*|| for good)
    agree with the oracle's within one iteration, and show the section's
    point: E^AC (cond 72079) converges within 10 iterations, the others
    (cond 2046, 2044, 284) take at least five times as many."""
    out = studies.preconditioning_study(max_iter=150, rtols=(1e-6,))
    xs = np.array(vertex.solve_lp(A, b, c)[0])
    assert np.linalg.norm(np.array(out["x_ref"]) - xs) <= 1e-10 * np.linalg.norm(xs)
    print(json.dumps(out["table"]))
    for name in ("none", "sk", "ruiz", "ac"):
        D, E = _scaling(name)
        dr_ref = B.iterations_to(_alg1_iterates(D, E, range(1, 151)), xs, 1e-6)
        ad = B.admm(A, b, c, 5, D=D, E=E, iters=151)
        admm_ref = B.iterations_to(ad[1:], xs, 1e-6)
        got_dr = out["table"][f"dr/{name}"]["iterations_to"]["1e-06"]
        got_admm = out["table"][f"admm/{name}"]["iterations_to"]["1e-06"]
        assert got_dr is not None and abs(got_dr - dr_ref) <= 1, (name, got_dr, dr_ref)
        assert got_admm is not None and abs(got_admm - admm_ref) <= 1, (name, got_admm, admm_ref)
    for p in ("dr", "admm"):
        ac = out["table"][f"{p}/ac"]["iterations_to"]["1e-06"]
        assert ac <= 10
        for name in ("none", "sk", "ruiz"):
            assert out["table"][f"{p}/{name}"]["iterations_to"]["1e-06"] >= 5 * ac


def test_admm_iterates_on_a_socp_with_many_cones():
    """The ADMM cone phase on the scaled C3 recipe (orthant plus Lorentz cones
    of 3..64 coordinates, multi-lane cones): the device's x after k
    iterations against the oracle's ADMM from x2 = z = 0 (the cached FP64
    operator on the device, m = 150; the oracle's QR projection)."""
    inst = I.socp(scale=0.001)
    A = inst.to_scipy().toarray()
    ref = B.admm(A, inst.b, inst.c, inst.n_orth, list(inst.soc_dims), iters=31)
    s = capi.acs_settings_default(splitting=capi.SPLIT_ADMM, cond_first=0, precision=capi.PREC_FP64)
    h = capi.acs_problem_create(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.b, inst.c,
                                inst.n_orth, inst.soc_dims, s)
    try:
        for k in (1, 2, 7, 30):
            st = capi.acs_solve(h, 0.0, k)
            _, x, _, _, _, _ = capi.acs_get(h, inst.m, inst.n)
            assert st == capi.MAX_ITER
            assert np.linalg.norm(x - ref[k]) <= 1e-9 * (1.0 + np.linalg.norm(ref[k])), k
    finally:
        capi.acs_problem_destroy(h)
