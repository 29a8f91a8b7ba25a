"""The comparison iterations of Section III-B (Douglas-Rachford, ADMM) in the
oracle, pinned against identities and known optima, and the Section III-A
comparison on the worked example (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle import alg, baselines as B, cones as C, vertex

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
A = np.array(GOLD["A"])
b = np.array(GOLD["b"])
c = np.array(GOLD["c"])


def _x_star():
    return np.array(vertex.solve_lp(A, b, c)[0])


def _scalings():
    return {"none": (None, None),
            "sk": (np.array(GOLD["D_SK"]), np.array(GOLD["E_SK"])),
            "ruiz": B.ruiz(A),
            "ac": (None, np.array(GOLD["E_AC"]))}


@pytest.mark.parametrize("mu", [1.0, 0.5, 3.0])
def test_dr_state_is_algorithm1s_s(mu):
    """Algorithm 1 is Section III-B's DR with the same mu: z of DR after k
    iterations equals s of Algorithm 1 (its own projection via Subspace)."""
    for k in (1, 2, 5, 30):
        _, z = B.douglas_rachford(A, b, c, 5, mu=mu, iters=k)
        _, _, s, _, _ = alg.algorithm1(A, b, c, 5, mu=mu, iters=k)
        assert np.linalg.norm(z - s) <= 1e-8 * (1.0 + np.linalg.norm(s)), (k, np.abs(z - s).max())


def _prox_g_lstsq(As, bs, cs, mu):
    """argmin (cs)'x + ||x - v||^2/(2 mu) s.t. As x = bs by the KKT system
    solved with lstsq (independent of the oracle's QR projection)."""
    m, n = As.shape
    K = np.block([[np.eye(n), As.T], [As, np.zeros((m, m))]])

    def prox(v):
        rhs = np.concatenate([v - mu * cs, bs])
        return np.linalg.lstsq(K, rhs, rcond=None)[0][:n]
    return prox


@pytest.mark.parametrize("mu", [1.0, 0.7])
def test_admm_is_dr_with_the_steps_swapped(mu):
    """ADMM's x1 sequence equals that of DR with prox_g taken first, on
    zeta = x1 + z_prev/mu (textbook identity; prox_g here from the KKT system)."""
    x2_0 = np.array([0.5, 1.0, 2.0, 0.0, 0.3])
    xs = B.admm(A, b, c, 5, mu=mu, iters=25, x2_0=x2_0)
    # ADMM's prox of g/mu is prox_{g} with parameter 1/mu
    prox = _prox_g_lstsq(A, b, c, 1.0 / mu)
    zeta = np.maximum(x2_0, 0.0)                    # zeta^1 = x1^1 + 0
    np.testing.assert_allclose(xs[0], zeta, atol=1e-14)
    for k in range(1, 25):
        g = prox(zeta)
        x1 = np.maximum(2.0 * g - zeta, 0.0)
        zeta = zeta + x1 - g
        assert np.linalg.norm(xs[k] - x1) <= 1e-9 * (1.0 + np.linalg.norm(x1)), k


def test_dr_and_admm_reach_the_vertex_optimum():
    xs = _x_star()
    xd, _ = B.douglas_rachford(A, b, c, 5, iters=400)
    xa = B.admm(A, b, c, 5, iters=400)
    assert np.linalg.norm(xd[-1] - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.linalg.norm(xa[-1] - xs) <= 1e-9 * np.linalg.norm(xs)


def test_dr_and_admm_on_a_lorentz_cone():
    """min x1 s.t. x2 = 1, x3 = 1, x in L^3: x* = (sqrt 2, 1, 1)."""
    As = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    bs, cs = np.array([1.0, 1.0]), np.array([1.0, 0.0, 0.0])
    want = np.array([np.sqrt(2.0), 1.0, 1.0])
    xd, _ = B.douglas_rachford(As, bs, cs, 0, [3], iters=500)
    xa = B.admm(As, bs, cs, 0, [3], iters=500)
    np.testing.assert_allclose(xd[-1], want, atol=1e-9)
    np.testing.assert_allclose(xa[-1], want, atol=1e-9)
    assert C.dist_K(xd[-1], 0, [3]) <= 1e-12


def test_scaling_is_a_change_of_variables():
    """Any positive D, E leave the optimum x* = E u* unchanged."""
    xs = _x_star()
    rng = np.random.default_rng(3)
    D, E = rng.uniform(0.5, 2.0, 3), rng.uniform(0.5, 2.0, 5)
    xd, _ = B.douglas_rachford(A, b, c, 5, D=D, E=E, iters=600)
    assert np.linalg.norm(xd[-1] - xs) <= 1e-8 * np.linalg.norm(xs)


def test_ruiz_equilibrates():
    D, E = B.ruiz(A, 40)
    S = np.abs(D[:, None] * A * E[None, :])
    np.testing.assert_allclose(S.max(axis=1), 1.0, atol=1e-10)
    np.testing.assert_allclose(S.max(axis=0), 1.0, atol=1e-10)
    assert np.linalg.cond(S) < 300 < GOLD["cond_A"]


def test_study_ruiz_matches_the_oracles():
    from paper_2103_00736_gb300 import studies
    D1, E1 = studies.ruiz(A)
    D2, E2 = B.ruiz(A)
    np.testing.assert_allclose(D1, D2, rtol=1e-14)
    np.testing.assert_allclose(E1, E2, rtol=1e-14)
    sc = studies.worked_scalings()
    np.testing.assert_allclose(sc["sk"][0], GOLD["D_SK"])
    np.testing.assert_allclose(sc["ac"][1], GOLD["E_AC"])
    np.testing.assert_allclose(np.array(studies.WORKED_A), A)


def _alg1_iterates(D, E, iters):
    """x = E u of Algorithm 1 on the scaled data after 1..iters iterations."""
    Dv = np.ones(3) if D is None else D
    Ev = np.ones(5) if E is None else E
    As, bs, cs = (Dv[:, None] * A) * Ev[None, :], Dv * b, Ev * c
    out, s = [], np.zeros(5)
    for _ in range(iters):
        x, _, s, _, _ = alg.algorithm1(As, bs, cs, 5, s0=s, iters=1)
        out.append(Ev * x)
    return out


def test_section_iii_a_comparison():
    """The worked example's point (Section III-A): the lower condition number
    of the Sinkhorn-Knopp scaling (2044 against 2046) does not speed DR, ADMM
    or Algorithm 1 up, Ruiz (cond ~ 284) barely does, while the adaptive-
    conditioning scaling (cond 72079) converges in a handful of iterations."""
    xs = _x_star()
    table = {}
    for name, (D, E) in _scalings().items():
        xd, _ = B.douglas_rachford(A, b, c, 5, D=D, E=E, iters=300)
        xa = B.admm(A, b, c, 5, D=D, E=E, iters=300)
        x1 = _alg1_iterates(D, E, 150)
        table[name] = {k: B.iterations_to(v, xs, 1e-6) for k, v in (("dr", xd), ("admm", xa), ("alg1", x1))}
    print(table)
    for alg_name in ("dr", "admm", "alg1"):
        it = {k: table[k][alg_name] for k in table}
        assert it["ac"] is not None and it["ac"] <= 10, (alg_name, it)
        for other in ("none", "sk", "ruiz"):
            assert it[other] is not None and it[other] >= 5 * it["ac"], (alg_name, it)
        assert it["sk"] >= it["none"], (alg_name, it)


def test_admm_iterates_leave_the_rescaling_rule_nothing_to_work_with():
    """ADMM's x = proj_K(a) and z = proj_K(-a)/mu are exactly complementary,
    so step 8's ratio o is 0, inf or nan on every coordinate: the reason the
    ADMM form runs without rescaling."""
    rng = np.random.default_rng(5)
    n_orth, dims = 6, [3, 4]
    a = rng.standard_normal(n_orth + sum(dims))
    mu = 0.7
    x = C.proj_K(a, n_orth, dims)
    z = C.proj_K(-a, n_orth, dims) / mu
    o = alg.conditioning_vector(x, z, n_orth, dims)
    assert all((v == 0.0) or np.isinf(v) or np.isnan(v) for v in o), o
    # while DR's pair (x, z) = ((p + s)/2, (p - s)/(2 mu)) from two different s is not
    s_old, s_new = a, rng.standard_normal(a.size)
    p = C.abs_K(s_old, n_orth, dims)
    od = alg.conditioning_vector((p + s_new) / 2, (p - s_new) / (2 * mu), n_orth, dims)
    assert np.isfinite(od).any() and (od[np.isfinite(od)] > 0).any()
