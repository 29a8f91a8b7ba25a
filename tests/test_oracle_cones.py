"""Pins for the oracle's cone operators (Definition 1).

The projection is pinned by properties that characterise it independently
of the closed form: membership, the variational inequality of a projection
onto a closed convex set, brute-force distance comparison against random
points of K, idempotence, and the Moreau decomposition (K is self-dual).
abs_K is pinned by Lemma 1's norm identity (Eq. 17).
"""
import numpy as np
import pytest

from oracle import cones as C


def _rand_cone_point(rng, d):
    """Random point of the Lorentz cone of size d (d >= 1)."""
    if d == 1:
        return np.array([rng.exponential()])
    xb = rng.standard_normal(d - 1) * rng.exponential()
    return np.concatenate([[np.linalg.norm(xb) + rng.exponential() * rng.integers(0, 2)], xb])


def _in_K(v, n_orth, dims, tol=1e-12):
    if np.any(v[:n_orth] < -tol):
        return False
    off = C.soc_offsets(n_orth, dims)
    for a, e in zip(off[:-1], off[1:]):
        if np.linalg.norm(v[a + 1:e]) > v[a] + tol * (1 + abs(v[a])):
            return False
    return True


CASES = [(5, []), (0, [3]), (0, [2, 7, 4]), (3, [5, 2]), (0, [64]), (2, [3, 3, 3, 10])]


@pytest.mark.parametrize("n_orth,dims", CASES)
def test_projection_is_nearest_point(n_orth, dims):
    rng = np.random.default_rng(1)
    n = n_orth + sum(dims)
    for _ in range(40):
        v = rng.standard_normal(n) * 3
        pv = C.proj_K(v, n_orth, dims)
        assert _in_K(pv, n_orth, dims)
        # variational inequality: (v - P v)'(u - P v) <= 0 for all u in K
        sizes = [1] * n_orth + list(dims)
        for _ in range(200):
            u = np.concatenate([_rand_cone_point(rng, d) for d in sizes])
            assert (v - pv) @ (u - pv) <= 1e-9 * (1 + np.linalg.norm(v) * np.linalg.norm(u))
            assert np.linalg.norm(v - pv) <= np.linalg.norm(v - u) + 1e-12


@pytest.mark.parametrize("n_orth,dims", CASES)
def test_idempotence_and_moreau(n_orth, dims):
    rng = np.random.default_rng(2)
    n = n_orth + sum(dims)
    for _ in range(100):
        v = rng.standard_normal(n)
        p = C.proj_K(v, n_orth, dims)
        np.testing.assert_allclose(C.proj_K(p, n_orth, dims), p, atol=1e-14)
        q = C.proj_K(-v, n_orth, dims)
        # Moreau: v = P_K(v) + P_{K polar}(v), K polar = -K for a self-dual cone
        np.testing.assert_allclose(p - q, v, atol=1e-13)
        assert abs(p @ q) <= 1e-12 * (1 + v @ v)


@pytest.mark.parametrize("n_orth,dims", CASES)
def test_abs_preserves_norm(n_orth, dims):
    rng = np.random.default_rng(3)
    n = n_orth + sum(dims)
    for _ in range(100):
        v = rng.standard_normal(n)
        a = C.abs_K(v, n_orth, dims)
        assert abs(np.linalg.norm(a) - np.linalg.norm(v)) <= 1e-13 * (1 + np.linalg.norm(v))


def test_special_cases():
    # inside -> unchanged, polar -> 0, orthogonal axis -> halfway point
    np.testing.assert_array_equal(C.proj_K(np.array([2.0, 1.0, -1.0]), 0, [3]), [2.0, 1.0, -1.0])
    np.testing.assert_array_equal(C.proj_K(np.array([-2.0, 1.0, -1.0]), 0, [3]), [0.0, 0.0, 0.0])
    np.testing.assert_allclose(C.proj_K(np.array([0.0, 1.0, 0.0]), 0, [3]), [0.5, 0.5, 0.0])
    # boundary ties: |vbar| == v1 stays, |vbar| == -v1 maps to 0
    np.testing.assert_array_equal(C.proj_K(np.array([1.0, 0.6, 0.8]), 0, [3]), [1.0, 0.6, 0.8])
    np.testing.assert_array_equal(C.proj_K(np.array([-1.0, 0.6, 0.8]), 0, [3]), [0.0, 0.0, 0.0])
    # zero tail, negative head
    np.testing.assert_array_equal(C.proj_K(np.array([-1.0, 0.0]), 0, [2]), [0.0, 0.0])
    # orthant: abs is the plain absolute value
    v = np.array([-1.5, 0.0, 2.0])
    np.testing.assert_array_equal(C.abs_K(v, 3, []), np.abs(v))


def test_size_two_cone_is_rotated_quadrant():
    # K_2 = {w1 >= |w2|} is R+^2 rotated by 45 degrees
    rng = np.random.default_rng(4)
    R = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)   # orthogonal and R = R^-1
    for _ in range(100):
        v = rng.standard_normal(2)
        ref = R @ np.maximum(R @ v, 0.0)
        np.testing.assert_allclose(C.proj_K(v, 0, [2]), ref, atol=1e-14)


def test_cone_identity_and_check():
    e = C.cone_identity(9, 2, [3, 4])
    np.testing.assert_array_equal(e, [1, 1, 1, 0, 0, 1, 0, 0, 0])
    with pytest.raises(ValueError):
        C.check_cones(9, 2, [3, 3])
    with pytest.raises(ValueError):
        C.check_cones(4, 3, [1])
