"""Pins of the refinement-step model used by the BF16-storage parity test
(tests/refinement_model.py) against the oracle: with the exact matrix in the
correction it is Algorithm 2 itself, and its BF16 rounding is the nearest
BF16 value with ties to even."""
import numpy as np

from oracle import alg
from paper_2103_00736_gb300 import instances as I

import refinement_model as RM


def test_model_with_exact_correction_is_algorithm2():
    inst = I.small_lp()
    A = inst.to_scipy()
    ref = alg.algorithm2(A, inst.b, inst.c, inst.n, [], L=alg.LP_SCHEDULE, max_iter=50, tol=0.0, keep_x=50)
    got = RM.refined_iterates(A, inst.b, inst.c, inst.n, [], iters=50)
    for k in (1, 2, 10, 50):
        xr = ref.x_history[k - 1]
        assert np.linalg.norm(got[k - 1] - xr) <= 1e-10 * np.linalg.norm(xr), k


def test_model_with_rounded_correction_differs():
    """BF16 values in the correction move the iterates by far more than
    FP32 arithmetic would (so the BF16 parity test needs this model)."""
    inst = I.small_lp()
    A = inst.to_scipy()
    exact = RM.refined_iterates(A, inst.b, inst.c, inst.n, [], iters=20)
    bf = RM.refined_iterates(A, inst.b, inst.c, inst.n, [], iters=20, correction_values=RM.bf16_round(A.data))
    dev = np.linalg.norm(bf[-1] - exact[-1]) / np.linalg.norm(exact[-1])
    assert dev > 1e-5


def test_bf16_round_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8, -3.0 - 2 ** -7, 1e-30, 65504.0, 0.1])
    got = RM.bf16_round(x)
    # exact BF16 values stay, ties go to the even mantissa, others to the nearest
    assert got[0] == 1.0
    assert got[1] == 1.0                        # tie between 1 and 1 + 2^-7: even is 1
    assert got[2] == 1.0 + 2 ** -6              # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert got[3] == -3.0                       # tie between -3 (even) and -3 - 2^-6 (spacing 2^-6 there)
    for v, g in zip(x, got):
        assert abs(g - v) <= 2 ** -8 * abs(v) + 1e-45
