"""Algorithm 1 and Algorithm 2 (adaptive conditioning), step by step in FP64.

Algorithm 2 (Section IV), with the readings used throughout this code base:
  l <- 0;  repeat  l <- l + 1
    if l in L u {1}:                                          (step 4)
      for every cone i with first coordinate h+1 and every j in the cone:
        o_j <- |x_{h+1} - ||(x_{h+2},...,x_{h+n_i})|| | / |z_{h+1}|   (step 8)
      O <- diag(|o|)^min(1, t / (log max o - log min o))     (step 11)
      A_hat_cal <- range((A O)')                             (step 12)
      d <- (A O)^dagger b + (mu/2)(abs_{A_hat_cal}(O c) - O c)    (step 13)
      s <- O^{-1} x - mu O z                                 (step 14)
    p <- abs_{O^{-1} K}(s)                                   (step 17)
    r <- abs_{A_hat_cal}(p)                                  (step 18)
    s <- s/2 - r/2 + d                                       (step 19)
    x <- O (p + s) / 2                                       (step 20)
    z <- O^{-1} (p - s) / (2 mu)                             (step 21)
  until the stopping test holds.

Readings (the paper is silent or ambiguous on these):
  * log is the natural log; t > 0 caps the spread max(O)/min(O) at e^t
    (the Require line says 0 < t < 1, the experiments use t = 9.2 and 1.7).
  * Initial point x = z = e, the cone identity (1 on orthant coordinates,
    (1, 0, ..., 0) on every Lorentz cone); then o = 1 and O = I at l = 1, and
    s = (1 - mu) e.
  * o is the same for every coordinate of one cone, so O is constant on each
    cone and O^{-1} K = K, abs_{O^{-1} K} = abs_K; O' A_cal = range((A O)').
  * o_j = 0, inf or nan (x_{h+1} = ||xbar|| or z_{h+1} = 0, e.g. a
    coordinate with x_j = z_j = 0): a departure from the printed rule, not a
    reading of it.  Evaluated as printed (IEEE, or MATLAB whose max and min
    skip nan), an o of 0 or inf makes the log spread infinite, the exponent
    0 and O = I: one degenerate coordinate switches the rescaling off for the
    whole problem (conditioning_matrix_literal, rule="literal").  The oracle
    instead lets such entries carry no scale: the exponent of step 11 is
    computed from the finite positive o only, and the others take the
    limits of the rule under the cap: o = 0 the smallest scale
    min(o)^alpha, o = inf the largest max(o)^alpha, o = nan the geometric
    middle.  No finite positive o at all: O = I.  All finite o equal:
    exponent 1.
  * O is recomputed from the current x, z at each conditioning (not composed).
  * Steps 20-21 use p from the old s and the updated s, as printed.
  * The schedule L continues with its period up to max_iter.
  * y is not formed by the paper.  With M = A_hat A_hat' and
    b_tilde = b + mu A_hat c_hat the update is equivalently
        w = M^{-1} (b_tilde - A_hat p),  s <- (s + p)/2 - mu c_hat + A_hat' w,
    and y = w / mu is the multiplier of the affine constraint (at a fixed
    point A'y + z = c).  The oracle keeps the literal steps and derives
    w = M^{-1} b_tilde - M^{-1} A_hat p from the solve that step 18 already
    does; the identity d = A_hat' M^{-1} b_tilde - mu c_hat is asserted at
    every conditioning.

Pinned by: vertex enumeration and HiGHS on LPs, planted optima, closed-form
SOCPs, the textbook Douglas-Rachford identity, Lemma 2's fixed point and
Lemma 3's monotonicity (tests/test_oracle_alg.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp

from . import cones as C
from . import kkt
from .subspace import Subspace


@dataclass
class Schedule:
    """Conditioning iterations L: an explicit list plus {first, first+period, ...}."""
    first: int = 0          # 0 = no periodic part
    period: int = 0
    explicit: tuple = ()

    def __contains__(self, l: int) -> bool:
        if l in self.explicit:
            return True
        if self.first > 0 and l >= self.first:
            if self.period <= 0:
                return l == self.first
            return (l - self.first) % self.period == 0
        return False


LP_SCHEDULE = Schedule(first=300, period=100)      # Section V-A
SOCP_SCHEDULE = Schedule(first=200, period=100)    # Section V-C
NO_SCHEDULE = Schedule()


def conditioning_vector(x: np.ndarray, z: np.ndarray, n_orth: int, soc_dims) -> np.ndarray:
    """o_j of Algorithm 2 step 8, the same value on every coordinate of a cone."""
    xh, xt, sizes = C.heads_and_tail_norms(x, n_orth, soc_dims)
    zh, _, _ = C.heads_and_tail_norms(z, n_orth, soc_dims)
    with np.errstate(divide="ignore", invalid="ignore"):
        o_cone = np.abs(xh - xt) / np.abs(zh)
    return np.repeat(o_cone, sizes)


def conditioning_exponent(o: np.ndarray, t: float) -> float:
    """min(1, t / (log max o - log min o)) of step 11 over the finite positive o."""
    ok = np.isfinite(o) & (o > 0.0)
    if not np.any(ok):
        return 0.0
    spread = math.log(float(o[ok].max())) - math.log(float(o[ok].min()))
    if spread <= 0.0:
        return 1.0
    return min(1.0, t / spread)


def conditioning_matrix_literal(x, z, n_orth, soc_dims, t):
    """diag(O) of step 11 evaluated as printed in IEEE arithmetic, with max and
    min ignoring nan (MATLAB's max/min): an o of 0 or inf makes
    log max o - log min o infinite, so alpha = min(1, t / inf) = 0 and
    O = |o|^0 = 1 everywhere (0^0 = inf^0 = nan^0 = 1): the rescaling is
    switched off.  With only nan among the non-finite o, alpha > 0 and the
    nan entries give O_j = nan (the printed rule is undefined there).  This
    is not the rule the oracle uses (conditioning_matrix); it is kept to
    show what the literal evaluation does."""
    o = conditioning_vector(x, z, n_orth, soc_dims)
    with np.errstate(divide="ignore", invalid="ignore"):
        lo = np.log(np.abs(o))
        if np.all(np.isnan(lo)):
            return np.full_like(o, np.nan), float("nan")
        spread = float(np.nanmax(lo) - np.nanmin(lo))
        alpha = min(1.0, t / spread) if spread > 0 else 1.0
        return np.power(np.abs(o), alpha), alpha


def conditioning_matrix(x, z, n_orth, soc_dims, t):
    """diag(O) of step 11: |o|^alpha, with the limits above for o in {0, inf, nan}."""
    o = conditioning_vector(x, z, n_orth, soc_dims)
    alpha = conditioning_exponent(o, t)
    ok = np.isfinite(o) & (o > 0.0)
    if not np.any(ok):
        return np.ones_like(o), alpha
    lo = np.empty_like(o)
    lo[ok] = np.log(o[ok])
    lmin, lmax = lo[ok].min(), lo[ok].max()
    lo[~ok & (o == 0.0)] = lmin
    lo[~ok & np.isinf(o)] = lmax
    lo[np.isnan(o)] = 0.5 * (lmin + lmax)
    return np.exp(alpha * lo), alpha


@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    s: np.ndarray
    O: np.ndarray
    iters: int
    status: str
    res: dict
    history: list = field(default_factory=list)
    x_history: list = field(default_factory=list)
    O_history: list = field(default_factory=list)


def algorithm2(A, b, c, n_orth: int, soc_dims=(), mu: float = 1.0, t: float = 9.2,
               L: Schedule = LP_SCHEDULE, max_iter: int = 1000, tol: float = 1e-6,
               check_every: int = 1, x0=None, z0=None, keep_x: int = 0,
               solver: str = "auto", on_iter=None, rule: str = "finite") -> Result:
    """Algorithm 2 in FP64.  Stops when every relative KKT residual (kkt.residuals)
    is <= tol at a check, or after max_iter iterations (status 'max_iter').
    rule: step 11 as the oracle reads it ("finite", conditioning_matrix) or
    evaluated as printed ("literal", conditioning_matrix_literal; a nan O
    ends the run with status 'breakdown')."""
    A = sp.csr_matrix(A, dtype=np.float64)
    m, n = A.shape
    soc_dims = np.asarray(soc_dims, dtype=np.int64)
    C.check_cones(n, n_orth, soc_dims)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    e = C.cone_identity(n, n_orth, soc_dims)
    x = e.copy() if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    z = e.copy() if z0 is None else np.asarray(z0, dtype=np.float64).copy()

    out = Result(x=x, y=np.zeros(m), z=z, s=np.zeros(n), O=np.ones(n), iters=0,
                 status="max_iter", res={})
    l = 0
    O = sub = d = s = g = None
    while l < max_iter:
        l += 1
        if l in L or l == 1:
            if rule == "literal":
                O, alpha = conditioning_matrix_literal(x, z, n_orth, soc_dims, t)
                if not np.all(np.isfinite(O)):
                    out.status, out.iters = "breakdown", l
                    return out
            else:
                O, alpha = conditioning_matrix(x, z, n_orth, soc_dims, t)    # steps 5-11
            sub = Subspace(A, O, solver=solver)                              # step 12
            c_hat = O * c
            d = sub.pinv_t(b) + 0.5 * mu * (sub.abs(c_hat) - c_hat)          # step 13
            s = x / O - mu * O * z                                           # step 14
            g = sub.solve_M(b + mu * (sub.Ah @ c_hat))
            d_one_solve = sub.AhT @ g - mu * c_hat
            assert np.linalg.norm(d - d_one_solve) <= 1e-7 * (1.0 + np.linalg.norm(d)), \
                "one-solve identity for d failed"
            out.O_history.append((l, O.copy(), alpha))
        p = C.abs_K(s, n_orth, soc_dims)                                     # step 17
        v = sub.solve_M(sub.Ah @ p)                                          # step 18:
        r = 2.0 * (sub.AhT @ v) - p                                          #   abs_A(p)
        s = 0.5 * s - 0.5 * r + d                                            # step 19
        x = O * (p + s) / 2.0                                                # step 20
        z = (p - s) / (O * 2.0 * mu)                                         # step 21
        y = (g - v) / mu
        if keep_x and l <= keep_x:
            out.x_history.append(x.copy())
        if on_iter is not None:
            on_iter(l, s, p, O, d)
        if l % check_every == 0 or l == max_iter:
            res = kkt.residuals(A, b, c, x, y, z, n_orth, soc_dims)
            out.history.append((l, res))
            if kkt.max_residual(res) <= tol:
                out.status = "solved"
                out.x, out.y, out.z, out.s, out.O, out.iters, out.res = x, y, z, s, O, l, res
                return out
    res = kkt.residuals(A, b, c, x, y, z, n_orth, soc_dims)
    out.x, out.y, out.z, out.s, out.O, out.iters, out.res = x, y, z, s, O, l, res
    return out


def algorithm1(A, b, c, n_orth: int, soc_dims=(), mu: float = 1.0, s0=None,
               iters: int = 100, solver: str = "auto"):
    """Algorithm 1 for a fixed number of iterations; returns (x, z, s, p, d)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    m, n = A.shape
    sub = Subspace(A, np.ones(n), solver=solver)                             # step 1
    d = sub.pinv_t(b) + 0.5 * mu * (sub.abs(c) - c)                          # step 2
    s = np.zeros(n) if s0 is None else np.asarray(s0, dtype=np.float64).copy()
    p = C.abs_K(s, n_orth, soc_dims)
    for _ in range(iters):
        p = C.abs_K(s, n_orth, soc_dims)                                     # step 4
        r = sub.abs(p)                                                       # step 5
        s = 0.5 * s - 0.5 * r + d                                            # step 6
    x = (p + s) / 2.0
    z = (p - s) / (2.0 * mu)
    return x, z, s, p, d
