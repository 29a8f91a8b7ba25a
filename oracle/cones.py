"""Cone projections and reflections (Section II, Definition 1).

K = K_{n_1} x ... x K_{n_k}, each K_{n_i} a Lorentz cone
{w : w_1 >= ||(w_2, ..., w_{n_i})||_2}.  A size-1 Lorentz cone is the
half-line R+, so the nonnegative orthant is the product of n_orth size-1
cones; in this code base the orthant coordinates come first and the cones
of size >= 2 follow in the order of ``soc_dims``.

proj_C(v) = argmin_{u in C} ||u - v||_2 and abs_C(v) = 2 proj_C(v) - v
(Definition 1).  For a Lorentz cone the projection has the textbook closed
form (Boyd & Vandenberghe, Convex Optimization, Sec. 8.1.1, Exercise 8.3):
with v = (v1, vbar) and t = ||vbar||,
    t <= v1   -> v               (already inside)
    t <= -v1  -> 0               (inside the polar cone)
    otherwise -> ((v1 + t)/2) * (1, vbar/t).
Ties use "<=" in both tests; in the third branch t > |v1| >= 0, so the
division is safe.

Pinned by: idempotence, the Moreau decomposition v = proj_K(v) - proj_K(-v)
with orthogonal parts, norm preservation of abs_K (Lemma 1, Eq. 17), and a
brute-force 1-D minimisation on tiny cones (tests/test_oracle_cones.py).
"""
from __future__ import annotations

import numpy as np


def soc_offsets(n_orth: int, soc_dims) -> np.ndarray:
    """Start index of every Lorentz cone of size >= 2, plus the end (length n_soc+1)."""
    dims = np.asarray(soc_dims, dtype=np.int64)
    return n_orth + np.concatenate([[0], np.cumsum(dims)]).astype(np.int64)


def check_cones(n: int, n_orth: int, soc_dims) -> None:
    """K is a product of Lorentz cones (Section II): n_orth size-1 cones, then
    cones of size >= 2, covering all n coordinates."""
    dims = np.asarray(soc_dims, dtype=np.int64)
    if n_orth < 0 or np.any(dims < 2) or n_orth + int(dims.sum()) != n:
        raise ValueError("cone sizes must be n_orth >= 0, each soc dim >= 2, total n")


def _soc_heads_and_tail_norms(v: np.ndarray, n_orth: int, soc_dims):
    """(v1 per cone, ||vbar|| per cone, start offsets) for the cones of size >= 2."""
    off = soc_offsets(n_orth, soc_dims)
    if off.size == 1:
        return np.zeros(0), np.zeros(0), off
    heads = v[off[:-1]]
    return heads, np.sqrt(_tail_sq_grouped(v, off)), off


def _tail_sq_grouped(v: np.ndarray, off: np.ndarray) -> np.ndarray:
    """Per-cone sum of squares of the tail, grouped by cone size (vectorised)."""
    starts, ends = off[:-1], off[1:]
    dims = ends - starts
    out = np.empty(starts.size)
    for d in np.unique(dims).tolist():
        sel = np.flatnonzero(dims == d)
        idx = starts[sel][:, None] + np.arange(1, d)[None, :]
        t = v[idx]
        out[sel] = np.einsum("ij,ij->i", t, t)
    return out


def proj_soc(v: np.ndarray) -> np.ndarray:
    """Projection of one vector onto a Lorentz cone (closed form above)."""
    v = np.asarray(v, dtype=np.float64)
    v1 = v[0]
    t = float(np.linalg.norm(v[1:]))
    if t <= v1:
        return v.copy()
    if t <= -v1:
        return np.zeros_like(v)
    a = 0.5 * (v1 + t)
    out = np.empty_like(v)
    out[0] = a
    out[1:] = (a / t) * v[1:]
    return out


def proj_K(v: np.ndarray, n_orth: int, soc_dims) -> np.ndarray:
    """proj_K for K = R+^{n_orth} x prod_i K_{d_i} (Definition 1)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.empty_like(v)
    out[:n_orth] = np.maximum(v[:n_orth], 0.0)
    heads, t, off = _soc_heads_and_tail_norms(v, n_orth, soc_dims)
    if heads.size == 0:
        return out
    inside = t <= heads
    polar = (~inside) & (t <= -heads)
    mid = ~(inside | polar)
    a = np.where(mid, 0.5 * (heads + t), 0.0)
    # per-cone factor applied to the tail; head value set separately
    tail_factor = np.where(inside, 1.0, np.where(mid, a / np.where(mid, t, 1.0), 0.0))
    head_value = np.where(inside, heads, a)
    dims = np.diff(off)
    factor = np.repeat(tail_factor, dims)
    out[n_orth:] = v[n_orth:] * factor
    out[off[:-1]] = head_value
    return out


def abs_K(v: np.ndarray, n_orth: int, soc_dims) -> np.ndarray:
    """abs_K(v) = 2 proj_K(v) - v (Definition 1); for R+ this is |v|."""
    return 2.0 * proj_K(v, n_orth, soc_dims) - v


def dist_K(v: np.ndarray, n_orth: int, soc_dims) -> float:
    """Euclidean distance from v to K."""
    return float(np.linalg.norm(v - proj_K(v, n_orth, soc_dims)))


def cone_identity(n: int, n_orth: int, soc_dims) -> np.ndarray:
    """e: 1 on every orthant coordinate and (1, 0, ..., 0) on every Lorentz cone."""
    e = np.zeros(n)
    e[:n_orth] = 1.0
    off = soc_offsets(n_orth, soc_dims)
    e[off[:-1]] = 1.0
    return e


def heads_and_tail_norms(v: np.ndarray, n_orth: int, soc_dims):
    """Per cone (orthant coordinates first, each a cone of size 1): v_{h+1} and
    ||(v_{h+2}, ..., v_{h+n_i})||, plus the size of every cone."""
    heads_s, t_s, off = _soc_heads_and_tail_norms(v, n_orth, soc_dims)
    heads = np.concatenate([v[:n_orth], heads_s])
    tails = np.concatenate([np.zeros(n_orth), t_s])
    sizes = np.concatenate([np.ones(n_orth, dtype=np.int64), np.diff(off)])
    return heads, tails, sizes
