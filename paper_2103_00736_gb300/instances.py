"""Seeded synthetic conic programs with a known primal-dual optimum.

This module holds no arithmetic of the solver: it only draws problem data.
Both the CUDA path and the CPU oracle are fed from it, so that the two
sides always see bit-identical inputs.

Every instance is min c'x s.t. Ax = b, x in K, with K the product of an
n_orth-dimensional nonnegative orthant (coordinates [0, n_orth)) followed by
Lorentz cones of sizes ``soc_dims`` (the problem statement of Section II,
Eq. (1)).  An optimal pair is planted: a primal point x* in K, a dual slack
s* in K with x*'s* = 0 per cone, and a free multiplier y*; then
b = A x* and c = A'y* + s*, so (x*, y*, s*) satisfies the KKT system of
Lemma 2 (Eqs. 19a-19c) exactly in exact arithmetic.

Seeds follow one rule: instance i of workload k uses
``SEED_BASE + 1000*k + i`` with numpy's PCG64 ``default_rng``.  The order of
the draws inside each recipe is part of the definition of the instance.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED_BASE = 20210301

# workload index used in the seed rule
K_SMALL_LP, K_LARGE_LP, K_SOCP, K_BATCH, K_SERVE, K_DENSE = 0, 1, 2, 3, 4, 5


def seed_for(k: int, i: int = 0) -> int:
    return SEED_BASE + 1000 * k + i


@dataclass
class Instance:
    """A conic program in CSR form plus its planted optimum."""
    m: int
    n: int
    row_ptr: np.ndarray      # int64 [m+1]
    col: np.ndarray          # int32 [nnz], sorted within each row
    val: np.ndarray          # float64 [nnz]
    b: np.ndarray            # float64 [m]
    c: np.ndarray            # float64 [n]
    n_orth: int
    soc_dims: np.ndarray     # int32 [n_soc], each >= 2
    x_star: np.ndarray       # float64 [n]
    y_star: np.ndarray       # float64 [m]
    s_star: np.ndarray       # float64 [n]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def obj_star(self) -> float:
        return float(self.c @ self.x_star)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.m, self.n))


# --------------------------------------------------------------------------
# sparse helpers (pattern assembly only)
# --------------------------------------------------------------------------

def coo_to_csr(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """Sort (row, col) pairs into CSR; duplicates are not allowed."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate entries in pattern")
    rows = rows[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return row_ptr, cols[order].astype(np.int32), np.asarray(vals, dtype=np.float64)[order]


def _csr_matvec(row_ptr, col, val, x):
    """y = A x for CSR data (used only to derive b from the planted x*)."""
    m = row_ptr.size - 1
    prod = val * x[col]
    out = np.zeros(m)
    nz_rows = np.flatnonzero(np.diff(row_ptr))
    out[nz_rows] = np.add.reduceat(prod, row_ptr[nz_rows]) if prod.size else 0.0
    return out


def _csr_rmatvec(row_ptr, col, val, y, n):
    """x = A' y for CSR data (used only to derive c from the planted y*, s*)."""
    m = row_ptr.size - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(col, weights=val * y[rows], minlength=n)


def _distinct_rows_per_column(rng, m: int, n: int, k: int) -> np.ndarray:
    """k distinct uniform row indices for each of n columns, shape [n, k]."""
    r = rng.integers(0, m, size=(n, k))
    while True:
        r.sort(axis=1)
        dup = np.any(r[:, 1:] == r[:, :-1], axis=1) if k > 1 else np.zeros(n, bool)
        bad = np.flatnonzero(dup)
        if bad.size == 0:
            return r
        r[bad] = rng.integers(0, m, size=(bad.size, k))


def _cover_empty_rows(rng, m: int, n: int, rows: np.ndarray, cols: np.ndarray):
    """Give every empty row one extra entry in a random column (keeps full row rank plausible)."""
    counts = np.bincount(rows, minlength=m)
    empty = np.flatnonzero(counts == 0)
    if empty.size == 0:
        return rows, cols
    extra_c = rng.integers(0, n, size=empty.size)
    return np.concatenate([rows, empty]), np.concatenate([cols, extra_c])


# --------------------------------------------------------------------------
# planted optimum
# --------------------------------------------------------------------------

def _plant_orthant(rng, n: int, frac_pos: float):
    """x*_j ~ U[0.5,2] on a random fraction of coordinates, s*_j ~ U[0.5,2] on the rest."""
    k = int(round(frac_pos * n))
    support = rng.choice(n, size=k, replace=False)
    x = np.zeros(n)
    x[support] = rng.uniform(0.5, 2.0, size=k)
    s = rng.uniform(0.5, 2.0, size=n)
    s[support] = 0.0
    return x, s


def _plant_soc_blocks(rng, dims: np.ndarray):
    """Complementary pairs per Lorentz cone.

    80% of blocks: boundary pair x = a(1,u), s = b(1,-u), u uniform on the unit sphere;
    10%: x interior (x1 = a, |xbar| = a/2) with s = 0; 10%: the mirror (x = 0, s interior).
    """
    xs, ss = [], []
    kind = rng.random(dims.size)
    for d, kd in zip(dims.tolist(), kind.tolist()):
        u = rng.standard_normal(d - 1)
        u /= np.linalg.norm(u)
        a, bb = rng.uniform(0.5, 2.0, size=2)
        x = np.zeros(d)
        s = np.zeros(d)
        if kd < 0.8:
            x[0], x[1:] = a, a * u
            s[0], s[1:] = bb, -bb * u
        elif kd < 0.9:
            x[0], x[1:] = a, 0.5 * a * u
        else:
            s[0], s[1:] = bb, 0.5 * bb * u
        xs.append(x)
        ss.append(s)
    if not xs:
        return np.zeros(0), np.zeros(0)
    return np.concatenate(xs), np.concatenate(ss)


def _finish(name, m, n, row_ptr, col, val, n_orth, soc_dims, x, s, rng, meta=None):
    y = rng.standard_normal(m)
    b = _csr_matvec(row_ptr, col, val, x)
    c = _csr_rmatvec(row_ptr, col, val, y, n) + s
    return Instance(m=m, n=n, row_ptr=row_ptr, col=col, val=val, b=b, c=c,
                    n_orth=int(n_orth), soc_dims=np.asarray(soc_dims, dtype=np.int32),
                    x_star=x, y_star=y, s_star=s, name=name, meta=meta or {})


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def small_lp(seed: int = seed_for(K_SMALL_LP), m: int = 200, n: int = 500,
             density: float = 0.05, n_support: int = 150) -> Instance:
    """Sparse LP, m x n at the given density, N(0,1) entries, |supp x*| = n_support.

    Exactly round(density*m*n) positions drawn uniformly without replacement;
    the whole pattern is re-drawn while any row or column is empty.
    """
    rng = np.random.default_rng(seed)
    nnz = int(round(density * m * n))
    for _ in range(1000):
        pos = rng.choice(m * n, size=nnz, replace=False)
        rows, cols = pos // n, pos % n
        if np.bincount(rows, minlength=m).min() > 0 and np.bincount(cols, minlength=n).min() > 0:
            break
    else:
        raise ValueError("density too low to draw a pattern without empty rows and columns")
    vals = rng.standard_normal(nnz)
    row_ptr, col, val = coo_to_csr(m, n, rows, cols, vals)
    x, s = _plant_orthant(rng, n, n_support / n)
    return _finish(f"lp{m}x{n}", m, n, row_ptr, col, val, n, [], x, s, rng)


def large_lp(seed: int = seed_for(K_LARGE_LP), scale: float = 1.0, nnz_per_col: int = 10,
             row_scale_decades: float = 2.0, frac_pos: float = 0.3) -> Instance:
    """Large sparse LP: m = 200000*scale, n = 1e6*scale, nnz_per_col distinct
    uniform rows per column with N(0,1) values, then rows scaled by
    10^U[-row_scale_decades, row_scale_decades]; 30% of x* positive."""
    rng = np.random.default_rng(seed)
    m = max(int(round(200_000 * scale)), 2)
    n = max(int(round(1_000_000 * scale)), 5)
    r = _distinct_rows_per_column(rng, m, n, nnz_per_col)
    rows = r.reshape(-1)
    cols = np.repeat(np.arange(n), nnz_per_col)
    rows, cols = _cover_empty_rows(rng, m, n, rows, cols)
    vals = rng.standard_normal(rows.size)
    rscale = 10.0 ** rng.uniform(-row_scale_decades, row_scale_decades, size=m)
    vals = vals * rscale[rows]
    row_ptr, col, val = coo_to_csr(m, n, rows, cols, vals)
    x, s = _plant_orthant(rng, n, frac_pos)
    return _finish(f"lp{m}x{n}", m, n, row_ptr, col, val, n, [], x, s, rng,
                   meta={"scale": scale})


def socp(seed: int = seed_for(K_SOCP), scale: float = 1.0, nnz_per_col: int = 8,
         dmin: int = 3, dmax: int = 64) -> Instance:
    """SOCP: a 100000*scale orthant followed by 20000*scale Lorentz cones with
    dims U{dmin..dmax}; m = 150000*scale, nnz_per_col N(0,1) entries per column."""
    rng = np.random.default_rng(seed)
    n_orth = max(int(round(100_000 * scale)), 1)
    n_soc = max(int(round(20_000 * scale)), 1)
    dims = rng.integers(dmin, dmax + 1, size=n_soc).astype(np.int32)
    n = n_orth + int(dims.sum())
    m = max(int(round(150_000 * scale)), 2)
    k = min(nnz_per_col, m)
    r = _distinct_rows_per_column(rng, m, n, k)
    rows = r.reshape(-1)
    cols = np.repeat(np.arange(n), k)
    rows, cols = _cover_empty_rows(rng, m, n, rows, cols)
    vals = rng.standard_normal(rows.size)
    row_ptr, col, val = coo_to_csr(m, n, rows, cols, vals)
    xo, so = _plant_orthant(rng, n_orth, 0.3)
    xc, sc = _plant_soc_blocks(rng, dims)
    x = np.concatenate([xo, xc])
    s = np.concatenate([so, sc])
    return _finish(f"socp{m}x{n}", m, n, row_ptr, col, val, n_orth, dims, x, s, rng,
                   meta={"scale": scale})


def bernoulli_lp(seed: int, m: int, n: int, density: float = 0.02, frac_pos: float = 0.3,
                 pattern_seed: int | None = None) -> Instance:
    """LP with a Bernoulli(density) pattern (>= 1 entry per row and column), N(0,1) values.

    With ``pattern_seed`` the matrix is drawn from that seed (so several
    instances can share one A) and only the planted optimum uses ``seed``.
    """
    rng_a = np.random.default_rng(seed if pattern_seed is None else pattern_seed)
    cells = m * n
    nnz = int(rng_a.binomial(cells, density))
    nnz = max(nnz, max(m, n))
    pos = rng_a.choice(cells, size=nnz, replace=False)
    rows, cols = pos // n, pos % n
    # cover empty rows and columns with one extra entry each
    er = np.flatnonzero(np.bincount(rows, minlength=m) == 0)
    ec = np.flatnonzero(np.bincount(cols, minlength=n) == 0)
    if er.size or ec.size:
        taken = set((rows * n + cols).tolist())
        add_r, add_c = [], []
        for i in er.tolist():
            while True:
                j = int(rng_a.integers(0, n))
                if i * n + j not in taken:
                    taken.add(i * n + j); add_r.append(i); add_c.append(j); break
        for j in ec.tolist():
            while True:
                i = int(rng_a.integers(0, m))
                if i * n + j not in taken:
                    taken.add(i * n + j); add_r.append(i); add_c.append(j); break
        rows = np.concatenate([rows, np.array(add_r, dtype=rows.dtype)])
        cols = np.concatenate([cols, np.array(add_c, dtype=cols.dtype)])
    vals = rng_a.standard_normal(rows.size)
    row_ptr, col, val = coo_to_csr(m, n, rows, cols, vals)
    rng = np.random.default_rng(seed) if pattern_seed is not None else rng_a
    x, s = _plant_orthant(rng, n, frac_pos)
    return _finish(f"lp{m}x{n}", m, n, row_ptr, col, val, n, [], x, s, rng)


def planted_lp(A_csr_row_ptr, col, val, m: int, n: int, seed: int, frac_pos: float = 0.3,
               name: str = "lp") -> Instance:
    """Plant an optimum (x*, y*, s*) for a given CSR matrix (K = R+^n)."""
    rng = np.random.default_rng(seed)
    x, s = _plant_orthant(rng, n, frac_pos)
    return _finish(name, m, n, np.asarray(A_csr_row_ptr, np.int64), np.asarray(col, np.int32),
                   np.asarray(val, np.float64), n, [], x, s, rng)


def batch_sizes(count: int = 4096, mmin: int = 50, mmax: int = 2000, ratio: float = 2.5,
                seed: int = seed_for(K_BATCH, 100_000)):
    """(m, n) for each batch member: m = round(exp U[ln mmin, ln mmax]), n = round(ratio*m)."""
    rng = np.random.default_rng(seed)
    ms = np.rint(np.exp(rng.uniform(math.log(mmin), math.log(mmax), size=count))).astype(int)
    return [(int(m), int(round(ratio * m))) for m in ms]


def batch_member(i: int, count: int = 4096, shared: int | None = None, m_shared: int = 1000,
                 mmin: int = 50, mmax: int = 2000, sizes=None) -> Instance:
    """Member i of batch(count, ...), generated alone (the same arrays)."""
    if shared is None:
        shared = count // 4
    if i < shared:
        m = m_shared
        n = int(round(2.5 * m))
        inst = bernoulli_lp(seed_for(K_BATCH, i), m, n, pattern_seed=seed_for(K_BATCH, 999))
    else:
        m, n = (batch_sizes(count, mmin, mmax) if sizes is None else sizes)[i]
        inst = bernoulli_lp(seed_for(K_BATCH, i), m, n)
    inst.meta["shared_A"] = i < shared
    return inst


def batch(count: int = 4096, shared: int | None = None, m_shared: int = 1000,
          mmin: int = 50, mmax: int = 2000) -> list[Instance]:
    """Uneven LP batch: the first ``shared`` members (default count/4) share one
    A of size m_shared x 2.5*m_shared; the rest draw their own sizes and A."""
    sizes = batch_sizes(count, mmin, mmax)
    return [batch_member(i, count, shared, m_shared, mmin, mmax, sizes) for i in range(count)]


def serve_request_kind(i: int, mmin: int = 100, mmax: int = 100_000) -> tuple[int, bool]:
    """(m, with Lorentz cones) of serve_request(i) without generating it: the
    first two draws of its generator."""
    rng = np.random.default_rng(seed_for(K_SERVE, i))
    m = int(round(math.exp(rng.uniform(math.log(mmin), math.log(mmax)))))
    return m, bool(rng.random() < 0.5)


def serve_request(i: int, mmin: int = 100, mmax: int = 100_000) -> Instance:
    """Request i of the served stream: m log-uniform in [mmin, mmax], n = 3m,
    nnz/col U{5..10}; every other request (by a coin) puts half of n into
    Lorentz cones with dims U{3..64}."""
    rng = np.random.default_rng(seed_for(K_SERVE, i))
    m = int(round(math.exp(rng.uniform(math.log(mmin), math.log(mmax)))))
    n_target = 3 * m
    with_soc = bool(rng.random() < 0.5)
    if with_soc:
        dims = []
        tot = 0
        while tot < n_target // 2:
            d = int(rng.integers(3, 65))
            dims.append(d)
            tot += d
        dims = np.array(dims, dtype=np.int32)
        n_orth = max(n_target - tot, 1)
    else:
        dims = np.zeros(0, dtype=np.int32)
        n_orth = n_target
    n = n_orth + int(dims.sum())
    per_col = rng.integers(5, 11, size=n)
    per_col = np.minimum(per_col, m)
    rows = np.empty(int(per_col.sum()), dtype=np.int64)
    cols = np.repeat(np.arange(n), per_col)
    pos = 0
    for kk in np.unique(per_col).tolist():
        js = np.flatnonzero(per_col == kk)
        r = _distinct_rows_per_column(rng, m, js.size, kk)
        # place column blocks back in column order
        starts = np.concatenate([[0], np.cumsum(per_col)[:-1]])
        idx = (starts[js][:, None] + np.arange(kk)[None, :]).reshape(-1)
        rows[idx] = r.reshape(-1)
        pos += r.size
    rows, cols = _cover_empty_rows(rng, m, n, rows, cols)
    vals = rng.standard_normal(rows.size)
    row_ptr, col, val = coo_to_csr(m, n, rows, cols, vals)
    xo, so = _plant_orthant(rng, n_orth, 0.3)
    xc, sc = _plant_soc_blocks(rng, dims)
    return _finish(f"req{i}", m, n, row_ptr, col, val, n_orth, dims,
                   np.concatenate([xo, xc]), np.concatenate([so, sc]), rng,
                   meta={"with_soc": with_soc})


def poisson_arrivals(count: int, rate: float, seed: int = seed_for(K_SERVE, 999_999)) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def paper_e2_lp(seed: int, m: int = 80, n: int = 100):
    """Dense LP of the conditioning-schedule study (Section IV-A): A ~ N(0,1),
    b = A xdot with xdot ~ U[0,1], c ~ N(0,1), K = R+^n.  No planted optimum.
    Returns (row_ptr, col, val, b, c) with a full dense pattern."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    xdot = rng.uniform(0.0, 1.0, size=n)
    c = rng.standard_normal(n)
    row_ptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), m)
    return row_ptr, col, A.reshape(-1).copy(), A @ xdot, c


def _dense_csr(A: np.ndarray):
    m, n = A.shape
    row_ptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), m)
    return row_ptr, col, A.reshape(-1)


def _no_optimum(m: int, n: int):
    nan = np.full(n, np.nan)
    return nan, np.full(m, np.nan), nan.copy()


def dense_lp(n: int, seed: int | None = None) -> Instance:
    """Dense LP of the paper's LP experiments (Section V-A): m = floor(0.8 n),
    A with i.i.d. entries U[-1,1], b = A |xdot| with xdot ~ N(0,1) i.i.d.,
    c ~ N(0,1) i.i.d., K = R+^n (drawn in that order).  No planted optimum
    (x_star, y_star, s_star are nan); A is stored as a CSR with full rows."""
    rng = np.random.default_rng(seed_for(K_DENSE, n) if seed is None else seed)
    m = (4 * n) // 5
    A = rng.uniform(-1.0, 1.0, size=(m, n))
    xdot = rng.standard_normal(n)
    c = rng.standard_normal(n)
    b = A @ np.abs(xdot)
    row_ptr, col, val = _dense_csr(A)
    xs, ys, ss = _no_optimum(m, n)
    return Instance(m=m, n=n, row_ptr=row_ptr, col=col, val=val, b=b, c=c, n_orth=n,
                    soc_dims=np.zeros(0, np.int32), x_star=xs, y_star=ys, s_star=ss,
                    name=f"dense_lp_{n}", meta={"planted": False})


def _lorentz_reflection(v: np.ndarray, h: int) -> np.ndarray:
    """The paper's abs_K of Definition 1 on a product of Lorentz cones of size
    h, needed by its SOCP recipe to form b (input generation only; neither
    solver uses it): per cone (v1, vbar), t = ||vbar||: v if t <= v1, -v if
    t <= -v1, else (t, (v1 / t) vbar)."""
    V = v.reshape(-1, h).copy()
    t = np.linalg.norm(V[:, 1:], axis=1)
    v1 = V[:, 0].copy()
    inside, polar = t <= v1, t <= -v1
    mid = ~(inside | polar)
    V[polar] = -V[polar]
    V[mid, 0] = t[mid]
    V[mid, 1:] *= (v1[mid] / t[mid])[:, None]
    return V.reshape(-1)


def dense_socp(n: int, h: int, seed: int | None = None) -> Instance:
    """Dense SOCP of the paper's SOCP experiments (Section V-C): n a multiple of
    h, m = floor(0.8 n), A i.i.d. U[-1,1], b = A abs_K(xdot) with xdot ~
    U[0,1] i.i.d., c ~ U[0,1] i.i.d., K = (K_h)^(n/h), K_h the Lorentz cone
    of size h.  No planted optimum."""
    if n % h:
        raise ValueError("n must be a multiple of the cone size h")
    rng = np.random.default_rng(seed_for(K_DENSE, 1_000_000 + 100 * n + h) if seed is None else seed)
    m = (4 * n) // 5
    A = rng.uniform(-1.0, 1.0, size=(m, n))
    xdot = rng.uniform(0.0, 1.0, size=n)
    c = rng.uniform(0.0, 1.0, size=n)
    b = A @ _lorentz_reflection(xdot, h)
    row_ptr, col, val = _dense_csr(A)
    xs, ys, ss = _no_optimum(m, n)
    return Instance(m=m, n=n, row_ptr=row_ptr, col=col, val=val, b=b, c=c, n_orth=0,
                    soc_dims=np.full(n // h, h, np.int32), x_star=xs, y_star=ys, s_star=ss,
                    name=f"dense_socp_{n}_h{h}", meta={"planted": False})
