"""The seeded synthetic workloads: each recipe produces what it states
(shapes, densities, per-column counts, cone sizes, the shared A of the
batched workload, a complementary planted pair inside the cone), and the
same seed gives the same arrays.  Host only."""
import numpy as np

from oracle import cones
from paper_2103_00736_gb300 import instances as I


def _col_counts(inst):
    return np.bincount(inst.col, minlength=inst.n)


def _row_counts(inst):
    return np.diff(inst.row_ptr)


def _complementary_in_cone(inst, tol=1e-12):
    x, s = inst.x_star, inst.s_star
    assert cones.dist_K(x, inst.n_orth, inst.soc_dims) <= tol
    assert cones.dist_K(s, inst.n_orth, inst.soc_dims) <= tol
    assert abs(x @ s) <= tol * (1 + np.linalg.norm(x) * np.linalg.norm(s))
    # per cone: x_i' s_i = 0 (each term of a sum of nonnegatives is zero)
    assert np.all(np.abs(x[:inst.n_orth] * s[:inst.n_orth]) <= tol)
    off = inst.n_orth + np.concatenate([[0], np.cumsum(inst.soc_dims)]).astype(int)
    for a, e in zip(off[:-1], off[1:]):
        assert abs(x[a:e] @ s[a:e]) <= 1e-10


def test_small_lp_recipe():
    inst = I.small_lp()
    assert (inst.m, inst.n, inst.nnz) == (200, 500, 5000)
    assert _row_counts(inst).min() > 0 and _col_counts(inst).min() > 0
    assert np.count_nonzero(inst.x_star) == 150
    pos = inst.x_star > 0
    assert np.all((inst.x_star[pos] >= 0.5) & (inst.x_star[pos] <= 2.0))
    assert np.all((inst.s_star[~pos] >= 0.5) & (inst.s_star[~pos] <= 2.0))
    _complementary_in_cone(inst)


def test_large_lp_recipe_scaled():
    inst = I.large_lp(scale=0.002)
    assert (inst.m, inst.n) == (400, 2000)
    cc = _col_counts(inst)
    assert cc.min() >= 10                      # 10 distinct rows per column (+ row covers)
    A = inst.to_scipy()
    rn = np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    assert rn.max() / rn.min() > 1e2           # rows scaled over four decades
    assert abs(np.mean(inst.x_star > 0) - 0.3) < 0.05
    _complementary_in_cone(inst)


def test_socp_recipe_scaled():
    inst = I.socp(scale=0.002)
    assert inst.n_orth == 200 and len(inst.soc_dims) == 40
    assert inst.soc_dims.min() >= 3 and inst.soc_dims.max() <= 64
    assert inst.n == inst.n_orth + int(inst.soc_dims.sum())
    assert _col_counts(inst).min() >= 8
    _complementary_in_cone(inst)


def test_batch_recipe():
    mem = I.batch(count=16, m_shared=120, mmin=50, mmax=400)
    shared = mem[:4]
    for x in shared[1:]:
        assert np.array_equal(x.row_ptr, shared[0].row_ptr)
        assert np.array_equal(x.col, shared[0].col) and np.array_equal(x.val, shared[0].val)
        assert not np.array_equal(x.b, shared[0].b)          # their own planted optima
    assert all(x.meta["shared_A"] for x in shared) and not any(x.meta["shared_A"] for x in mem[4:])
    for x in mem:
        assert 50 <= x.m <= 400 or x.m == 120
        assert x.n == int(round(2.5 * x.m))
        assert _row_counts(x).min() > 0 and _col_counts(x).min() > 0
        assert 0.01 < x.nnz / (x.m * x.n) < 0.04                # Bernoulli(2 %) with covers
        _complementary_in_cone(x)


def test_serve_request_recipe():
    reqs = [I.serve_request(i, mmax=2000) for i in range(12)]
    assert any(r.meta["with_soc"] for r in reqs) and not all(r.meta["with_soc"] for r in reqs)
    for r in reqs:
        assert 100 <= r.m <= 2000
        assert r.n == r.n_orth + int(r.soc_dims.sum())
        if r.meta["with_soc"]:
            assert r.soc_dims.min() >= 3 and r.soc_dims.max() <= 64
            assert int(r.soc_dims.sum()) >= (3 * r.m) // 2
        else:
            assert r.n == 3 * r.m and len(r.soc_dims) == 0
        cc = _col_counts(r)
        assert np.percentile(cc, 5) >= 5 and np.percentile(cc, 95) <= 11
        _complementary_in_cone(r)


def test_seeds_reproduce_instances():
    a, b = I.serve_request(5, mmax=500), I.serve_request(5, mmax=500)
    for f in ("row_ptr", "col", "val", "b", "c", "soc_dims"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert I.seed_for(I.K_BATCH, 7) == 20210301 + 3000 + 7


def test_poisson_arrivals():
    t = I.poisson_arrivals(20000, 100.0)
    gaps = np.diff(t)
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.01) < 0.0005                   # rate 100/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05          # exponential gaps


def test_members_generated_alone_equal_the_batch_and_stream():
    mem = I.batch(count=16, m_shared=120, mmin=50, mmax=400)
    for i in (0, 3, 4, 15):
        x = I.batch_member(i, count=16, m_shared=120, mmin=50, mmax=400)
        for f in ("row_ptr", "col", "val", "b", "c", "x_star"):
            assert np.array_equal(getattr(x, f), getattr(mem[i], f)), (i, f)
    for i in range(8):
        r = I.serve_request(i, mmax=1500)
        assert I.serve_request_kind(i, mmax=1500) == (r.m, bool(len(r.soc_dims)))
