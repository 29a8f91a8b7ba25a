"""GPU parity of the batched launch (many uneven programs in one persistent
launch) through the C ABI, against the FP64 CPU oracle.

Bars (the same as for a single solve):
  * end results: every member SOLVED; every relative KKT residual <= 1e-6
    when re-evaluated by the oracle's residual function on the returned
    (x, y, z); objective within 1e-6 relative of the planted optimum (solves
    that check the objective stop at a KKT residual of 2e-7: a residual of
    1e-6 alone does not bound the objective error by 1e-6);
  * FP64 iterates of members equal the oracle's to 1e-7 relative over the
    first iterations (no rescaling before l = 300 under the LP schedule);
  * a member gives the same answer alone (single-problem launch) and in the
    batch, under every mapping, within the tolerance above.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import alg, kkt  # noqa: E402

LP = dict(cond_first=300, cond_period=100)


def _kkt(inst, x, y, z):
    return kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)


def _worked_example():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    A = np.array(g["A"])
    return I.Instance(m=3, n=5, row_ptr=np.arange(0, 16, 5, dtype=np.int64),
                      col=np.tile(np.arange(5, dtype=np.int32), 3), val=A.reshape(-1),
                      b=np.array(g["b"]), c=np.array(g["c"]), n_orth=5,
                      soc_dims=np.zeros(0, np.int32), x_star=np.array([0, 0, 4.25719522, 0.19851252, 0.51359132]),
                      y_star=np.zeros(3), s_star=np.zeros(5), name="worked")


def _oracle_solves(inst, max_iter=4000):
    r = alg.algorithm2(inst.to_scipy(), inst.b, inst.c, inst.n_orth, inst.soc_dims, L=alg.LP_SCHEDULE,
                       max_iter=max_iter, tol=1e-6, check_every=10)
    return r.status == "solved"


def _mixed_members():
    """Small LP of the paper's recipe, the scaled batch recipe (a quarter
    sharing one A), uneven Bernoulli LPs, and the Section III-A example.
    Members of the batch recipe that the oracle itself does not solve within
    4000 iterations are left out (at 2% density some small members need tens
    of thousands of iterations of Algorithm 2 under the LP schedule)."""
    mem = [I.small_lp()]
    rec = I.batch(count=24, m_shared=300, mmin=50, mmax=600)
    mem += rec[:6] + [r for r in rec[6:] if _oracle_solves(r)]
    mem += [I.bernoulli_lp(I.seed_for(I.K_BATCH, 50_000 + k), m, int(2.5 * m), density=0.05)
            for k, m in enumerate((7, 33, 128))]
    mem.append(_worked_example())
    return mem


@pytest.fixture(scope="module")
def mixed():
    return _mixed_members()


def _check_member(inst, x, y, z, tol=1e-6):
    r = _kkt(inst, x, y, z)
    assert kkt.max_residual(r) <= tol, (inst.name, r)
    if inst.name != "worked":
        assert abs(r["obj_p"] - inst.obj_star) <= 1e-6 * (1 + abs(inst.obj_star)), (inst.name, r)
    return r


@pytest.mark.parametrize("mapping", [(1024, 1), (256, 1), (512, 2), (256, 4)])
def test_batch_end_results(mixed, mapping):
    with capi.Batch(mixed, mapping=mapping, **LP) as B:
        rc = B.solve(tol=2e-7, max_iter=20000)
        worst, st, iters, res = B.results()
        assert rc == capi.SOLVED and np.all(st == capi.SOLVED), (st, iters)
        info = capi.acs_batch_info(B.h)
        assert info["members"] == len(mixed)
        assert info["matrices"] == len(mixed) - 5           # 6 members share one A
        for i, inst in enumerate(mixed):
            s, x, y, z, it, r = B.get(i)
            assert s == capi.SOLVED and it == iters[i]
            ours = _check_member(inst, x, y, z)
            # the library's own record agrees with the oracle's evaluation
            for k, key in enumerate(("r_p", "r_d", "r_gap", "r_cone")):
                assert abs(r[k] - ours[key]) <= 1e-9 + 1e-6 * ours[key], (i, key)
        # the unique optima: the worked example and the small LP
        np.testing.assert_allclose(B.get(len(mixed) - 1)[1], mixed[-1].x_star, atol=1e-4)
        x0 = B.get(0)[1]
        assert np.linalg.norm(x0 - mixed[0].x_star) <= 1e-4 * np.linalg.norm(mixed[0].x_star)


def test_batch_first_iterates_fp64(mixed):
    """FP64 correction solves: iterates of several members after k iterations
    equal the oracle's (exact projections) to 1e-7 relative."""
    pick = [0, 3, 8, len(mixed) - 2]
    sub = [mixed[i] for i in pick]
    refs = [alg.algorithm2(m.to_scipy(), m.b, m.c, m.n_orth, m.soc_dims, L=alg.LP_SCHEDULE,
                           max_iter=20, tol=0.0, keep_x=20) for m in sub]
    with capi.Batch(sub, precision=capi.PREC_FP64, cg_eta=1e-12, cg_tol=0.0, **LP) as B:
        for k in (1, 5, 20):
            rc = B.solve(tol=0.0, max_iter=k)
            assert rc == capi.MAX_ITER
            for i, ref in enumerate(refs):
                s, x, y, z, it, r = B.get(i)
                assert it == k
                xr = ref.x_history[k - 1]
                assert np.linalg.norm(x - xr) <= 1e-7 * np.linalg.norm(xr), (i, k)


def test_batch_member_alone_and_in_batch(mixed):
    """The same member solved by the single-problem launch and inside the
    batch: both converge, objectives agree to 1e-6 relative."""
    with capi.Batch(mixed, **LP) as B:
        assert B.solve(tol=2e-7, max_iter=20000) == capi.SOLVED
        for i in (0, 5, 14):
            inst = mixed[i]
            with capi.Solver(inst, **LP) as s:
                assert s.solve(tol=2e-7, max_iter=20000) == capi.SOLVED
                _, xa, ya, za, _, _ = s.get()
            _, xb, yb, zb, _, _ = B.get(i)
            oa, ob = inst.c @ xa, inst.c @ xb
            assert abs(oa - ob) <= 1e-6 * (1 + abs(oa)), (i, oa, ob)


def test_batch_graph_replay_is_deterministic(mixed):
    with capi.Batch(mixed[:12], mapping=(512, 1), **LP) as B:
        assert B.solve(tol=1e-6, max_iter=20000) == capi.SOLVED
        a = [B.get(i) for i in range(12)]
        assert B.solve(tol=1e-6, max_iter=20000) == capi.SOLVED
        info = capi.acs_batch_info(B.h)
        b = [B.get(i) for i in range(12)]
    for u, v in zip(a, b):
        assert u[4] == v[4]
        np.testing.assert_array_equal(u[1], v[1])
        np.testing.assert_array_equal(u[3], v[3])
    assert info["graph"] == 1                   # replayed from the captured CUDA graph


def test_batch_socp_members():
    """Lorentz cones in the batch: scaled SOCP recipe and served-stream
    requests with cones, under the SOCP schedule."""
    mem = [I.socp(scale=0.002), I.socp(seed=I.seed_for(I.K_SOCP, 7), scale=0.001)]
    mem += [r for r in (I.serve_request(i, mmax=400) for i in range(12)) if r.meta["with_soc"]][:3]
    with capi.Batch(mem, t=1.7, cond_first=200, cond_period=100) as B:
        rc = B.solve(tol=2e-7, max_iter=20000)
        worst, st, iters, res = B.results()
        assert rc == capi.SOLVED, (st, iters)
        for i, inst in enumerate(mem):
            s, x, y, z, it, r = B.get(i)
            _check_member(inst, x, y, z)


def test_batch_autotune_picks_a_valid_mapping(mixed):
    with capi.Batch(mixed, **LP) as B:
        (th, g), ms = capi.acs_batch_autotune(B.h, max_iter=20)
        assert th in (256, 512, 1024) and g in (1, 2, 4)
        assert (ms > 0).any() and np.all(ms[ms >= 0] > 0)
        rc = B.solve(tol=2e-7, max_iter=20000)
        assert rc == capi.SOLVED
        for i in (0, 9, len(mixed) - 1):
            _check_member(mixed[i], *B.get(i)[1:4])
        print("autotune", (th, g), ms)


def test_batch_dense_and_cg_projection_agree(mixed):
    """Members with m <= 256 use the cached dense operator by default; the same
    batch with CG projections everywhere reaches the same optima.  Solved to a
    KKT residual of 1e-7: a residual of 1e-6 alone does not bound the
    objective error by 1e-6 (one member ends 1.7e-6 away at 2e-7 residuals)."""
    sub = [m for m in mixed if m.m <= 256][:8]
    objs = []
    for proj in (capi.PROJ_AUTO, capi.PROJ_CG):
        with capi.Batch(sub, projection=proj, **LP) as B:
            assert B.solve(tol=1e-7, max_iter=50000) == capi.SOLVED
            objs.append([_check_member(inst, *B.get(i)[1:4])["obj_p"] for i, inst in enumerate(sub)])
    np.testing.assert_allclose(objs[0], objs[1], rtol=2e-6, atol=1e-6)


def test_batch_cg_stall_switches_to_cached_operator():
    """Members with 256 < m <= 512 of the batch recipe under CG first
    (dense_max_m = 0): where Jacobi-CG averages more than 40 iterations per
    outer iteration after a rescaling, the member switches to the cached
    operator; every member still reaches the planted optimum."""
    rec = I.batch(count=96, m_shared=300, mmin=50, mmax=600)
    sub = [r for r in rec[24:] if 256 < r.m <= 512][:10]
    with capi.Batch(sub, dense_max_m=0, dense_switch_max_m=1024, dense_switch_cg=40, **LP) as B:
        rc = B.solve(tol=1e-7, max_iter=20000)
        worst, st, iters, res = B.results()
        cnt = capi.acs_batch_counters(B.h, len(sub))
        assert rc == capi.SOLVED, (st, iters)
        for i, inst in enumerate(sub):
            _check_member(inst, *B.get(i)[1:4])
    assert np.all(cnt[:, 0] > 0)                 # every member started with CG
    assert np.any(cnt[:, 7] > 0), cnt            # some switched and factorised
    print("switched:", int(np.sum(cnt[:, 7] > 0)), "of", len(sub))


def test_batch_bf16_storage(mixed):
    """The batched launch with BF16 storage of A (CG projections): same bars."""
    sub = mixed[:10]
    with capi.Batch(sub, projection=capi.PROJ_CG, a_storage=capi.STORE_BF16, **LP) as B:
        assert B.solve(tol=2e-7, max_iter=20000) == capi.SOLVED
        for i, inst in enumerate(sub):
            _check_member(inst, *B.get(i)[1:4])


@pytest.mark.slow
def test_batch_full_size_sampled():
    """The full batched workload (4096 members, m log-uniform in [50, 2000],
    a quarter sharing one 1000 x 2500 A) in the launch the benchmark times:
    at least 85 % solved within 5000 iterations each (3653 measured; the rest
    are small sparse members that the oracle itself solves slowly or not at
    all under the LP schedule), every shared-A member solved, and sampled
    solved members re-evaluated by the oracle's residual function."""
    mem = I.batch(count=4096)
    with capi.Batch(mem, mapping=(512, 1), **LP) as B:
        B.solve(tol=1e-6, max_iter=5000)
        worst, st, iters, res = B.results()
        assert (st == capi.SOLVED).mean() >= 0.85, (st == capi.SOLVED).sum()
        assert np.all(st[:1024] == capi.SOLVED)
        assert np.all((st == capi.SOLVED) | (st == capi.MAX_ITER))
        solved = np.flatnonzero(st == capi.SOLVED)
        for i in solved[np.linspace(0, solved.size - 1, 24).astype(int)]:
            s, x, y, z, it, r = B.get(int(i))
            rr = _kkt(mem[i], x, y, z)
            assert kkt.max_residual(rr) <= 1e-6, (int(i), rr)
