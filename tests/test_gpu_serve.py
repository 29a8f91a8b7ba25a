"""The serving loop (continuous batching) through the C ABI.

Bars:
  * a request's result is the same served (time-sliced, paused and resumed
    across rounds, in a changing mix) as solved alone in a batched launch of
    the same mapping: same status and iteration count, iterates equal to
    1e-12 relative (the pause/resume is exact);
  * against the single-problem launch (another launch shape): both solved
    (to a KKT residual of 2e-7, which the objective bar needs), objectives
    within 1e-6 relative, and every relative KKT residual of the served
    result <= 1e-6 when re-evaluated by the oracle;
  * admission waits for memory: with a budget that holds a few requests at a
    time every request still finishes; a request that can never fit is
    refused at submission.
"""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402
from oracle import kkt  # noqa: E402

def _kkt(inst, x, y, z):
    return kkt.residuals(inst.to_scipy(), inst.b, inst.c, x, y, z, inst.n_orth, inst.soc_dims)


@pytest.fixture(scope="module")
def requests():
    """Requests of the served-stream recipe (LP and SOCP, m up to 900) plus
    the small LP of the paper's recipe and two uneven batch members."""
    reqs = [I.serve_request(i, mmin=100, mmax=900) for i in range(14)]
    reqs += [I.small_lp()] + I.batch(count=12, m_shared=300, mmin=60, mmax=400)[4:6]
    return reqs


def _serve(reqs, stagger_s=0.002, tol=2e-7, **cfg):
    out = {}
    with capi.Server(**cfg) as S:
        ids = []
        for k, r in enumerate(reqs):
            ids.append(S.submit(r, tol=tol, max_iter=20000))
            if stagger_s and k % 3 == 2:
                time.sleep(stagger_s)           # later ones arrive while earlier ones run
        for k, rid in enumerate(ids):
            assert S.wait(rid, timeout_s=300.0) != capi.ERR_DEVICE_TIMEOUT
            out[k] = S.result(rid)
        stats = S.stats()
    return out, stats


def _alone_in_batches(reqs, tol=2e-7):
    """Each request solved alone in a batched launch of the serving mapping
    (one launch per cone type, each with that type's schedule)."""
    out = {}
    for socp in (False, True):
        ks = [k for k, r in enumerate(reqs) if bool(len(r.soc_dims)) == socp]
        if not ks:
            continue
        sched = capi.SOCP_SCHEDULE if socp else capi.LP_SCHEDULE
        with capi.Batch([reqs[k] for k in ks], mapping=(256, 1), share=[-1] * len(ks), **sched) as B:
            B.solve(tol=tol, max_iter=20000)
            for j, k in enumerate(ks):
                out[k] = B.get(j)
    return out


def test_served_equals_alone(requests):
    """Fixed teams: every round does a request's arithmetic in the same order,
    so the time-sliced, paused and resumed result is the batched-alone one."""
    served, stats = _serve(requests, round_ms=0.25, adaptive_teams=0)
    assert stats["rounds"] > 3 and stats["finished"] == len(requests)
    alone = _alone_in_batches(requests)
    for k, inst in enumerate(requests):
        st, x, y, z, it, res, lat = served[k]
        sb, xb, yb, zb, itb, resb = alone[k]
        assert st == sb == capi.SOLVED, (k, st, sb)
        assert it == itb, (k, it, itb)
        np.testing.assert_allclose(x, xb, rtol=1e-12, atol=1e-12 * np.abs(xb).max())
        np.testing.assert_allclose(y, yb, rtol=1e-12, atol=1e-12 * np.abs(yb).max())
    print("rounds", stats["rounds"], "mean active", stats["active_mean"], "mean round ms", stats["round_ms_mean"])


def test_served_with_adaptive_teams_within_tolerance(requests):
    """Work-sized teams (the default): a request's team changes from round to
    round with the mix, which changes reduction orders; results agree with
    the batched-alone ones within the stated tolerance."""
    served, stats = _serve(requests, round_ms=0.25)
    alone = _alone_in_batches(requests)
    for k, inst in enumerate(requests):
        st, x, y, z, it, res, lat = served[k]
        sb, xb, yb, zb, itb, resb = alone[k]
        assert st == sb == capi.SOLVED, (k, st, sb)
        r = _kkt(inst, x, y, z)
        assert kkt.max_residual(r) <= 1e-6, (k, r)
        ob = inst.c @ xb
        assert abs(r["obj_p"] - ob) <= 1e-6 * (1 + abs(ob)), (k, r["obj_p"], ob)
        assert np.linalg.norm(x - xb) <= 1e-4 * (1 + np.linalg.norm(xb)), k


def test_served_matches_single_problem_launch(requests):
    served, _ = _serve(requests, round_ms=1.0)
    for k, inst in enumerate(requests):
        st, x, y, z, it, res, lat = served[k]
        assert st == capi.SOLVED
        r = _kkt(inst, x, y, z)
        assert kkt.max_residual(r) <= 1e-6, (k, r)
        sched = capi.SOCP_SCHEDULE if len(inst.soc_dims) else capi.LP_SCHEDULE
        with capi.Solver(inst, **sched) as s:
            assert s.solve(tol=2e-7, max_iter=20000) == capi.SOLVED
            _, xa, _, _, _, _ = s.get()
        oa = inst.c @ xa
        assert abs(r["obj_p"] - oa) <= 1e-6 * (1 + abs(oa)), (k, r["obj_p"], oa)
        assert lat > 0


def _bytes_bound(r):
    """An upper bound of a request's pool block: matrix (A and A', padded at
    most 2x, 16 bytes a stored entry), vectors, cached dense scratch, slack."""
    dense = 16 * r.m * r.m if r.m <= 1024 else 0
    return 2 * 2 * r.nnz * 16 + 8 * 32 * (r.m + r.n) + 200 * r.n + 150 * r.m + dense + 64 * 256


def test_admission_waits_for_memory(requests):
    # a budget of about two and a half of the largest requests
    budget = int(2.5 * max(_bytes_bound(r) for r in requests))
    served, stats = _serve(requests, stagger_s=0.0, budget_bytes=budget, round_ms=0.5)
    assert stats["pool_peak_bytes"] <= budget
    assert stats["admitted"] == len(requests) and stats["rounds"] >= 3
    for k, inst in enumerate(requests):
        st, x, y, z, it, res, lat = served[k]
        assert st == capi.SOLVED
        assert kkt.max_residual(_kkt(inst, x, y, z)) <= 1e-6
    with capi.Server(budget_bytes=1 << 20) as S:
        with pytest.raises(capi.AcsError) as e:      # cached factor alone 4 MB: never fits
            S.submit(I.bernoulli_lp(I.seed_for(I.K_SERVE, 77_000), 500, 1250, density=0.02))
        assert e.value.code == capi.ERR_LIMIT


def test_large_requests_run_alone(requests):
    """With large_nnz lowered, the bigger requests take the whole-GPU path
    between rounds; results stay correct."""
    served, stats = _serve(requests, large_nnz=12000, round_ms=0.5)
    assert stats["large"] > 0 and stats["rounds"] > 0
    for k, inst in enumerate(requests):
        st, x, y, z, it, res, lat = served[k]
        assert st == capi.SOLVED
        assert kkt.max_residual(_kkt(inst, x, y, z)) <= 1e-6


def test_poisson_stream_from_several_threads(requests):
    """Requests arriving on a Poisson clock (300/s) from two submitting
    threads; every result is correct and p50 <= p99 latencies are reported."""
    arr = I.poisson_arrivals(len(requests), 300.0)
    lat = {}
    with capi.Server(round_ms=1.0) as S:
        t0 = time.perf_counter()
        ids = {}
        lock = threading.Lock()

        def client(ks):
            for k in ks:
                dt = arr[k] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                rid = S.submit(requests[k], tol=1e-6, max_iter=20000)
                with lock:
                    ids[k] = rid

        th = [threading.Thread(target=client, args=(list(range(j, len(requests), 2)),)) for j in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for k, rid in ids.items():
            assert S.wait(rid, 300.0) == capi.SOLVED
            st, x, y, z, it, res, ms = S.result(rid)
            lat[k] = ms
            assert kkt.max_residual(_kkt(requests[k], x, y, z)) <= 1e-6
    v = np.array(list(lat.values()))
    print("latency p50 %.2f ms p99 %.2f ms" % (np.percentile(v, 50), np.percentile(v, 99)))


@pytest.mark.slow
def test_served_full_recipe_sampled():
    """Requests of the served recipe at full size (m up to 1e5, half with
    cones) through the server with its defaults: every request solved, and
    every result re-evaluated by the oracle's residual function."""
    reqs = [I.serve_request(i) for i in range(16)]
    with capi.Server(budget_bytes=8 << 30) as S:
        ids = [S.submit(r, tol=1e-6, max_iter=5000) for r in reqs]
        for k, rid in enumerate(ids):
            assert S.wait(rid, 600.0) == capi.SOLVED
            st, x, y, z, it, res, lat = S.result(rid)
            r = _kkt(reqs[k], x, y, z)
            assert kkt.max_residual(r) <= 1e-6, (k, reqs[k].m, r)


def test_wait_while_another_thread_takes_the_result(requests):
    """Several threads wait on one request while another takes its result:
    every waiter returns the status or ACS_ERR_ARG (the request is gone),
    never touches a freed request."""
    with capi.Server(round_ms=0.5) as S:
        for k in range(3):
            rid = S.submit(requests[k], tol=1e-6, max_iter=20000)
            got = []
            th = [threading.Thread(target=lambda: got.append(S.wait(rid, 60.0))) for _ in range(6)]
            for t in th:
                t.start()
            m, n = int(requests[k].m), int(requests[k].n)
            while True:                                  # take the result as soon as it exists
                st = capi.acs_server_result(S.h, rid, m, n)[0]
                if st != capi.ERR_ARG:                   # ERR_ARG: not finished yet
                    break
                time.sleep(0.0005)
            for t in th:
                t.join()
            assert st == capi.SOLVED
            assert len(got) == 6 and all(g in (capi.SOLVED, capi.ERR_ARG) for g in got), got
            assert S.wait(rid, 1.0) == capi.ERR_ARG
