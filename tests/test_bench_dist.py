"""The multi-GPU path of the benchmark on CPU: replicas under a process
group of two gloo ranks (127.0.0.1).  The only collective is the maximum of
the timed region over ranks; the whole-job throughput is the units of all
ranks over that maximum."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, l = bench.dist_info()
    local_ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    v = bench.replica_throughput(w, 3, m / 1e3)
    dist.barrier()
    out.put((r, w, l, m, v))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, l, m, v) in enumerate(res):
        assert (r, w, l) == (rank, world, rank)
        assert m == 150.0                               # both ranks see the maximum
        assert abs(v - world * 3 / 0.150) < 1e-9        # 40 solves/s for the job


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(1, 5, 2.0) == 2.5


def test_affine_residuals_of_the_bench():
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    from paper_2103_00736_gb300 import instances as I
    inst = I.socp(scale=0.001)
    r = bench.affine_residuals(inst, inst.x_star, inst.y_star, inst.s_star)
    assert max(r.values()) < 1e-12, r
    x = inst.x_star + 1e-3 * np.random.default_rng(0).standard_normal(inst.n)
    r = bench.affine_residuals(inst, x, inst.y_star, inst.s_star)
    assert r["r_p"] > 1e-6 and r["obj_rel_err"] > 0
    assert bench.worst_of([{"a": 1.0}, {"a": 3.0, "b": 2.0}]) == {"a": 3.0, "b": 2.0}


def test_roofline_entry():
    import json
    import os
    import bench
    r = bench.roofline_entry("k", 400e9, 200.0, 360e9, step_ms_median=201.0)
    peak = json.load(open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")) else 6800.0
    assert r["achieved"] == 2000.0 and r["peak"] == peak and r["frac"] == 2000.0 / peak
    assert r["frac_of_spec"] == 2000.0 / bench.HBM_SPEC_GBS and r["traffic_gbs"] == 1800.0
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["step_ms_median"] == 201.0
    assert bench.roofline_entry("k", 1e9, 1.0)["traffic_gbs"] is None
    json.dumps(r)


def test_oracle_extrapolation_rules():
    import bench
    s = {"first_iter_s": 5.0, "per_iter_s": 2.0, "iters": 3}
    v, d = bench.oracle_solves_per_s(s, "large_lp")
    n, pre, r = bench.ORACLE_ITERS_LARGE_LP, bench.ORACLE_PRE_COND_ITERS, bench.ORACLE_LATE_COST_RATIO
    assert abs(1 / v - (5.0 + (pre - 1) * 2.0 + (n - pre) * r * 2.0)) < 1e-9
    assert f"{n} iterations the oracle needs" in d
    v, d = bench.oracle_solves_per_s(s, "socp")
    assert abs(1 / v - (5.0 + (bench.GPU_ITERS_SOCP - 1) * 2.0)) < 1e-9
    assert "has not been run to completion" in d
    v, d = bench.oracle_solves_per_s({"complete_s": 0.25, "iters": 310, "status": "solved"}, "small_lp")
    assert v == 4.0 and "complete solve" in d
    with pytest.raises(ValueError):
        bench.oracle_solves_per_s(s, "batch")


def test_oracle_baseline_object():
    """Only rank 0 of a 1-GPU run times the oracle; the object has the
    contract's keys, its value is the faster of the one-thread and the
    all-cores run, and both runs are listed."""
    import argparse
    import bench
    a = argparse.Namespace(no_cpu=False, cpu_iters=2)
    assert bench.oracle_baseline("small_lp", a, 1, 1) is None
    assert bench.oracle_baseline("small_lp", a, 0, 2) is None
    assert bench.oracle_baseline("small_lp", argparse.Namespace(no_cpu=True, cpu_iters=2), 0, 1) is None
    b = bench.oracle_baseline("small_lp", a, 0, 1)
    assert {"value", "unit", "cores", "kind", "sample"} <= set(b)
    assert b["value"] > 0 and b["kind"] == "oracle" and "complete solve" in b["sample"]
    runs = b["runs"]
    assert [r["cores"] for r in runs] == sorted({1, bench.nproc()}) and b["host_cores"] == bench.nproc()
    best = max(runs, key=lambda r: r["value"])
    assert b["value"] == best["value"] and b["cores"] == best["cores"]
    assert all(f"{r['cores']} thread(s)" in r["sample"] for r in runs)
