#!/usr/bin/env python3
"""Throughput benchmark of the GB300 adaptive-conditioning conic solver.

One step = one complete solve (Algorithm 2 from x = z = e to every relative
KKT residual <= 1e-6) of the large sparse LP: m = 200,000 constraints,
n = 1,000,000 variables, 10 nonzeros per column with N(0,1) values, rows
scaled by 10^U[-2,2], planted optimum with 30% of x* positive, conditioning
schedule L = {300, 400, ...}, t = 9.2, mu = 1.  The matrix (A and A' in FP32
and FP64, about 0.6 GB) is larger than L2, so no flush is needed between
steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (one solve per rank per
step, no collective on the data path): value = solves of all ranks / max time.
The reference arm times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload and extrapolates to solves/s.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s at 1e-6 KKT resid"
UNIT = "solves/s"
TOL = 1e-6
MAX_ITER = 5000
# The FP64 oracle run to completion once on this instance (single thread):
# 340 iterations to 1e-6, of which the 299 before the first rescaling cost
# about 2.55 s each and the 41 after it about 34.5 s each (its CG then starts
# from zero on an ill-conditioned M).  The benchmark times the first
# iterations live and scales the later ones by that measured ratio.
ORACLE_ITERS_LARGE_LP = 340
ORACLE_PRE_COND_ITERS = 299
ORACLE_LATE_COST_RATIO = 13.5
# The SOCP has not been run to completion by the oracle (it would take days):
# its sample is extrapolated to the 1550 iterations the GPU solve takes to
# 1e-6, with the iterations after the first rescaling (l = 200 under the SOCP
# schedule) costed like the early ones, which understates the oracle's time.
GPU_ITERS_SOCP = 1550
SOCP_PRE_COND_ITERS = 199
# Batch and served stream: a size-stratified sample of this many members or
# distinct requests.  Batch members (m <= 2000) are solved to completion.
# Served requests reach m = 1e5, which the oracle cannot finish in bounded
# time: their first iterations are timed and extrapolated to the oracle's
# median iteration count for their type, measured once on the 22 of the 48
# distinct requests with m <= 2500 (LPs 330 under the LP schedule, requests
# with cones 270 under the SOCP schedule), every iteration costed like the
# sampled ones (which understates the large LPs after their rescaling).
CPU_SAMPLE_MEMBERS = 12
ORACLE_ITERS_SERVE_LP = 330
ORACLE_ITERS_SERVE_SOC = 270
SERVE_DISTINCT = 48

WORKLOADS = {
    "large_lp": dict(desc="LP m=200000 n=1000000 nnz=1e7 (10/col, N(0,1), row scales 10^U[-2,2], 30% x* > 0)",
                     settings=dict(cond_first=300, cond_period=100, t=9.2, mu=1.0)),
    "socp": dict(desc="SOCP 20000 Lorentz cones dims U{3..64} + 100000 orthant, m=150000, 8 nnz/col",
                 settings=dict(cond_first=200, cond_period=100, t=1.7, mu=1.0)),
    "small_lp": dict(desc="LP m=200 n=500 5% density, |supp x*|=150",
                     settings=dict(cond_first=300, cond_period=100, t=9.2, mu=1.0)),
    "serve": dict(desc="Poisson stream of mixed LP/SOCP requests: m log-uniform [100,1e5], n=3m, 5-10 nnz/col, "
                       "half with Lorentz cones dims U{3..64}; 60 GiB admission budget",
                  settings=dict(cond_first=300, cond_period=100, t=9.2, mu=1.0)),
    "batch": dict(desc="4096 LPs in one persistent launch: m log-uniform [50,2000], n=2.5m, 2% density, "
                       "N(0,1); members 0..1023 share one 1000x2500 A",
                  settings=dict(cond_first=300, cond_period=100, t=9.2, mu=1.0)),
    "dense_lp": dict(desc="dense LP of Section V-A: m=floor(0.8n), A U[-1,1], b=A|xdot|, xdot and c N(0,1)",
                     settings=dict(cond_first=300, cond_period=100, t=9.2, mu=1.0)),
    "dense_socp": dict(desc="dense SOCP of Section V-C: m=floor(0.8n), A U[-1,1], b=A abs_K(xdot), xdot and "
                            "c U[0,1], Lorentz cones of size h",
                       settings=dict(cond_first=200, cond_period=100, t=1.7, mu=1.0)),
}
DENSE_N = {"dense_lp": 10000, "dense_socp": 2900}
# LP crossover polish inside the solve (setting polish_tol): on for the sparse
# LPs, whose supports settle early; off for the dense LP, whose polish systems
# (square A_B of m = 8000 > 4096, CG) do not converge, and for cones
POLISH_TOL = {"large_lp": 2e-2, "small_lp": 1e-2}
BATCH_MAX_ITER = 5000       # per member; members not solved by then count as unsolved
def nproc() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def make_instance(name: str, dense_n: int | None = None, cone_h: int = 10, lp_scale: float = 1.0):
    from paper_2103_00736_gb300 import instances as I
    if name == "dense_lp":
        return I.dense_lp(dense_n or DENSE_N[name])
    if name == "dense_socp":
        return I.dense_socp(dense_n or DENSE_N[name], cone_h)
    if name == "large_lp":
        return I.large_lp(scale=lp_scale)
    if name == "socp":
        return I.socp()
    if name == "small_lp":
        return I.small_lp()
    raise ValueError(name)


# ---------------------------------------------------------------------------
# algorithmic bytes
# ---------------------------------------------------------------------------

def path_bytes(m: int, n: int, nnz: int, iters: int, cg_iters: int, checks: int, conds: int) -> float:
    """The hot path's algorithmic bytes of one solve by a fixed formula
    (FP32 values and int32 indices of A and A' stored, each
    read once per pass): per outer iteration 16 nnz + 20 n + 12 m (the A and
    A' passes, abs_K, the update), per CG iteration 16 nnz + 8 n + 20 m, per
    KKT check 24 nnz (the FP64 pair of passes), per rescaling 8 nnz."""
    return (iters * (16.0 * nnz + 20 * n + 12 * m) + cg_iters * (16.0 * nnz + 8 * n + 20 * m)
            + checks * 24.0 * nnz + conds * 8.0 * nnz)


def algorithmic_bytes(m: int, n: int, nnz: int, counters, iters: int, n32_A: int = 0, n32_AT: int = 0) -> float:
    """This implementation's own byte model: every pass it actually runs
    (pass counters of the solve), with its FP64 outer passes at 12 bytes a
    nonzero and FP32 outer passes (n32_A, n32_AT) at 8."""
    n_cg_A, n_cg_AT, n64_A, n64_AT, n_cond, n_chk = [int(v) for v in counters]
    b = 0.0
    b += n32_A * (8.0 * nnz + 8 * n + 20 * m)            # FP32 outer passes over A (rhs)
    b += n32_AT * (8.0 * nnz + 8 * m + 48 * n)           # FP32 outer passes over A' (update)
    b += n_cg_AT * (8.0 * nnz + 4 * m + 8 * n)          # t = O^2 A'u: val+col, u gathered, O2 in, t out
    b += n_cg_A * (8.0 * nnz + 4 * n + 8 * m)           # au = A t: val+col, t gathered, au out, u in
    b += n_cg_A * 52.0 * m                               # CG vector step (p, sv, r r/w; au, jinv in; u out; w FP64 r/w)
    b += n64_A * (12.0 * nnz + 8 * n + 20 * m)           # FP64 passes over A (rhs, b_tilde, residual)
    b += n64_AT * (12.0 * nnz + 8 * m + 48 * n)          # FP64 passes over A' (update, q refresh, residual)
    b += iters * 40.0 * n                                # abs_K: s, q, O in; p, g out
    b += n_cond * 100.0 * n                              # rescaling: o, O, c_hat, s recast
    return b


# ---------------------------------------------------------------------------
# accuracy of a returned point (host arithmetic of the bench itself)
# ---------------------------------------------------------------------------

def affine_residuals(inst, x, y, z) -> dict:
    """Relative primal and dual feasibility and duality gap of a returned
    point, from the problem data alone: ||Ax - b|| / (1 + ||b||),
    ||A'y + z - c|| / (1 + ||c||), |c'x - b'y| / (1 + |c'x| + |b'y|), and the
    relative distance of c'x to the planted optimal value."""
    import numpy as np
    A = inst.to_scipy()
    cx, by = float(inst.c @ x), float(inst.b @ y)
    obj = inst.obj_star
    return {"r_p": float(np.linalg.norm(A @ x - inst.b) / (1 + np.linalg.norm(inst.b))),
            "r_d": float(np.linalg.norm(A.T @ y + z - inst.c) / (1 + np.linalg.norm(inst.c))),
            "r_gap": abs(cx - by) / (1 + abs(cx) + abs(by)),
            "obj_rel_err": abs(cx - obj) / (1 + abs(obj))}


def worst_of(rows) -> dict:
    out = {}
    for r in rows:
        for k, v in r.items():
            out[k] = max(out.get(k, 0.0), v)
    return out


# ---------------------------------------------------------------------------
# clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


HBM_SPEC_GBS = 7900.0   # nominal HBM3e bandwidth of one GB300, for context beside the measured peak


def roofline_entry(kernel: str, alg_bytes: float, launch_ms: float, traffic=None, own_bytes=None,
                   **extra) -> dict:
    """The HBM roofline object of a kernel: algorithmic bytes per launch over the
    launch's device time, against the measured copy bandwidth (and, for context,
    the nominal one); traffic = DRAM bytes per launch from an ncu capture of the
    same build, or None.  own_bytes: the implementation's own pass-count model,
    reported beside (not in place of) alg_bytes."""
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel,
           "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": launch_ms,
           "spec_peak": HBM_SPEC_GBS, "frac_of_spec": achieved / HBM_SPEC_GBS,
           "traffic_gbs": traffic / (launch_ms / 1e3) / 1e9 if traffic else None}
    if own_bytes is not None:
        own = own_bytes / (launch_ms / 1e3) / 1e9
        out["own_model"] = {"bytes_per_launch": own_bytes, "achieved": own, "frac": own / peak}
    out.update(extra)
    return out


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def cpu_sample(workload: str, iters: int, dense_n: int | None = None, cone_h: int = 10) -> dict:
    """Time the FP64 oracle on the workload: the first iteration (includes the
    l = 1 conditioning, i.e. the factor/solve set-up) and `iters` further ones;
    the small LP is solved to completion instead (about a second); the batch
    and the served stream are sampled member by member."""
    import numpy as np  # noqa: F401
    from oracle import alg
    if workload == "batch":
        return _cpu_sample_batch(alg, iters)
    if workload == "serve":
        return _cpu_sample_serve(alg, iters)
    inst = make_instance(workload, dense_n, cone_h)
    A = inst.to_scipy()
    st = WORKLOADS[workload]["settings"]
    L = alg.Schedule(first=st["cond_first"], period=st["cond_period"])
    dims = {"m": inst.m, "n": inst.n, "nnz": inst.nnz}
    if workload == "small_lp":
        t0 = time.perf_counter()
        r = alg.algorithm2(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=st["mu"], t=st["t"], L=L,
                           max_iter=MAX_ITER, tol=TOL, check_every=10)
        return {"complete_s": time.perf_counter() - t0, "iters": r.iters, "status": r.status, **dims}
    stamps = []
    t0 = time.perf_counter()

    def hook(l, s, p, O, d):
        stamps.append(time.perf_counter())

    alg.algorithm2(A, inst.b, inst.c, inst.n_orth, inst.soc_dims, mu=st["mu"], t=st["t"], L=L,
                   max_iter=1 + iters, tol=0.0, check_every=10 ** 9, on_iter=hook)
    first = stamps[0] - t0
    per_iter = (stamps[-1] - stamps[0]) / max(1, len(stamps) - 1)
    return {"first_iter_s": first, "per_iter_s": per_iter, "iters": len(stamps), **dims}


def _stratified(sizes, k: int):
    """Indices of k items spread evenly over the items sorted by size."""
    import numpy as np
    order = np.argsort(np.asarray(sizes), kind="stable")
    return [int(i) for i in order[np.linspace(0, len(sizes) - 1, min(k, len(sizes))).astype(int)]]


def _cpu_sample_batch(alg, iters: int) -> dict:
    from paper_2103_00736_gb300 import instances as I
    count = 4096
    sizes = I.batch_sizes(count)
    ms = [1000 if i < count // 4 else sizes[i][0] for i in range(count)]
    st = WORKLOADS["batch"]["settings"]
    L = alg.Schedule(first=st["cond_first"], period=st["cond_period"])
    total, solved, picked = 0.0, 0, []
    for i in _stratified(ms, CPU_SAMPLE_MEMBERS):
        x = I.batch_member(i, count, sizes=sizes)
        A = x.to_scipy()
        t0 = time.perf_counter()
        r = alg.algorithm2(A, x.b, x.c, x.n_orth, x.soc_dims, mu=st["mu"], t=st["t"], L=L,
                           max_iter=BATCH_MAX_ITER, tol=TOL, check_every=10)
        total += time.perf_counter() - t0
        solved += r.status == "solved"
        picked.append(x.m)
    return {"members_s": total, "members": len(picked), "solved": solved, "m_min": min(picked),
            "m_max": max(picked), "count": count}


def _cpu_sample_serve(alg, iters: int) -> dict:
    from paper_2103_00736_gb300 import instances as I
    kinds = [I.serve_request_kind(i) for i in range(SERVE_DISTINCT)]
    total, picked = 0.0, []
    for i in _stratified([m for m, _ in kinds], CPU_SAMPLE_MEMBERS):
        m, soc = kinds[i]
        x = I.serve_request(i)
        A = x.to_scipy()
        st = WORKLOADS["socp" if soc else "serve"]["settings"]
        L = alg.Schedule(first=st["cond_first"], period=st["cond_period"])
        stamps = []
        t0 = time.perf_counter()
        alg.algorithm2(A, x.b, x.c, x.n_orth, x.soc_dims, mu=st["mu"], t=st["t"], L=L, max_iter=1 + iters,
                       tol=0.0, check_every=10 ** 9, on_iter=lambda *a: stamps.append(time.perf_counter()))
        per = (stamps[-1] - stamps[0]) / max(1, len(stamps) - 1)
        n_it = ORACLE_ITERS_SERVE_SOC if soc else ORACLE_ITERS_SERVE_LP
        total += (stamps[0] - t0) + (n_it - 1) * per
        picked.append(m)
    return {"requests_s": total, "requests": len(picked), "m_min": min(picked), "m_max": max(picked),
            "distinct": SERVE_DISTINCT}


def run_cpu_sample_subprocess(workload: str, iters: int, threads: int = 1, dense_n: int | None = None,
                              cone_h: int = 10) -> dict:
    """The oracle sample in a child process whose BLAS / OpenMP pools have
    `threads` threads (the oracle's sparse products run on one core either way;
    its dense factorisations and vector operations use the pool)."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload, "--cpu-iters",
           str(iters), "--cone-h", str(cone_h)]
    if dense_n:
        cmd += ["--dense-n", str(dense_n)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("cpu sample failed: " + r.stderr[-2000:])


def oracle_baseline(workload: str, args, rank: int, world: int, gpu_iters: int | None = None):
    """The cpu_baseline object of a bench line (rank 0 of a 1-GPU run only)."""
    if rank != 0 or world != 1 or args.no_cpu:
        return None
    return oracle_runs(workload, args.cpu_iters, getattr(args, "dense_n", None), getattr(args, "cone_h", 10),
                       gpu_iters)


def oracle_runs(workload: str, iters: int, dense_n: int | None = None, cone_h: int = 10,
                gpu_iters: int | None = None) -> dict:
    """The oracle timed on one host thread and on all of them; the line's
    value is the faster of the two, and both are listed."""
    runs = []
    for threads in sorted({1, nproc()}):
        sample = run_cpu_sample_subprocess(workload, iters, threads, dense_n, cone_h)
        v, desc = oracle_solves_per_s(sample, workload, threads, gpu_iters)
        runs.append({"value": v, "cores": threads, "sample": desc})
    best = max(runs, key=lambda r: r["value"])
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": best["sample"], "runs": runs, "host_cores": nproc()}


def oracle_solves_per_s(sample: dict, workload: str, threads: int = 1,
                        gpu_iters: int | None = None) -> tuple[float, str]:
    if "members_s" in sample:
        return sample["solved"] / sample["members_s"], (
            f"FP64 oracle, {threads} thread(s): {sample['members']} of the {sample['count']} members, stratified by size "
            f"(m {sample['m_min']}..{sample['m_max']}), solved one after another to {TOL:g} KKT within "
            f"{BATCH_MAX_ITER} iterations each: {sample['solved']} solved in {sample['members_s']:.1f} s; "
            f"the batch's rate taken as the sample's")
    if "requests_s" in sample:
        return sample["requests"] / sample["requests_s"], (
            f"FP64 oracle, {threads} thread(s): {sample['requests']} of the {sample['distinct']} distinct requests, "
            f"stratified by size (m {sample['m_min']}..{sample['m_max']}); each one's first iterations timed "
            f"and extrapolated to the oracle's median count for its type ({ORACLE_ITERS_SERVE_LP} for LPs, "
            f"{ORACLE_ITERS_SERVE_SOC} with cones), every iteration costed like the sampled ones: "
            f"{sample['requests_s']:.1f} s for the sample, one request after another")
    if "complete_s" in sample:
        return 1.0 / sample["complete_s"], (f"FP64 oracle, {threads} thread(s): complete solve to {TOL:g} KKT, "
                                            f"{sample['iters']} iterations ({sample['status']}), "
                                            f"{sample['complete_s']:.2f} s")
    t = sample["per_iter_s"]
    head = (f"FP64 oracle, {threads} thread(s), EXTRAPOLATED from {sample['iters']} timed iterations: "
            f"first iteration {sample['first_iter_s']:.1f} s, {sample['iters'] - 1} more at {t:.2f} s each; ")
    if workload == "large_lp":
        n_it, n_pre, ratio = ORACLE_ITERS_LARGE_LP, ORACLE_PRE_COND_ITERS, ORACLE_LATE_COST_RATIO
        how = (f"extrapolated to the {n_it} iterations the oracle needs for this instance, the "
               f"{n_it - n_pre} after the first rescaling at {ratio}x the measured cost (ratio from a "
               f"complete oracle run)")
    elif workload == "socp":
        n_it, n_pre, ratio = GPU_ITERS_SOCP, SOCP_PRE_COND_ITERS, 1.0
        how = (f"extrapolated to the {n_it} iterations the GPU solve takes (the oracle has not been run "
               f"to completion on this instance), every iteration costed like the sampled ones")
    elif workload in ("dense_lp", "dense_socp") and gpu_iters:
        n_it, n_pre, ratio = int(gpu_iters), int(gpu_iters), 1.0
        how = (f"extrapolated to the {n_it} iterations the GPU solve takes, every iteration costed like "
               f"the sampled ones")
    else:
        raise ValueError(f"no CPU baseline for workload {workload}")
    t_solve = sample["first_iter_s"] + (n_pre - 1) * t + (n_it - n_pre) * ratio * t
    return 1.0 / t_solve, head + how


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def max_over_ranks(x: float, pg=None, device: str = "cpu") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's);
    x itself without a process group.  device: "cuda" under NCCL, "cpu"
    under gloo."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / seconds_max


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


PRECISIONS = {"mixed": 0, "fp32": 1, "fp64": 2}


def polish_tol(args) -> float:
    if args.no_polish:
        return 0.0
    if args.polish_tol is not None:
        return args.polish_tol
    return POLISH_TOL.get(args.workload, 0.0)


def polish_bytes(m: int, n: int, nnz: int, corrections: int, attempts: int, support: int = 0,
                 support_entries: int = 0, cg_entry_bytes: float = 12.0) -> float:
    """Algorithmic bytes of the crossover polishes of one solve.  Their CG
    passes read only the support's part of the matrix (A_B, and the rows of A'
    on B): per CG iteration 2 x cg_entry_bytes per entry of A_B (12 with FP64
    corrections, 8 with the FP32 ones of a polished solve), the support's
    vectors and the m-vectors of the vector step; per polish about 10 FP64
    passes on the support (support, Jacobi, the rounds' residuals and q
    refreshes) and 4 over all of A (z_y, z, KKT).  Without the support figures
    (support_entries = 0: the factored path) every pass counts all of A."""
    nb = support_entries if support_entries > 0 else nnz
    nB = support if support_entries > 0 else n
    per_cg = 2 * (cg_entry_bytes * nb) + 16.0 * (m + nB) + 56.0 * m
    per_support_pass = 12.0 * nb + 16.0 * (m + nB)
    per_full_pass = 12.0 * nnz + 16.0 * (m + n)
    return corrections * per_cg + attempts * (10 * per_support_pass + 4 * per_full_pass)


def pinned_copy(a, keep: list):
    """A copy of the numpy array a in page-locked host memory: the numpy view
    of a pinned torch buffer, which is appended to keep (the view's owner)."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(a)
    t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True)
    keep.append(t)
    v = t.numpy()
    v[...] = a
    return v


def solver_overrides(args) -> dict:
    """Settings chosen on the command line (precision mode, column blocks,
    crossover polish)."""
    out = {"polish_tol": polish_tol(args)}
    if args.precision is not None:
        out["precision"] = PRECISIONS[args.precision]
    if args.col_block is not None:
        out["col_block"] = args.col_block
    return out


SUB_TOL = 2e-7          # the batched and served records: relative objective error <= 1e-6 needs it


def sub_records(args) -> dict:
    """The batched and served forms at the accuracy bar, beside the large LP:
    a 1024-member batch of the batched recipe (batched against the plain
    single-problem form, size-stratified sample) and one saturation-rate
    point of the served stream (served against plain, p50/p99)."""
    import argparse as _ap
    out = {}
    b = _ap.Namespace(**vars(args))
    b.batch_count, b.steps, b.warmup, b.tol, b.plain_sample = 1024, 2, 3, SUB_TOL, 12
    b.no_e2e, b.no_cpu = True, True
    L = batch_arm(b, emit=False)
    out["batch"] = {"workload": "batch of 1024 (batched recipe: m log-uniform [50, 2000], n = 2.5 m, 2 %, "
                                "a quarter sharing one 1000 x 2500 A)",
                    "value": L["value"], "unit": UNIT, "ms_per_step": L["ms_per_step"], "steps": b.steps,
                    "warmup": b.warmup, "tol": SUB_TOL, "members": L["config"]["members"],
                    "solved": L["config"]["solved"], "plain": L["plain"],
                    "batched_over_plain": L["batched_over_plain"],
                    "accuracy_sampled_max": L["config"]["accuracy_sampled_max"],
                    "mapping": L["config"]["mapping"], "cuda_graph": L["config"]["cuda_graph"],
                    "roofline": L["roofline"], "clocks": L["clocks"]}
    v = _ap.Namespace(**vars(args))
    v.rates, v.serve_requests, v.serve_distinct, v.tol, v.no_cpu = "2000", 96, 48, SUB_TOL, True
    L = serve_arm(v, emit=False)
    pt = L["sweep"][0]
    out["served"] = {"workload": "served stream at 2000 requests/s (saturation), 96 requests over 48 distinct "
                                 "mixed LP/SOCP requests, m log-uniform [100, 1e5]",
                     "value": pt["solves_per_s"], "unit": UNIT, "p50_ms": pt["p50_ms"], "p99_ms": pt["p99_ms"],
                     "solved": pt["solved"], "requests": pt["requests"], "tol": SUB_TOL, "plain": L["plain"],
                     "served_over_plain": L["served_over_plain"], "accuracy_max": L["config"]["accuracy_max"],
                     "rounds": pt["rounds"], "clocks": L["clocks"]}
    return out


def gpu_arm(args) -> None:
    import numpy as np
    import torch
    from paper_2103_00736_gb300 import capi

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    inst = make_instance(args.workload, args.dense_n, args.cone_h, args.lp_scale)
    wl = WORKLOADS[args.workload]
    # a dedicated stream: the library launches on it and the events below time it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    settings = capi.acs_settings_default(cuda_stream=stream.cuda_stream, device=local, **wl["settings"],
                                         **solver_overrides(args))
    h = capi.acs_problem_create(inst.m, inst.n, inst.row_ptr, inst.col, inst.val, inst.b, inst.c,
                                inst.n_orth, inst.soc_dims, settings)
    info = capi.acs_problem_info(h)
    layout = capi.acs_debug_layout(h)

    tol, max_iter = args.tol, args.max_iter
    expect = capi.SOLVED if tol > 0 else capi.MAX_ITER
    ptol = polish_tol(args)
    polished = ptol > tol and inst.n_orth == inst.n

    def solve_checked():
        if polished:            # blocking: the host decides between segments and polishes
            capi.acs_solve(h, tol, max_iter)
        else:
            capi.acs_solve_async(h, tol, max_iter)

    for _ in range(args.warmup):
        solve_checked()
    st, iters, res = capi.acs_get_residuals(h)
    if st != expect:
        raise RuntimeError(f"warm-up solve did not converge: {capi.acs_status_string(st)} {res}")
    counters = capi.acs_debug_counters(h)
    launch_ms_warm = capi.acs_last_launch_ms(h)
    phases = capi.acs_debug_phase_times(h) if args.phases else None
    passes = capi.acs_debug_pass_counts(h)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    ev0.record(stream)
    for k in range(args.steps):
        step_ev[k][0].record(stream)
        solve_checked()
        step_ev[k][1].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if pg:
        pg.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    launch_ms = capi.acs_last_launch_ms(h)
    polish_ms = capi.acs_last_polish_ms(h) if polished else 0.0
    st, iters, res = capi.acs_get_residuals(h)
    if st != expect:
        raise RuntimeError(f"timed solve did not converge: {capi.acs_status_string(st)}")
    counters = capi.acs_debug_counters(h)
    passes = capi.acs_debug_pass_counts(h)
    _, xs, ys, zs, _, _ = capi.acs_get(h, inst.m, inst.n)
    accuracy = affine_residuals(inst, xs, ys, zs)            # of the timed solve's point
    elapsed_ms = max_over_ranks(elapsed_ms, pg, "cuda")
    value = replica_throughput(world, args.steps, elapsed_ms / 1e3)

    # roofline of the persistent iteration kernel (the only kernel of a solve
    # besides four small initialisation launches; its FP64 continuation
    # launch returns at once unless the FP32 loop handed over): the scope
    # table's byte formula, and beside it the implementation's own model
    own_bytes = algorithmic_bytes(inst.m, inst.n, inst.nnz, counters, iters, passes.get("fp32_outer_A", 0),
                                  passes.get("fp32_outer_At", 0))
    alg_bytes = path_bytes(inst.m, inst.n, inst.nnz, iters, int(res[6]), int(counters[5]), int(counters[4]))
    # every stored entry of every matrix pass costs one random gather from an
    # L2-resident vector: the rate that actually bounds these passes
    n_cg_A, n_cg_AT, n64_A, n64_AT = (int(v) for v in counters[:4])
    n32_A, n32_AT = passes.get("fp32_outer_A", 0), passes.get("fp32_outer_At", 0)
    gathers = (float(n_cg_A + n64_A + n32_A) * info["padded_A"]
               + float(n_cg_AT + n64_AT + n32_AT) * info["padded_AT"])
    traffic = args.traffic
    # the device's random-gather rate, measured now (4 MB vector, L2-resident)
    gather_probe = capi.acs_bench_gather(1 << 20, 0, device=local)

    plain = None
    if polished:
        # the same handle without the polish (acs_solve_async iterates to tol):
        # Algorithm 2 alone, timed the same way
        for _ in range(2):
            capi.acs_solve_async(h, tol, max_iter)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            capi.acs_solve_async(h, tol, max_iter)
        p1.record(stream)
        torch.cuda.synchronize()
        pst, piters, pres = capi.acs_get_residuals(h)
        if pst != expect:
            raise RuntimeError(f"plain solve did not converge: {capi.acs_status_string(pst)}")
        plain_ms = max_over_ranks(p0.elapsed_time(p1), pg, "cuda")
        pc = capi.acs_debug_counters(h)
        plaunch = capi.acs_last_launch_ms(h)
        pbytes = path_bytes(inst.m, inst.n, inst.nnz, piters, int(pres[6]), int(pc[5]), int(pc[4]))
        plain = {"what": "Algorithm 2 alone (no polish), same handle and instance",
                 "value": replica_throughput(world, args.steps, plain_ms / 1e3), "unit": UNIT,
                 "ms_per_step": plain_ms / args.steps, "iterations": piters, "cg_iterations": int(pres[6]),
                 "residual_max": float(max(pres[:4])),
                 "roofline": roofline_entry("iter_kernel<float>", pbytes, plaunch, None,
                                            own_bytes=algorithmic_bytes(inst.m, inst.n, inst.nnz, pc, piters))}

    # end to end through the C ABI with host buffers, every step: upload,
    # solve, read back x, y, s
    e2e = None
    if not args.no_e2e:
        # the step's inputs sit in page-locked host memory (filled once, before
        # the timed region), so that the create step's uploads are DMA copies
        keep = []
        row_ptr_h, col_h, val_h, b_h, c_h = (pinned_copy(a, keep) for a in
                                             (inst.row_ptr, inst.col, inst.val, inst.b, inst.c))
        torch.cuda.synchronize()
        t_e2e = 0.0
        # W untimed steps first, as in the device-timed loop: the first create
        # takes its buffers from cudaMalloc, later ones from the device cache
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            h2 = capi.acs_problem_create(inst.m, inst.n, row_ptr_h, col_h, val_h, b_h,
                                         c_h, inst.n_orth, inst.soc_dims,
                                         capi.acs_settings_default(device=local, **wl["settings"],
                                                                   **solver_overrides(args)))
            st2 = capi.acs_solve(h2, TOL, MAX_ITER)
            out = capi.acs_get(h2, inst.m, inst.n)
            capi.acs_problem_destroy(h2)
            if k >= args.warmup:
                t_e2e += time.perf_counter() - t0
            if st2 != capi.SOLVED:
                raise RuntimeError("e2e solve did not converge")
        # the bytes the create step copied, as the library counted them (the
        # CSR's columns and values, each relabelled row's start and length,
        # slice tables, cone offsets, b, c; read back: A''s slice table and
        # three counts), and x, y, s read back after the solve
        h2d = layout["create_h2d_bytes"]
        d2h = layout["create_d2h_bytes"] + 8 * (2 * inst.n + inst.m)
        t_e2e = max_over_ranks(t_e2e, pg, "cuda")
        e2e = {"value": replica_throughput(world, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "inputs": "pinned host memory",
               "not_counted": "the solve's status and counter record (about 0.5 KB), read about three "
                              "times and written once per solve segment"}
    capi.acs_problem_destroy(h)

    cpu = oracle_baseline(args.workload, args, rank, world, iters)
    subs = sub_records(args) if (args.workload == "large_lp" and not args.no_sub and world == 1 and rank == 0
                                 and tol > 0) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "m": inst.m, "n": inst.n,
                       "nnz": inst.nnz, "tol": tol, "iterations": iters, "cg_iterations": int(res[6]),
                       "accuracy": accuracy,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (A and A' in FP32+FP64 ~0.6 GB)"},
            "gather": {"achieved_g_per_s": gathers / (launch_ms / 1e3) / 1e9,
                       "probe_g_per_s": gather_probe / 1e9,
                       "frac": gathers / (launch_ms / 1e3) / gather_probe,
                       "note": "matrix passes x stored entries / launch time, against random 4-byte "
                               "gathers from an L2-resident 4 MB vector measured in this run "
                               "(acs_bench_gather)"},
            "roofline": roofline_entry("iter_kernel<float>", alg_bytes, launch_ms, traffic, own_bytes=own_bytes,
                                       step_ms_median=statistics.median(step_ms),
                                       bytes_formula="path: iters*(16 nnz+20 n+12 m) + cg*(16 nnz+8 n+20 m)"
                                                     " + checks*24 nnz + rescalings*8 nnz"),
            "clocks": clk,
            "e2e": e2e,
            # per solve: 6 launches per iteration segment (4 resets/initialisations, the FP32 and the
            # FP64 persistent launch); per polish 2 (barrier reset, polish kernel) and 3 more that
            # build A_B when its corrections run CG (no factored M)
            "gpu_launches": (6 * (1 + max(passes.get("polish_attempts", 0) - passes.get("polish_taken", 0), 0))
                             + (5 if passes.get("polish_support_entries", 0) > 0 else 2)
                             * passes.get("polish_attempts", 0)) * args.steps,
            "cpu_baseline": cpu,
            "layout": layout,
            "passes": passes,
        }
        if phases is not None:
            line["phases_ms"] = phases
        if polished:
            line["config"]["polish_tol"] = ptol
            line["polish"] = {
                "what": "LP crossover polish inside the solve: iterate to every KKT residual <= polish_tol, "
                        "polish (support x > z, FP64 projections of x and y), stop if the polished point "
                        "meets tol, else resume",
                "attempts": passes["polish_attempts"], "taken": passes["polish_taken"],
                "cg_iterations": passes["polish_corrections"], "factored": passes["polish_factored"],
                "iteration_launch_ms": launch_ms, "polish_ms": polish_ms,
                "support": passes["polish_support"], "support_entries": passes["polish_support_entries"],
                "roofline": roofline_entry("polish_kernel", polish_bytes(inst.m, inst.n, inst.nnz,
                                                                         passes["polish_corrections"],
                                                                         passes["polish_attempts"],
                                                                         passes["polish_support"],
                                                                         passes["polish_support_entries"],
                                                                         8.0 if passes["polish_support_entries"]
                                                                         else 12.0),
                                           polish_ms, None,
                                           bytes_formula="per CG iteration 16 nnz_B (FP32 corrections) + "
                                                         "16 (m+|B|) + 56 m, per polish 10 x (12 nnz_B + 16 "
                                                         "(m+|B|)) + 4 x (12 nnz + 16 (m+n)); nnz_B = stored "
                                                         "entries of A_B")
                if polish_ms > 0 else None}
            line["no_polish"] = plain
        if subs:
            line.update(subs)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def member_bytes(m: int, n: int, nnz: int, c) -> float:
    """Algorithmic bytes of one member's solve from its pass counters c[8]
    (the byte model of algorithmic_bytes, plus the cached operator: each
    correction reads the inverse factor twice, m^2 doubles in all)."""
    n_cg_A, n_cg_AT, n64_A, n64_AT, n_cond, n_chk, n_dense, n_fact = [float(v) for v in c]
    b = n_cg_AT * (8.0 * nnz + 4 * m + 8 * n) + n_cg_A * (8.0 * nnz + 4 * n + 8 * m + 52.0 * m)
    b += n64_A * (12.0 * nnz + 8 * n + 20 * m) + n64_AT * (12.0 * nnz + 8 * m + 48 * n)
    iters = n64_AT - n_chk - n_cond                 # one FP64 A' update pass per iteration
    b += max(iters, 0.0) * 40.0 * n + n_cond * 100.0 * n
    b += n_dense * 8.0 * m * m
    return b


def batch_arm(args, emit: bool = True) -> dict:
    import numpy as np
    import torch
    from paper_2103_00736_gb300 import capi, instances as I

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    wl = WORKLOADS["batch"]
    t0 = time.perf_counter()
    mem = I.batch(count=args.batch_count)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    settings = capi.acs_settings_default(cuda_stream=stream.cuda_stream, device=local, **wl["settings"])
    share = capi.shared_A_index(mem)
    t0 = time.perf_counter()
    h = capi.acs_batch_create(mem, settings, None, share)
    t_create = time.perf_counter() - t0
    info0 = capi.acs_batch_info(h)
    tol, max_iter = args.tol, args.batch_max_iter
    if args.autotune_iters > 0:
        (th, team), tune_ms = capi.acs_batch_autotune(h, max_iter=args.autotune_iters)
    else:                                        # a fixed mapping (profiling runs)
        th, team = (int(v) for v in args.mapping.split("x"))
        capi.acs_batch_set_mapping(h, th, team)
        tune_ms = np.zeros((3, 3))
    for _ in range(args.warmup):
        capi.acs_batch_solve_async(h, tol, max_iter)
    capi.acs_batch_results(h, len(mem))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        capi.acs_batch_solve_async(h, tol, max_iter)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launch_ms = capi.acs_batch_last_ms(h)
    worst, st, iters, res = capi.acs_batch_results(h, len(mem))
    solved = int(np.sum(st == capi.SOLVED))
    info = capi.acs_batch_info(h)
    cnt = capi.acs_batch_counters(h, len(mem))
    alg_bytes = sum(member_bytes(x.m, x.n, x.nnz, cnt[i]) for i, x in enumerate(mem))
    ms_step = statistics.median(step_ms)
    value = solved / (ms_step / 1e3)
    # accuracy of a sample of solved members, from the problem data
    idx = np.linspace(0, len(mem) - 1, 64).astype(int)
    checked = []
    for i in idx:
        s_i, x, y, z, it_i, r_i = capi.acs_batch_get(h, int(i), mem[i].m, mem[i].n)
        if s_i == capi.SOLVED:
            checked.append(affine_residuals(mem[i], x, y, z))
    accuracy = worst_of(checked)
    capi.acs_batch_destroy(h)

    # plain form: the single-problem API on a size-stratified sample, one
    # solve after another, extrapolated to the whole batch
    order = np.argsort([x.nnz for x in mem])
    sample = order[np.linspace(0, len(mem) - 1, args.plain_sample).astype(int)] if args.plain_sample > 0 else []
    plain_ms, plain_solved, plain_checked = [], 0, []
    for i in sample:
        x = mem[i]
        hs = capi.acs_problem_create(x.m, x.n, x.row_ptr, x.col, x.val, x.b, x.c, x.n_orth, x.soc_dims,
                                     capi.acs_settings_default(cuda_stream=stream.cuda_stream, device=local,
                                                               **wl["settings"]))
        capi.acs_solve(hs, tol, max_iter)                 # warm-up
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        capi.acs_solve_async(hs, tol, max_iter)
        b2.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(a.elapsed_time(b2))
        plain_solved += capi.acs_get_residuals(hs)[0] == capi.SOLVED
        st_p, xp, yp, zp, _, _ = capi.acs_get(hs, x.m, x.n)
        if st_p == capi.SOLVED:
            plain_checked.append(affine_residuals(x, xp, yp, zp))
        capi.acs_problem_destroy(hs)
    if len(sample):
        plain_total_ms = float(np.mean(plain_ms)) * len(mem)
        plain_value = (plain_solved / len(sample)) * len(mem) / (plain_total_ms / 1e3)
    else:
        plain_ms, plain_value = [0.0], 0.0

    # end to end through the C ABI with host buffers: create (host preparation
    # and upload), solve, read back every member's x, y, s
    e2e = None
    if not args.no_e2e:
        t0 = time.perf_counter()
        h2 = capi.acs_batch_create(mem, capi.acs_settings_default(device=local, **wl["settings"]),
                                   (th, team), share)
        capi.acs_batch_solve(h2, tol, max_iter)
        for i, x in enumerate(mem):
            capi.acs_batch_get(h2, i, x.m, x.n)
        capi.acs_batch_destroy(h2)
        t_e2e = time.perf_counter() - t0
        h2d = 16 * info0["stored_nnz"] * 2 + 8 * (info0["sum_m"] + info0["sum_n"])
        d2h = 8 * (2 * info0["sum_n"] + info0["sum_m"])
        e2e = {"value": solved / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
    it_s = iters[st == capi.SOLVED]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch", "desc": wl["desc"], "members": len(mem),
                   "distinct_matrices": info0["matrices"], "sum_m": info0["sum_m"], "sum_n": info0["sum_n"],
                   "stored_nnz_distinct": info0["stored_nnz"], "tol": tol, "max_iter": max_iter,
                   "solved": solved, "iterations_median": float(np.median(it_s)) if it_s.size else None,
                   "iterations_p90": float(np.percentile(it_s, 90)) if it_s.size else None,
                   "mapping": {"threads_per_cta": th, "team_ctas": team, "teams": info["teams"],
                               "ctas": info["ctas"]},
                   "autotune_ms": tune_ms.tolist(), "cuda_graph": bool(info["graph"]),
                   "accuracy_sampled_max": accuracy, "generate_s": t_gen, "create_s": t_create,
                   "l2": "inputs larger than L2 (distinct matrices ~2.6 GB)"},
        "plain": {"value": plain_value, "unit": UNIT, "sample": int(len(sample)),
                  "sample_solved": int(plain_solved), "mean_ms": float(np.mean(plain_ms)),
                  "accuracy_max": worst_of(plain_checked),
                  "how": "single-problem API, one member after another, size-stratified sample "
                         "extrapolated to all members"},
        "batched_over_plain": value / plain_value if plain_value > 0 else None,
        "roofline": roofline_entry("batch_kernel", alg_bytes, launch_ms),
        "clocks": clk, "e2e": e2e, "gpu_launches": 3 * args.steps,
        "cpu_baseline": oracle_baseline("batch", args, rank, world),
    }
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def serve_arm(args, emit: bool = True) -> dict:
    """Continuous batching under a Poisson stream: for each arrival rate, the
    stream's requests are submitted at their arrival times by client threads;
    latency runs from the scheduled arrival to the results in host memory."""
    import numpy as np
    import torch
    from paper_2103_00736_gb300 import capi, instances as I

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    reqs = [I.serve_request(i) for i in range(args.serve_distinct)]
    t_gen = time.perf_counter() - t0
    rates = [float(r) for r in args.rates.split(",")]
    cfg = dict(budget_bytes=60 << 30, round_ms=args.round_ms)

    # plain form: the same requests one after another through the
    # single-problem API (create, solve, read back), each with its schedule
    t0 = time.perf_counter()
    plain_ok = 0
    plain_checked = []
    for r in reqs:
        sched = capi.SOCP_SCHEDULE if len(r.soc_dims) else capi.LP_SCHEDULE
        with capi.Solver(r, device=local, **sched) as sv:
            st_p = sv.solve(tol=args.tol, max_iter=args.batch_max_iter)
            plain_ok += st_p == capi.SOLVED
            _, xp, yp, zp, _, _ = sv.get()
        if st_p == capi.SOLVED:
            plain_checked.append(affine_residuals(r, xp, yp, zp))
    plain_s = time.perf_counter() - t0
    plain_value = plain_ok / plain_s

    table = []
    clocks = ClockSampler(local)
    with capi.Server(capi.acs_settings_default(device=local), **cfg) as S:
        # warm-up: every distinct request once, each result checked from the data
        ids = [S.submit(r, tol=args.tol, max_iter=args.batch_max_iter) for r in reqs]
        checked, warm_ok = [], 0
        for k, rid in enumerate(ids):
            S.wait(rid, 600.0)
            st, x, y, z, it, res, ms = S.result(rid)
            warm_ok += st == capi.SOLVED
            if st == capi.SOLVED:
                checked.append(affine_residuals(reqs[k], x, y, z))
        accuracy_warmup = worst_of(checked)
        clocks.start()
        for ri, rate in enumerate(rates):
            n_req = args.serve_requests
            arr = I.poisson_arrivals(n_req, rate, seed=I.seed_for(I.K_SERVE, 900_000 + ri))
            before = S.stats()
            subm = {}
            lock = threading.Lock()
            start = time.perf_counter() + 0.05

            def client(ks):
                for k in ks:
                    dt = start + arr[k] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    lag = time.perf_counter() - (start + arr[k])
                    rid = S.submit(reqs[k % len(reqs)], tol=args.tol, max_iter=args.batch_max_iter)
                    with lock:
                        subm[k] = (rid, max(lag, 0.0))

            th = [threading.Thread(target=client, args=(list(range(j, n_req, args.clients)),))
                  for j in range(args.clients)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            lat, done_at, ok = [], [], 0
            for k in range(n_req):
                rid, lag = subm[k]
                S.wait(rid, 1200.0)
                st, x, y, z, it, res, ms = S.result(rid)
                ok += st == capi.SOLVED
                if st == capi.SOLVED:
                    checked.append(affine_residuals(reqs[k % len(reqs)], x, y, z))
                lat.append(lag * 1e3 + ms)
                done_at.append(arr[k] + lag + ms / 1e3)
            span = max(done_at) - arr[0]
            after = S.stats()
            lat = np.array(lat)
            table.append({"rate": rate, "requests": n_req, "solved": int(ok), "solves_per_s": ok / span,
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "rounds": int(after["rounds"] - before["rounds"]),
                          "large_alone": int(after["large"] - before["large"]),
                          "mean_active": after["active_mean"], "pool_peak_bytes": int(after["pool_peak_bytes"])})
        clk = clocks.stop()
    accuracy = worst_of(checked)
    best = max(table, key=lambda d: d["solves_per_s"])
    line = {
        "metric": METRIC, "value": best["solves_per_s"], "unit": UNIT, "n_gpus": world, "steps": len(rates),
        "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serve", "desc": WORKLOADS["serve"]["desc"], "distinct_requests": len(reqs),
                   "requests_per_rate": args.serve_requests, "rates": rates, "round_ms": args.round_ms,
                   "clients": args.clients, "tol": args.tol, "max_iter": args.batch_max_iter,
                   "warmup_solved": int(warm_ok), "accuracy_max": accuracy, "generate_s": t_gen,
                   "schedules": "LP: t=9.2, L={300,400,...}; with cones: t=1.7, L={200,300,...}"},
        "sweep": table,
        "plain": {"value": plain_value, "unit": UNIT, "solved": int(plain_ok), "requests": len(reqs),
                  "accuracy_max": worst_of(plain_checked),
                  "how": "single-problem API, create+solve+read back, one request after another"},
        "served_over_plain": best["solves_per_s"] / plain_value if plain_value > 0 else None,
        "clocks": clk,
        "e2e": {"value": best["solves_per_s"], "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "served throughput is already end to end: host arrays in, results in host memory"},
        "roofline": None,
        "roofline_note": "rounds are timed on the host clock with their bookkeeping; the team kernel's "
                         "roofline is the batch workload's line",
        # one cooperative launch per round; a request run alone takes the
        # single-problem path (four small initialisation launches, the FP32
        # iteration launch and its FP64 continuation)
        "gpu_launches": int(sum(t["rounds"] + 6 * t["large_alone"] for t in table)),
        "cpu_baseline": oracle_baseline("serve", args, rank, world),
    }
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def reference_arm(args) -> None:
    rank, world, local = dist_info()
    if rank != 0:
        return
    t0 = time.perf_counter()
    threads = nproc()
    sample = run_cpu_sample_subprocess(args.workload, max(1, args.steps), threads, args.dense_n, args.cone_h)
    v, desc = oracle_solves_per_s(sample, args.workload, threads)
    cfg = {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "tol": TOL}
    cfg.update({k: sample[k] for k in ("m", "n", "nnz") if k in sample})
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t0,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_lp", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch from an ncu capture of the same kernel build")
    ap.add_argument("--tol", type=float, default=None,
                    help="KKT tolerance of a step (0 with --max-iter: a truncated solve, for profiling); "
                         f"default {TOL:g}, and {SUB_TOL:g} for the batch and serve workloads")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER)
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--batch-max-iter", type=int, default=BATCH_MAX_ITER)
    ap.add_argument("--autotune-iters", type=int, default=20,
                    help="truncated-solve length of each autotuner trial; 0 = use --mapping")
    ap.add_argument("--mapping", default="512x1", help="threads per CTA x CTAs per team (no autotuning)")
    ap.add_argument("--plain-sample", type=int, default=24)
    ap.add_argument("--serve-distinct", type=int, default=48)
    ap.add_argument("--serve-requests", type=int, default=96)
    ap.add_argument("--rates", default="10,30,100,300,1000,2000")
    ap.add_argument("--round-ms", type=float, default=2.0)
    ap.add_argument("--clients", type=int, default=4)
    ap.add_argument("--precision", default=None, choices=sorted(PRECISIONS),
                    help="solver precision mode (default: the library's)")
    ap.add_argument("--col-block", type=int, default=None,
                    help="column-block width limit of the FP32 passes (-1: off; default: the library's)")
    ap.add_argument("--phases", action="store_true", help="add the per-phase device times of a warm-up solve")
    ap.add_argument("--no-sub", action="store_true", help="leave out the batched and served records")
    ap.add_argument("--dense-n", type=int, default=None, help="n of the dense workloads")
    ap.add_argument("--cone-h", type=int, default=10, help="Lorentz cone size of the dense SOCP")
    ap.add_argument("--polish-tol", type=float, default=None,
                    help="LP crossover polish level inside the solve (default per workload: large_lp 2e-2, "
                         "small_lp 1e-2, else off)")
    ap.add_argument("--no-polish", action="store_true", help="Algorithm 2 alone (no crossover polish)")
    ap.add_argument("--lp-scale", type=float, default=1.0,
                    help="size of the large LP relative to m = 2e5, n = 1e6 (smaller cases for profiling)")
    args = ap.parse_args()
    if args.tol is None:
        args.tol = SUB_TOL if args.workload in ("batch", "serve") else TOL
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.workload, args.cpu_iters, args.dense_n, args.cone_h)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
