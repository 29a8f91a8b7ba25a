"""Studies of the paper's experiments run on the GPU (prints one JSON object).

    python -m paper_2103_00736_gb300.studies schedule [--instances 10] [--max-iter 6000]

schedule: the conditioning-schedule experiment of Section IV-A.  Ten seeded
dense LPs of the paper's recipe (80 x 100, A and c ~ N(0,1), b = A xdot with
xdot ~ U[0,1], K = R+^100, t = 9.2, mu = 1) solved to every relative KKT
residual <= 1e-6 under three schedules: no conditioning (L empty; the l = 1
rescaling of x = z = e is the identity), one conditioning at l = 300, and
conditioning at each of the first 50 iterations.  The paper shows the
result only as a figure (iterations to converge per schedule); this prints
the iteration counts per instance and their medians.  An instance that does
not converge within max_iter counts as max_iter + 1.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402

SCHEDULES = {
    "none": dict(cond_first=0),
    "one300": dict(cond_first=0, cond_list=[300]),
    "first50": dict(cond_first=0, cond_list=list(range(1, 51))),
}
E2_SEED_BASE = 50        # instance k of the study: seed_for(K_SMALL_LP, E2_SEED_BASE + k)


def e2_instance(k: int):
    return I.paper_e2_lp(I.seed_for(I.K_SMALL_LP, E2_SEED_BASE + k))


def schedule_study(instances: int = 10, max_iter: int = 6000, tol: float = 1e-6, **settings) -> dict:
    table = {name: [] for name in SCHEDULES}
    status = {name: [] for name in SCHEDULES}
    t0 = time.perf_counter()
    for k in range(instances):
        rp, col, val, b, c = e2_instance(k)
        for name, sched in SCHEDULES.items():
            s = capi.acs_settings_default(t=9.2, mu=1.0, **sched, **settings)
            h = capi.acs_problem_create(80, 100, rp, col, val, b, c, 100, [], s)
            try:
                st = capi.acs_solve(h, tol, max_iter)
                _, iters, _ = capi.acs_get_residuals(h)
            finally:
                capi.acs_problem_destroy(h)
            table[name].append(int(iters) if st == capi.SOLVED else max_iter + 1)
            status[name].append(capi.acs_status_string(st))
    wall = time.perf_counter() - t0
    return {"study": "conditioning schedule (Section IV-A)", "instances": instances, "max_iter": max_iter,
            "tol": tol, "iterations": table, "status": status,
            "median": {k: statistics.median(v) for k, v in table.items()},
            "ordering_holds": statistics.median(table["first50"]) < statistics.median(table["one300"])
            < statistics.median(table["none"]), "wall_s": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["schedule"])
    ap.add_argument("--instances", type=int, default=10)
    ap.add_argument("--max-iter", type=int, default=6000)
    args = ap.parse_args()
    print(json.dumps(schedule_study(args.instances, args.max_iter)), flush=True)


if __name__ == "__main__":
    main()
