"""Studies of the paper's experiments run on the GPU (prints one JSON object).

    python -m paper_2103_00736_gb300.studies schedule [--instances 10] [--max-iter 6000]
    python -m paper_2103_00736_gb300.studies preconditioning [--max-iter 200]

schedule: the conditioning-schedule experiment of Section IV-A.  Ten seeded
dense LPs of the paper's recipe (80 x 100, A and c ~ N(0,1), b = A xdot with
xdot ~ U[0,1], K = R+^100, t = 9.2, mu = 1) solved to every relative KKT
residual <= 1e-6 under three schedules: no conditioning (L empty; the l = 1
rescaling of x = z = e is the identity), one conditioning at l = 300, and
conditioning at each of the first 50 iterations.  The paper shows the
result only as a figure (iterations to converge per schedule); this prints
the iteration counts per instance and their medians.  An instance that does
not converge within max_iter counts as max_iter + 1.

preconditioning: the comparison of Section III-A on its worked example
(3 x 5, K = R+^5, mu = 1): Douglas-Rachford (the iteration of Algorithm 1)
and ADMM (Section III-B) with no preconditioning, the printed Sinkhorn-Knopp
scalings D^SK, E^SK, Ruiz equilibration, and the printed adaptive-conditioning
scaling E^AC (D^AC = I), each run on the scaled data min (Ec)'u s.t.
(DAE)u = Db, u >= 0 with no rescaling of its own (L empty; x = z = e at
l = 1 gives O = I) and mapped back by x = E u.  Prints, per case, the
iterations after which ||x_k - x*|| <= rtol ||x*|| holds for good, x* being
the solver's own solution of the unscaled problem at a KKT level of 1e-13.
The paper shows this only as a figure; its point is that the scaling with
the largest condition number (E^AC, cond 72079) converges fastest.
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


WORKED_A = ((3.57, 3.45, 3.33, 64.24, -72.76),
            (3.45, 3.33, 3.23, 95.14, -23.34),
            (3.33, 3.23, 3.13, 93.53, -17.43))
WORKED_B = (-10.44, 20.65, 22.94)
WORKED_C = (0.37, 1.93, -0.12, -0.38, 1.01)
WORKED_SCALINGS = {                        # (D, E) printed in Section III-A
    "sk": ((0.0217, 0.0215, 0.0222), (0.4722,) * 5),
    "ac": ((1.0, 1.0, 1.0), (0.0792, 0.0884, 14.5484, 292.9524, 316.2179)),
}
SPLITTINGS = {"dr": capi.SPLIT_DR, "admm": capi.SPLIT_ADMM}


def ruiz(A, iters: int = 20):
    """Ruiz equilibration in infinity norms: D <- D / sqrt(row max |DAE|),
    E <- E / sqrt(column max |DAE|), repeated.  Returns (D, E)."""
    import numpy as np
    A = np.abs(np.asarray(A, dtype=np.float64))
    D, E = np.ones(A.shape[0]), np.ones(A.shape[1])
    for _ in range(iters):
        S = D[:, None] * A * E[None, :]
        D = D / np.sqrt(S.max(axis=1))
        E = E / np.sqrt(S.max(axis=0))
    return D, E


def worked_scalings():
    import numpy as np
    out = {"none": (np.ones(3), np.ones(5)), "ruiz": ruiz(WORKED_A)}
    out.update({k: (np.array(d), np.array(e)) for k, (d, e) in WORKED_SCALINGS.items()})
    return out


def solve_dense(A, b, c, tol, max_iter, n_orth=None, soc_dims=(), **settings):
    """Solve a small dense problem through the C ABI; returns (status, x, y, z, iters)."""
    import numpy as np
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    row_ptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), m)
    s = capi.acs_settings_default(**settings)
    h = capi.acs_problem_create(m, n, row_ptr, col, A.reshape(-1), np.asarray(b, float), np.asarray(c, float),
                                n if n_orth is None else n_orth, list(soc_dims), s)
    try:
        st = capi.acs_solve(h, tol, max_iter)
        _, x, y, z, iters, _ = capi.acs_get(h, m, n)
    finally:
        capi.acs_problem_destroy(h)
    return st, x, y, z, iters


def scaled_iterates(D, E, splitting: int, iters, mu: float = 1.0):
    """x = E u after each of the given iteration counts on the worked example
    scaled by D, E (no rescaling: L empty), one solve from x = z = e per count."""
    import numpy as np
    A = (D[:, None] * np.asarray(WORKED_A)) * E[None, :]
    m, n = A.shape
    row_ptr = np.arange(0, m * n + 1, n, dtype=np.int64)
    col = np.tile(np.arange(n, dtype=np.int32), m)
    s = capi.acs_settings_default(cond_first=0, mu=mu, splitting=splitting, precision=capi.PREC_FP64)
    h = capi.acs_problem_create(m, n, row_ptr, col, A.reshape(-1), D * np.asarray(WORKED_B),
                                E * np.asarray(WORKED_C), n, [], s)
    out = []
    try:
        for k in iters:
            st = capi.acs_solve(h, 0.0, int(k))
            if st != capi.MAX_ITER:
                raise RuntimeError(capi.acs_status_string(st))
            _, u, _, _, _, _ = capi.acs_get(h, m, n)
            out.append(E * u)
    finally:
        capi.acs_problem_destroy(h)
    return out


def preconditioning_study(max_iter: int = 200, rtols=(1e-2, 1e-4, 1e-6, 1e-8)) -> dict:
    import numpy as np
    t0 = time.perf_counter()
    st, x_ref, _, _, _ = solve_dense(WORKED_A, WORKED_B, WORKED_C, 1e-13, 100000, precision=capi.PREC_FP64)
    if st != capi.SOLVED:
        raise RuntimeError(capi.acs_status_string(st))
    nref = float(np.linalg.norm(x_ref))
    table = {}
    for sname, (D, E) in worked_scalings().items():
        As = (D[:, None] * np.asarray(WORKED_A)) * E[None, :]
        for pname, split in SPLITTINGS.items():
            xs = scaled_iterates(D, E, split, range(1, max_iter + 1))
            err = [float(np.linalg.norm(x - x_ref)) / nref for x in xs]
            reach = {}
            for rt in rtols:
                k = next((i for i in range(len(err)) if all(e <= rt for e in err[i:])), None)
                reach[f"{rt:g}"] = None if k is None else k + 1
            table[f"{pname}/{sname}"] = {"cond": float(np.linalg.cond(As)), "iterations_to": reach,
                                         "final_error": err[-1]}
    return {"study": "preconditioning on the worked example (Section III-A)", "x_ref": x_ref.tolist(),
            "max_iter": max_iter, "table": table, "wall_s": time.perf_counter() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["schedule", "preconditioning"])
    ap.add_argument("--instances", type=int, default=10)
    ap.add_argument("--max-iter", type=int, default=None)
    args = ap.parse_args()
    if args.study == "schedule":
        print(json.dumps(schedule_study(args.instances, args.max_iter or 6000)), flush=True)
    else:
        print(json.dumps(preconditioning_study(args.max_iter or 200)), flush=True)


if __name__ == "__main__":
    main()
