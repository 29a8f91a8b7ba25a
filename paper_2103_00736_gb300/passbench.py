"""Per-phase device times of the persistent kernel on one instance, and the
device's random-gather rates (benchmark; prints one JSON object).

    python -m paper_2103_00736_gb300.passbench [--workload large_lp|socp] [--reps 50]
        [--widths 0,24576,12288] [--smem-sweep]

For every column-block width given (0 = the default, -1 = the L2-gather
layout) a problem is created on the instance and every phase kind that the
layout has is timed with acs_bench_passes (each repetition ends with a grid
barrier; the barrier alone is kind "barrier").  --smem-sweep also times the
L2-gather passes with more dynamic shared memory requested (a smaller L1).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_00736_gb300 import capi, instances as I  # noqa: E402

SCHED = {"large_lp": dict(cond_first=300, cond_period=100, t=9.2),
         "socp": dict(cond_first=200, cond_period=100, t=1.7)}
CB_KINDS = ("cb_At", "cb_tcomb", "cb_A", "cb_vec", "o32_rhs", "o32_rhs_comb", "o32_upd", "o32_upd_comb",
            "cb_stage32", "cb_stage64")
L2_KINDS = ("l2_At", "l2_A", "l2_vec")
COMMON = ("fp64_rhs", "fp64_At", "barrier", "abs_K", "kkt")
DIAG = ("cb_At_nogather", "cb_At_nostage", "stream_At", "stream_At_val")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large_lp", choices=sorted(SCHED))
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--widths", default="-1,0")
    ap.add_argument("--smem-sweep", action="store_true")
    ap.add_argument("--gather", action="store_true")
    ap.add_argument("--kinds", default="", help="comma-separated phase kinds (default: all the layout has)")
    args = ap.parse_args()
    out = {"workload": args.workload}
    t0 = time.perf_counter()
    inst = I.large_lp() if args.workload == "large_lp" else I.socp()
    out["generate_s"] = time.perf_counter() - t0
    out["m"], out["n"], out["nnz"] = inst.m, inst.n, inst.nnz
    for w in (int(v) for v in args.widths.split(",")):
        s = capi.Solver(inst, col_block=w, **SCHED[args.workload])
        try:
            # a short solve first: realistic iterate values and warm caches
            s.solve(tol=0.0, max_iter=3)
            lay = capi.acs_debug_layout(s.h)
            kinds = (CB_KINDS if lay["col_blocked"] else L2_KINDS) + COMMON
            if args.kinds:
                kinds = tuple(k for k in args.kinds.split(",") if k in kinds + (DIAG if lay["col_blocked"] else ()))
            res = {k: capi.acs_bench_passes(s.h, k, args.reps) for k in kinds}
            if args.smem_sweep and lay["col_blocked"]:
                for sm in (0, 196608):
                    for k in ("cb_At_nogather", "stream_At", "stream_At_val"):
                        res[f"{k}@smem{sm}"] = capi.acs_bench_passes(s.h, k, args.reps, sm)
            if args.smem_sweep and not lay["col_blocked"]:
                for sm in (65536, 98304, 131072, 163840, 196608):
                    for k in L2_KINDS + COMMON:
                        res[f"{k}@smem{sm}"] = capi.acs_bench_passes(s.h, k, args.reps, sm)
            out[f"width{w}"] = {"layout": lay, "us": res}
        finally:
            s.close()
    if args.gather:
        g = {}
        for mode, name in ((0, "default"), (1, "cg"), (2, "nc")):
            g[f"l2_{name}_4MB"] = capi.acs_bench_gather(1 << 20, mode)
            g[f"l2_{name}_800KB"] = capi.acs_bench_gather(1 << 18, mode)
        g["smem_128KB"] = capi.acs_bench_gather(1 << 15, 3)
        out["gathers_per_s"] = g
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
