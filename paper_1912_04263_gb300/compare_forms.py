"""Solve time of the three solver forms on the named workloads: the learned
rho policy in FP32, the residual-ratio rule in FP32 and the plain FP64 form
(ratio rule).  For each form one Solver is set up, solved once to warm up,
then solved `--reps` more times from a cold start; prints one JSON line per
workload and form with the median osqp_solve device time, the iteration
counts and the statuses.

    python -m paper_1912_04263_gb300.compare_forms [--workloads a,b,...] [--reps 3]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import qpgen  # noqa: E402
from paper_1912_04263_gb300 import binding as gb  # noqa: E402

DEFAULT = "random_100x1000,lasso_1000x100000,random_20000x200000,portfolio_100000x1000"
POLICY = os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy", "rho_policy.bin")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default=DEFAULT)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    pol = gb.load_policy(POLICY)
    forms = {"learned_fp32": dict(precision=gb.FP32, rho_policy=gb.RHO_LEARNED, policy_params=pol),
             "ratio_fp32": dict(precision=gb.FP32), "plain_fp64": dict(precision=gb.FP64)}
    for name in args.workloads.split(","):
        qp = qpgen.by_name(name, args.seed)
        for form, kw in forms.items():
            with gb.Solver(qp, **kw) as s:
                s.solve()  # warm-up
                ms, its, sts = [], [], []
                for _ in range(args.reps):
                    sts.append(s.solve())
                    info = s.info()
                    ms.append(info["solve_ms"])
                    its.append(info["iters"])
            print(json.dumps({"workload": name, "seed": args.seed, "form": form,
                              "median_solve_ms": float(np.median(ms)), "iters": its, "status": sts}), flush=True)


if __name__ == "__main__":
    main()
