"""Held-out evaluation of the learned rho policy on the learned-policy
workload as specified: 200 random QPs with n = 5000 and m = 50000 (P = M M'
+ 1e-2 I, M and A at 15% density), seeds 200000-200199, disjoint from the
training seeds (100000 and up).

Every problem is solved to eps_abs = eps_rel = 1e-3 with the residual-ratio
rule and with the learned policy (both FP32 PCG with FP64 reductions); every
fourth also with the plain FP64 form (ratio rule).  The problems are
generated by a pool of CPU processes (started before the first GPU call,
with the spawn method) while the GPU solves, one problem at a time, so that
the solve times are not disturbed.  Writes a JSON table (per-problem rows and
a summary: solve time, ADMM iterations, PCG steps, fraction solved, learned
versus ratio rule, learned FP32 versus plain FP64).

    python -m paper_1912_04263_gb300.policy_eval [--count 200] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEED0 = 200000
N, M = 5000, 50000


def generate(seed: int):
    """The held-out problem of this seed as plain arrays (worker process)."""
    import qpgen
    qp = qpgen.random_qp(N, M, seed)
    P, A = qp.P.tocsr(), qp.A.tocsr()
    return seed, (P.indptr, P.indices, P.data, A.indptr, A.indices, A.data, qp.q, qp.l, qp.u)


def solve_forms(gb, arrays, params, with_fp64: bool) -> dict:
    import numpy as np
    import scipy.sparse as sp
    import qpgen
    Pi, Pj, Pv, Ai, Aj, Av, q, l, u = arrays
    qp = qpgen.QP(sp.csr_matrix((Pv, Pj, Pi), shape=(N, N)), q, sp.csr_matrix((Av, Aj, Ai), shape=(M, N)), l, u)
    forms = [("ratio_fp32", dict(precision=gb.FP32)),
             ("learned_fp32", dict(precision=gb.FP32, rho_policy=gb.RHO_LEARNED, policy_params=params))]
    if with_fp64:
        forms.append(("ratio_fp64", dict(precision=gb.FP64)))
    row = {}
    for tag, kw in forms:
        with gb.Solver(qp, **kw) as s:
            st = s.solve()
            info = s.info()
            x, y, z = s.solution()
        # optimality conditions of the solution on the unscaled data (FP64, host)
        r_prim = float(np.max(np.abs(qp.A @ x - z)))
        r_dual = float(np.max(np.abs(qp.P @ x + qp.q + qp.A.T @ y)))
        row[tag] = {"status": st, "iters": info["iters"], "pcg_iters": info["pcg_iters"],
                    "solve_ms": info["solve_ms"], "obj": info["obj"], "r_prim": r_prim, "r_dual": r_dual,
                    "eps_prim": info["eps_prim"], "eps_dual": info["eps_dual"],
                    "fallbacks": info["policy_fallbacks"], "rho_updates": info["rho_updates"]}
    return row


def summarize(rows) -> dict:
    import numpy as np
    out = {}
    for tag in ("ratio_fp32", "learned_fp32", "ratio_fp64"):
        sel = [r[tag] for r in rows if tag in r]
        if not sel:
            continue
        out[tag] = {"problems": len(sel), "solved": int(sum(v["status"] == 1 for v in sel)),
                    "median_solve_ms": float(np.median([v["solve_ms"] for v in sel])),
                    "total_solve_ms": float(np.sum([v["solve_ms"] for v in sel])),
                    "median_iters": float(np.median([v["iters"] for v in sel])),
                    "median_pcg_iters": float(np.median([v["pcg_iters"] for v in sel]))}
    lr = [r["learned_fp32"]["solve_ms"] / r["ratio_fp32"]["solve_ms"] for r in rows]
    out["learned_vs_ratio_time_total"] = out["learned_fp32"]["total_solve_ms"] / out["ratio_fp32"]["total_solve_ms"]
    out["learned_vs_ratio_time_geomean"] = float(np.exp(np.mean(np.log(lr))))
    out["learned_faster_on"] = int(sum(v < 1.0 for v in lr))
    li = [r["learned_fp32"]["iters"] / r["ratio_fp32"]["iters"] for r in rows]
    out["learned_vs_ratio_iters_geomean"] = float(np.exp(np.mean(np.log(li))))
    sub = [r for r in rows if "ratio_fp64" in r]
    if sub:
        out["learned_fp32_vs_fp64_time_total"] = (sum(r["learned_fp32"]["solve_ms"] for r in sub) /
                                                  sum(r["ratio_fp64"]["solve_ms"] for r in sub))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=200)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy",
                                                  "eval_random_5000x50000.json"))
    ap.add_argument("--workers", type=int, default=max(1, min(15, (os.cpu_count() or 2) - 1)))
    ap.add_argument("--window", type=int, default=6, help="problems generated ahead of the GPU")
    args = ap.parse_args()
    t0 = time.time()
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(args.workers)  # before any GPU call
    from paper_1912_04263_gb300 import binding as gb
    params = gb.load_policy(os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy", "rho_policy.bin"))
    seeds = [SEED0 + i for i in range(args.count)]
    pending = [pool.apply_async(generate, (sd,)) for sd in seeds[:args.window]]
    nxt = args.window
    rows = []
    for i in range(len(seeds)):
        seed, arrays = pending.pop(0).get()
        if nxt < len(seeds):
            pending.append(pool.apply_async(generate, (seeds[nxt],)))
            nxt += 1
        row = {"seed": seed}
        row.update(solve_forms(gb, arrays, params, with_fp64=(i % 4 == 0)))
        rows.append(row)
        del arrays
        print(json.dumps({"seed": seed, "ratio_ms": round(row["ratio_fp32"]["solve_ms"], 2),
                          "learned_ms": round(row["learned_fp32"]["solve_ms"], 2),
                          "iters": [row["ratio_fp32"]["iters"], row["learned_fp32"]["iters"]]}), flush=True)
    pool.close()
    out = {"workload": f"random QP n = {N}, m = {M}, P = M M' + 1e-2 I, M and A at 15% density N(0,1), "
                       f"q ~ N(0,1), l = -U[0,1], u = U[0,1], eps_abs = eps_rel = 1e-3",
           "seeds": [seeds[0], seeds[-1]], "policy": "policy/rho_policy.bin", "summary": summarize(rows),
           "rows": rows, "seconds": round(time.time() - t0, 1)}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["summary"], indent=1))


if __name__ == "__main__":
    main()
