"""Train the learned rho / PCG-tolerance policy on trajectories the solver
generates itself, on the GPU, and evaluate it on held-out QPs.

The policy is not part of the paper.  Training problems mix the random,
Lasso and portfolio families (seeds disjoint from every evaluation seed).
Labels come from rollouts at every rho
decision (every 10 ADMM iterations): from the current state each candidate
(rho, lambda) pair, rho being the residual-ratio rule's proposal times a
multiplier, is held for 10 iterations, after which the ratio rule decides
until the solve ends (one CUDA-graph solve per rollout); the label is the
candidate with the least remaining work, PCG steps + 2 x ADMM iterations
(one step of policy improvement over the ratio rule).  The trajectory then
continues with the chosen candidate.
Features: log ||r_prim||, log ||r_dual|| (scaled problem), log rho,
log(1 + PCG steps in the last 10 iterations).  Targets: the chosen log
multiplier of the ratio rule's rho (0: follow the rule) and
log(lambda / 0.15).

Training runs on the device through the library's BF16 kernels (Adam, FP32
master weights); the weights are written with binding.save_policy.  The
held-out evaluation solves each problem with the ratio rule and with the
learned policy (FP32) and with the plain FP64 ratio-rule form, and writes a
JSON summary.

    python -m paper_1912_04263_gb300.policy_train --out DIR [--train N] [--eval N]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import qpgen  # noqa: E402
from paper_1912_04263_gb300 import binding as gb  # noqa: E402

# candidates, the ratio rule's own choice first so that ties keep it
LOG_MULTS = [0.0, -math.log(3.0), math.log(3.0), -math.log(10.0), math.log(10.0)]
LAMBDAS = [0.15, 0.05, 0.5]
LAMBDA0 = 0.15
EPS_MIN = 1e-7
TRAIN_SEED0 = 100000
EVAL_SEED0 = 200000


def features(c: dict, rho: float, pcg_steps: int) -> list:
    return [math.log(max(c["r_prim_s"], 1e-30)), math.log(max(c["r_dual_s"], 1e-30)), math.log(rho),
            math.log1p(pcg_steps)]


def pcg_eps(c: dict, lam: float) -> float:
    return max(lam * math.sqrt(max(c["r_prim_s"], 0.0) * max(c["r_dual_s"], 0.0)), EPS_MIN)


def trajectory(qp, max_decisions: int = 40, rollout_iters: int = 2000):
    """Decision points of one FP32 solve, each labelled by rollouts: from the
    current state, every candidate (rho, lambda) is held for the next 10
    iterations and the ratio rule decides after that, until the solve ends;
    the label is the candidate with the least remaining work (PCG steps + 2 x
    iterations), ties to the ratio rule's own choice.  The trajectory then
    continues with the chosen candidate."""
    s = gb.Solver(qp, precision=gb.FP32, loop_mode=gb.LOOP_HOST, rho_policy=gb.RHO_FIXED)
    ro = gb.Solver(qp, precision=gb.FP32, rho_policy=gb.RHO_RATIO, max_iter=rollout_iters)
    h, hr = s.h, ro.h
    n, m = s.n, s.m
    rho = 0.1
    gb.gbosqp_set_iterates(h, np.zeros(n), np.zeros(m), np.zeros(m), np.zeros(n), rho)
    st, per = gb.gbosqp_admm_iterations(h, 10)
    samples = []
    for _ in range(max_decisions):
        if st != 0:
            break
        c0 = gb.gbosqp_check(h)
        f = features(c0, rho, int(per.sum()))
        rho_r = c0["rho_ratio"]
        x, z, y, xt, _ = gb.gbosqp_get_iterates(h)
        best = None
        for lm in LOG_MULTS:
            for lc in LAMBDAS:
                r = min(max(rho_r * math.exp(lm), 1e-6), 1e6)
                gb.gbosqp_set_iterates(hr, x, z, y, xt, r)
                gb.gbosqp_set_pcg_lambda(hr, lc, pcg_eps(c0, lc))
                gb.gbosqp_resume(hr)
                st_r = gb.osqp_solve(hr)
                info = gb.osqp_get_info(hr)
                work = float(info["pcg_iters"] + 2 * info["iters"]) if st_r == gb.SOLVED else math.inf
                if best is None or work < best[0]:
                    best = (work, lm, lc, r)
        _, lm, lc, r = best
        samples.append(f + [lm, math.log(lc / LAMBDA0)])
        rho = r
        gb.gbosqp_set_iterates(h, x, z, y, xt, rho)
        gb.gbosqp_set_pcg_lambda(h, lc, pcg_eps(c0, lc))
        st, per = gb.gbosqp_admm_iterations(h, 10)
    s.close()
    ro.close()
    return samples


def init_params(feats: np.ndarray, seed: int) -> np.ndarray:
    """He-initialised weights (seeded on the host), zero biases, feature
    standardisation from the training set, clamp log 10, lambda in
    [0.05, 0.5], lambda output on."""
    rng = np.random.default_rng(seed)
    p = np.zeros(gb.POLICY_PARAMS, np.float32)
    p[0:4] = feats.mean(axis=0)
    p[4:8] = np.maximum(feats.std(axis=0), 1e-3)
    off = 8
    for rows, cols in [(64, 4), (64, 0), (64, 64), (64, 0), (2, 64), (2, 0)]:
        if cols:
            p[off:off + rows * cols] = rng.standard_normal(rows * cols) * math.sqrt(2.0 / cols)
            off += rows * cols
        else:
            off += rows
    p[off:off + 4] = [math.log(10.0), 0.05, 0.5, 1.0]
    return p


def train(samples: np.ndarray, steps: int = 4000, batch: int = 256, lr: float = 1e-3, seed: int = 7):
    feats = samples[:, :4].astype(np.float32)
    tgt = samples[:, 4:6].astype(np.float32)
    wgt = np.ones_like(tgt)
    p0 = init_params(feats, seed)
    rng = np.random.default_rng(seed + 1)
    batches = rng.integers(0, len(feats), size=(steps, batch)).astype(np.int32)
    p, hist = gb.gbosqp_mlp_train(p0, feats, tgt, wgt, batches, lr)
    return p, hist


def evaluate(params, problems) -> list:
    rows = []
    for name, qp in problems:
        row = {"problem": name}
        for tag, kw in [("ratio_fp32", dict(precision=gb.FP32)),
                        ("learned_fp32", dict(precision=gb.FP32, rho_policy=gb.RHO_LEARNED, policy_params=params)),
                        ("ratio_fp64", dict(precision=gb.FP64))]:
            with gb.Solver(qp, **kw) as s:
                s.solve()  # warm-up (graph instantiation, caches)
                t = time.perf_counter()
                st = s.solve()
                wall = time.perf_counter() - t
                info = s.info()
            row[tag] = {"status": st, "iters": info["iters"], "pcg_iters": info["pcg_iters"],
                        "solve_ms": info["solve_ms"], "wall_ms": wall * 1e3, "obj": info["obj"],
                        "fallbacks": info["policy_fallbacks"], "rho_updates": info["rho_updates"]}
        rows.append(row)
    return rows


def summarize(rows) -> dict:
    out = {}
    for tag in ("ratio_fp32", "learned_fp32", "ratio_fp64"):
        ms = [r[tag]["solve_ms"] for r in rows]
        it = [r[tag]["iters"] for r in rows]
        out[tag] = {"median_solve_ms": float(np.median(ms)), "total_solve_ms": float(np.sum(ms)),
                    "median_iters": float(np.median(it)),
                    "solved": int(sum(r[tag]["status"] == gb.SOLVED for r in rows))}
    out["learned_vs_ratio_time"] = out["learned_fp32"]["total_solve_ms"] / out["ratio_fp32"]["total_solve_ms"]
    out["learned_fp32_vs_fp64_time"] = out["learned_fp32"]["total_solve_ms"] / out["ratio_fp64"]["total_solve_ms"]
    return out


def training_problem(i: int, rng):
    """Training problem i: a random QP, a Lasso QP or a portfolio QP (in
    proportions 2 : 1 : 1), sizes drawn from rng, seed TRAIN_SEED0 + i."""
    seed = TRAIN_SEED0 + i
    kind = ("random", "random", "lasso", "portfolio")[i % 4]
    if kind == "random":
        n = int(rng.integers(500, 2501))
        return f"random_{n}", qpgen.random_qp(n, 10 * n, seed)
    if kind == "lasso":
        f = int(rng.integers(50, 401))
        return f"lasso_{f}x{20 * f}", qpgen.lasso_qp(f, 20 * f, seed)
    na = int(rng.integers(2000, 10001))
    k = int(rng.integers(20, 101))
    return f"portfolio_{na}x{k}", qpgen.portfolio_qp(na, k, seed)


def eval_problems(args):
    out = [(f"random_{args.eval_n}_s{EVAL_SEED0 + i}", qpgen.random_qp(args.eval_n, 10 * args.eval_n, EVAL_SEED0 + i))
           for i in range(args.eval)]
    out += [(f"random_5000_s{EVAL_SEED0 + 1000 + i}", qpgen.random_qp(5000, 50000, EVAL_SEED0 + 1000 + i))
            for i in range(args.eval_large)]
    out += [(f"lasso_300x6000_s{EVAL_SEED0 + 2000 + i}", qpgen.lasso_qp(300, 6000, EVAL_SEED0 + 2000 + i))
            for i in range(args.eval_family)]
    out += [(f"portfolio_8000x80_s{EVAL_SEED0 + 3000 + i}", qpgen.portfolio_qp(8000, 80, EVAL_SEED0 + 3000 + i))
            for i in range(args.eval_family)]
    if args.eval_full:
        out += [("lasso_1000x100000_s0", qpgen.lasso_qp(1000, 100000, 0)),
                ("portfolio_100000x1000_s0", qpgen.portfolio_qp(100000, 1000, 0)),
                ("random_20000x200000_s0", qpgen.random_qp(20000, 200000, 0, p_density=5e-4, a_density=0.01))]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "policy"))
    ap.add_argument("--train", type=int, default=400, help="training trajectories")
    ap.add_argument("--eval", type=int, default=24, help="held-out problems at n = --eval-n")
    ap.add_argument("--eval-n", type=int, default=3000)
    ap.add_argument("--eval-large", type=int, default=4, help="held-out problems at n = 5000")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--eval-family", type=int, default=6, help="held-out Lasso and portfolio problems each")
    ap.add_argument("--eval-full", action="store_true", help="also the full-size Lasso, portfolio, random QPs")
    ap.add_argument("--max-seconds", type=float, default=1e9, help="stop generating trajectories after this time")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    t0 = time.time()
    rng = np.random.default_rng(12345)
    samples = []
    done = 0
    for i in range(args.train):
        if time.time() - t0 > args.max_seconds:
            print(f"time budget reached after {i} trajectories", flush=True)
            break
        done += 1
        name, qp = training_problem(i, rng)
        samples.extend(trajectory(qp))
        if i % 20 == 0:
            print(f"trajectory {i}/{args.train} {name} samples={len(samples)} t={time.time() - t0:.0f}s", flush=True)
    S = np.array(samples, np.float64)
    np.save(os.path.join(args.out, "samples.npy"), S)
    p, hist = train(S, steps=args.steps)
    path = os.path.join(args.out, "rho_policy.bin")
    gb.save_policy(path, p)
    print(f"trained on {len(S)} samples: loss {hist[:50].mean():.4f} -> {hist[-50:].mean():.4f}", flush=True)
    rows = evaluate(p, eval_problems(args))
    summary = summarize(rows)
    for fam in ("random", "lasso", "portfolio"):
        sub = [r for r in rows if r["problem"].startswith(fam)]
        if sub:
            summary["family_" + fam] = summarize(sub)
    report = {"train_trajectories": int(done),
              "train_families": "random n in [500, 2500] (half), Lasso f in [50, 400] x 20f, portfolio "
                                "[2000, 10000] assets x [20, 100] factors",
              "samples": int(len(S)), "train_steps": int(args.steps), "batch": 256,
              "loss_first": float(hist[:50].mean()), "loss_last": float(hist[-50:].mean()),
              "label_mult_hist": np.histogram(S[:, 4], bins=[-3, -1.7, -0.5, 0.5, 1.7, 3])[0].tolist(),
              "label_mult_hist_bins": "rho multiplier x1/10, x1/3, x1, x3, x10",
              "summary": summary, "rows": rows, "seconds": time.time() - t0}
    with open(os.path.join(args.out, "eval.json"), "w") as fh:
        json.dump(report, fh, indent=1)
    print(json.dumps({"summary": summary, "samples": len(S)}), flush=True)


if __name__ == "__main__":
    main()
