"""Write tests/golden/full_size_optima.json: the FP64 oracle's optimum of each
benchmark workload (the full-size Lasso, portfolio and random QPs, seed 0,
and the 100 x 1000 random QP, seeds 0-9), against which the GPU solutions of
those workloads are judged (tests/test_gpu_full_size.py, bench.py).

Calls only oracle/ and qpgen/ (the seeded inputs).  For each workload:

* the oracle's direct ADMM (Algorithm 1 with an exact solve of eq. (kkt)) at
  eps_abs = eps_rel = 1e-7: f* and the 1-norms of x* and y* (the convexity
  bound |f - f*| <= max(||y||_1, ||y*||_1) ||r_prim|| + ||r_dual|| ||x - x*||_1
  is then applied with ||x - x*||_1 <= ||x||_1 + ||x*||_1), its residuals and
  iteration count;
* the oracle's own solve at eps = 1e-3 (the tolerance of the benchmark):
  its objective, residuals and iterations, for the same-eps comparison;
* x* in FP32 in full_size_xstar.npz (the bound's ||x - x*||_1 then carries
  at most 2^-24 ||x*||_1 of rounding).

  python tests/golden/make_full_size_optima.py [workload@seed ...]

Each workload takes from minutes (Lasso) to about an hour (the 20000 x
200000 random QP, whose 20000 x 20000 Schur complement is formed and
factored densely) on a few CPU cores.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import qpgen  # noqa: E402
from oracle import admm, checks  # noqa: E402

OUT = os.path.join(HERE, "full_size_optima.json")
XSTAR = os.path.join(HERE, "full_size_xstar.npz")
WORKLOADS = ["random_100x1000@%d" % k for k in range(10)] + ["lasso_1000x100000@0", "portfolio_100000x1000@0",
                                                             "random_20000x200000@0"]
TIGHT = 1e-7


def one(key: str, xstar: dict) -> dict:
    name, seed = key.split("@")
    qp = qpgen.by_name(name, int(seed))
    rec = {"workload": name, "seed": int(seed)}
    for tag, eps in (("eps_1e-3", 1e-3), ("tight", TIGHT)):
        t = time.time()
        r = admm.solve(qp, admm.Settings(eps_abs=eps, eps_rel=eps, max_iter=50000))
        v = checks.kkt_violation(qp, r.x, r.z, r.y)
        rec[tag] = {"eps": eps, "status": r.status, "iters": int(r.iters), "obj": float(r.obj),
                    "r_prim": float(v.prim), "r_dual": float(v.dual), "eps_prim": float(r.res.eps_prim),
                    "eps_dual": float(r.res.eps_dual), "x_norm1": float(np.sum(np.abs(r.x))),
                    "y_norm1": float(np.sum(np.abs(r.y))), "rho_history": [float(p) for p in r.rho_history],
                    "kkt_rel_residual": float(r.kkt_rel_residual), "seconds": round(time.time() - t, 1)}
        print(key, tag, rec[tag], flush=True)
        if tag == "tight":
            xstar[key] = r.x.astype(np.float32)
    return rec


def main(names, out=OUT, xout=XSTAR):
    data, xs = {}, {}
    if os.path.exists(out):
        with open(out) as f:
            data = json.load(f)
    if os.path.exists(xout):
        with np.load(xout) as z:
            xs = {k: z[k] for k in z.files}
    for key in names:
        data[key] = one(key, xs)
        with open(out, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        np.savez(xout, **xs)


if __name__ == "__main__":
    args = sys.argv[1:]
    out, xout = OUT, XSTAR
    if args[:1] == ["--out"]:  # separate files for runs in parallel: --out STEM workload ...
        out, xout, args = args[1] + ".json", args[1] + ".npz", args[2:]
    main(args or WORKLOADS, out, xout)
