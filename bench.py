#!/usr/bin/env python
"""Benchmark of the GPU ADMM QP solver on a synthetic workload shaped like
the paper's Lasso class (D: 100000 x 1000 at 15% density, ~15.1M nonzeros in
A), solved to eps_abs = eps_rel = 1e-3 with FP32 PCG and FP64 reductions.

One step = osqp_setup from device-resident CSR inputs (validation, A' and
[P A'] construction, Ruiz equilibration, preconditioner) + osqp_solve (the
whole ADMM loop as one CUDA graph) + the unscaled solution written to device
buffers.  value = solves per second over all ranks (replicas, one problem
per GPU, seed + rank).

Also reported: the same metric end to end from pinned host buffers through
the C ABI (e2e), the plain FP64 form, ADMM iterations/s, the roofline of the
dominant kernel (CUDA events, algorithmic bytes), SM clocks sampled during
the timed region, and the FP64 CPU oracle timed on the host (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-3 solve & ADMM it/s (learned FP32 vs plain FP64); SpMV GB/s"
WORKLOAD = "lasso_1000x100000"
WORKLOAD_TEXTS = {
    "lasso_1000x100000": ("Lasso QP: D 100000x1000 at 15% density N(0,1), variables (x, y, t), "
                          "n = m = 102000, eps_abs = eps_rel = 1e-3"),
    "portfolio_100000x1000": ("factor-model portfolio QP: F 100000x1000 at 50% density N(0,1), variables (x, y), "
                              "n = 101000, m = 101001, eps_abs = eps_rel = 1e-3"),
    "random_20000x200000": ("random QP: P = M M' + 1e-2 I with M 20000x20000 at 0.05% density, A 200000x20000 at 1% "
                            "density N(0,1), eps_abs = eps_rel = 1e-3"),
    "random_100x1000": ("random QP: P = M M' + 1e-2 I with M 100x100 at 15% density, A 1000x100 at 15% density "
                        "N(0,1), eps_abs = eps_rel = 1e-3"),
}


def workload_text(name: str) -> str:
    return WORKLOAD_TEXTS.get(name, name)


HBM_FALLBACK_GBS = 6800.0
POLICY_PATH = os.path.join(ROOT, "paper_1912_04263_gb300", "policy", "rho_policy.bin")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ------------------------------------------------------------- CPU leg --

def cpu_leg(workload: str, seed: int) -> dict:
    """The FP64 oracle (direct LDL' ADMM, as it stands) on one instance."""
    import qpgen
    from oracle import admm
    qp = qpgen.by_name(workload, seed)
    t = time.perf_counter()
    r = admm.solve(qp)
    dt = time.perf_counter() - t
    return {"seconds": dt, "status": r.status, "iters": r.iters, "obj": r.obj}


def run_cpu_leg(workload: str, seed: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", workload,
                        "--seed", str(seed)], capture_output=True, text=True, env=env, cwd=ROOT)
    if p.returncode != 0:
        raise RuntimeError("cpu leg failed:\n" + p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------- clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None
        self.out = None

    def start(self):
        """Start sampling right before the timed region: every row nvidia-smi
        prints before stop() falls inside it."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.out = open(self.path, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            self.out.close()
            os.unlink(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
            self.proc.wait()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- GPU arm --

def algorithmic_bytes(kernel: str, n: int, m: int, nnz: int, s: int = 4) -> int:
    """Bytes one launch must move at minimum: matrix values and column
    indices once, row pointers once, the gathered vector once, the row
    outputs once, and the extra vectors the kernel's epilogue reads."""
    if kernel == "pcg_kapply":  # rows n of [P A']; gathers [p; t]; writes Kp; reads p
        return nnz * (s + 4) + (n + 1) * 4 + (n + m) * s + n * s + n * s
    if kernel == "pcg_direction":  # rows m of A; gathers yv, pc (n each); writes t (m) and p (n)
        return nnz * (s + 4) + (m + 1) * 4 + 2 * n * s + m * s + n * s
    raise ValueError(kernel)


GOLDEN = os.path.join(ROOT, "tests", "golden", "full_size_optima.json")

# the other measured configurations: (workload, forms, seeds, timed steps)
EXTRA = [("random_100x1000", ["fp64"], list(range(10)), 3),
         ("portfolio_100000x1000", ["learned_fp32", "fp64"], [0], 2),
         ("random_20000x200000", ["learned_fp32", "fp64"], [0], 2)]


def golden_optimum(workload: str, seed: int):
    """The FP64 oracle's record of the workload, as committed in
    tests/golden/full_size_optima.json (written by
    tests/golden/make_full_size_optima.py): its tight solve (f*, ||x*||_1,
    ||y*||_1), its own solve at eps = 1e-3 and x* (FP32) where committed; or
    None."""
    import numpy as np
    key = f"{workload}@{seed}"
    try:
        with open(GOLDEN) as f:
            g = json.load(f)[key]
    except (OSError, KeyError, ValueError):
        return None
    if g["tight"]["status"] != "solved":
        return None
    ref = dict(g["tight"])
    ref["own_1e3"] = g.get("eps_1e-3")
    ref["xstar"] = None
    xpath = os.path.join(os.path.dirname(GOLDEN), "full_size_xstar.npz")
    if os.path.exists(xpath):
        with np.load(xpath) as z:
            if key in z.files:
                ref["xstar"] = z[key].astype(np.float64)
    return ref


def solution_errors(qp, x, y, z, obj, ref) -> dict:
    """Unscaled residuals of the GPU solution, r_prim = ||A x - z||_inf and
    r_dual = ||P x + q + A'y||_inf, and its objective 1/2 x'Px + q'x, in FP64
    on the host from the problem's own data; its objective error against the
    oracle's optimum ref: the relative difference |f - f*| / max(|f*|, 1),
    the convexity bound max(||y||_1, ||y*||_1) r_prim + r_dual ||x - x*||_1
    that |f - f*| must respect (with the committed x* in FP32, whose rounding
    adds 2^-24 ||x*||_1; else ||x||_1 + ||x*||_1 for the last norm), and the
    oracle's own objective at the same eps = 1e-3 (the inf-norm stopping rule
    does not bound the objective error by 1e-3: on problems with many
    inequality rows both solutions may sit far from f*)."""
    import numpy as np
    r_prim = float(np.max(np.abs(qp.A @ x - z), initial=0.0))
    r_dual = float(np.max(np.abs(qp.P @ x + qp.q + qp.A.T @ y), initial=0.0))
    f = float(0.5 * x @ (qp.P @ x) + qp.q @ x)
    out = {"r_prim": r_prim, "r_dual": r_dual, "obj": f, "obj_device": obj}
    if ref is not None:
        fs = ref["obj"]
        out["obj_star"] = fs
        out["obj_rel_err"] = abs(f - fs) / max(abs(fs), 1.0)
        if ref.get("xstar") is not None:
            dx = float(np.sum(np.abs(x - ref["xstar"]))) + 2.0 ** -24 * ref["x_norm1"]
        else:
            dx = float(np.sum(np.abs(x))) + ref["x_norm1"]
        out["obj_bound"] = max(float(np.sum(np.abs(y))), ref["y_norm1"]) * r_prim + r_dual * dx
        out["obj_within_bound"] = bool(abs(f - fs) <= 1.001 * out["obj_bound"] + 1e-9 * max(abs(fs), 1.0))
        own = ref.get("own_1e3")
        if own is not None:
            out["obj_oracle_1e3"] = own["obj"]
            out["obj_oracle_1e3_rel_err"] = abs(own["obj"] - fs) / max(abs(fs), 1.0)
    return out


def gpu_arm(args) -> None:
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import qpgen
    from paper_1912_04263_gb300 import binding as gb
    from paper_1912_04263_gb300 import replicas

    qp = qpgen.by_name(args.workload, replicas.replica_seed(args.seed, rank))
    n, m = qp.n, qp.m
    dev = torch.device("cuda", local)
    P, A = qp.P.tocsr(), qp.A.tocsr()
    import numpy as _np
    lo = _np.where(_np.isinf(qp.l), _np.sign(qp.l) * 1e20, qp.l)
    hi = _np.where(_np.isinf(qp.u), _np.sign(qp.u) * 1e20, qp.u)
    host = {"Prp": _np.ascontiguousarray(P.indptr, _np.int64), "Pcol": _np.ascontiguousarray(P.indices, _np.int32),
            "Pval": _np.ascontiguousarray(P.data, _np.float64), "Arp": _np.ascontiguousarray(A.indptr, _np.int64),
            "Acol": _np.ascontiguousarray(A.indices, _np.int32), "Aval": _np.ascontiguousarray(A.data, _np.float64),
            "q": _np.ascontiguousarray(qp.q), "l": _np.ascontiguousarray(lo), "u": _np.ascontiguousarray(hi)}
    devt = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
    h2d_bytes = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h_bytes = (n + 2 * m) * 8
    xo = torch.empty(n, dtype=torch.float64, device=dev)
    yo = torch.empty(m, dtype=torch.float64, device=dev)
    zo = torch.empty(m, dtype=torch.float64, device=dev)
    # a dedicated stream: the library runs on it and the CUDA events are
    # recorded on it (torch's default stream would be handle 0, which the
    # library treats as "create your own")
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()

    policy = None
    policy_file = args.policy_file or POLICY_PATH
    if os.path.exists(policy_file) and args.policy == "learned":
        policy = gb.load_policy(policy_file)

    def settings(prec):
        s = gb.default_settings(precision=prec, device=local)
        s.cuda_stream = stream.cuda_stream
        if args.loop == "host":
            s.loop_mode = gb.LOOP_HOST
        if prec == gb.FP32 and policy is not None:
            s.rho_policy = gb.RHO_LEARNED
            s.policy_params = policy.ctypes.data
        return s

    def setup_device(prec):
        return gb.osqp_setup_device(devt["Prp"], devt["Pcol"], devt["Pval"], devt["Arp"], devt["Acol"],
                                    devt["Aval"], devt["q"], devt["l"], devt["u"], n, m, settings(prec))

    def step(prec):
        h = setup_device(prec)
        st = gb.osqp_solve(h)
        gb.gbosqp_get_solution_device(h, xo, yo, zo)
        return h, st

    def setup_host(prec):
        s = settings(prec)
        s.P_is_upper = 0
        s.input_location = gb.HOST
        cp = gb.Csr(n, n, int(P.nnz), pinned["Prp"].data_ptr(), pinned["Pcol"].data_ptr(), pinned["Pval"].data_ptr())
        ca = gb.Csr(m, n, int(A.nnz), pinned["Arp"].data_ptr(), pinned["Acol"].data_ptr(), pinned["Aval"].data_ptr())
        h = gb.ctypes.c_void_p()
        rc = gb.lib().osqp_setup(gb.ctypes.byref(h), gb.ctypes.byref(cp), gb.ctypes.byref(ca),
                                 pinned["q"].data_ptr(), pinned["l"].data_ptr(), pinned["u"].data_ptr(),
                                 gb.ctypes.byref(s))
        if rc != gb.OK:
            raise gb.GbosqpError(rc, gb.lib().gbosqp_setup_error().decode())
        return h.value

    xh = np.empty(n)
    yh = np.empty(m)
    zh = np.empty(m)

    def step_e2e(prec):
        h = setup_host(prec)
        st = gb.osqp_solve(h)
        gb.lib().osqp_get_solution(h, xh.ctypes.data, yh.ctypes.data, zh.ctypes.data)
        return h, st

    def barrier():
        if dist:
            dist.barrier()

    def timed(fn, prec, steps):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        hs = []
        e0.record(stream)
        for _ in range(steps):
            hs.append(fn(prec))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        infos = [gb.osqp_get_info(h) for h, _ in hs]
        stats = [st for _, st in hs]
        return ms, infos, stats, [h for h, _ in hs]

    def maxrank(v):
        return replicas.max_over_ranks(v, dist, dev)

    # warm-up
    for _ in range(args.warmup):
        h, _ = step(gb.FP32)
        gb.osqp_cleanup(h)
    if args.lean:  # one untimed-by-events step, for profiler launch lists
        h, st = step(gb.FP32)
        torch.cuda.synchronize()
        info = gb.osqp_get_info(h)
        gb.osqp_cleanup(h)
        if rank == 0:
            print(json.dumps({"lean": True, "status": st, "iters": info["iters"], "pcg_iters": info["pcg_iters"],
                              "setup_launches": info["setup_launches"], "solve_launches": info["solve_launches"]}))
        return
    clock = ClockSampler(local)
    clock.start()
    ms, infos, stats, handles = timed(step, gb.FP32, args.steps)
    clocks = clock.stop()
    ms_step = maxrank(ms) / args.steps
    keep = handles[0]
    for h in handles[1:]:
        gb.osqp_cleanup(h)

    # error of the timed solution against the oracle's optimum (host, FP64)
    xk, yk, zk = np.empty(n), np.empty(m), np.empty(m)
    gb.lib().osqp_get_solution(keep, xk.ctypes.data, yk.ctypes.data, zk.ctypes.data)
    c1_err = solution_errors(qp, xk, yk, zk, gb.osqp_get_info(keep)["obj"], golden_optimum(args.workload, args.seed))

    # roofline of the dominant kernels on a live handle (CUDA events)
    reps = 50
    n_, m_, nnz_a, nnz_pat = gb.dims(keep)
    k_ms = {"pcg_kapply": gb.gbosqp_bench_kernel(keep, gb.K_PCG_KAPPLY, reps),
            "pcg_direction": gb.gbosqp_bench_kernel(keep, gb.K_PCG_DIRECTION, reps),
            "pcg_update": gb.gbosqp_bench_kernel(keep, gb.K_PCG_UPDATE, reps)}
    gbs = {"pcg_kapply": algorithmic_bytes("pcg_kapply", n_, m_, nnz_pat) / (k_ms["pcg_kapply"] * 1e-3) / 1e9,
           "pcg_direction": algorithmic_bytes("pcg_direction", n_, m_, nnz_a) / (k_ms["pcg_direction"] * 1e-3) / 1e9}
    dominant = max(("pcg_kapply", "pcg_direction"), key=lambda k: k_ms[k])
    gb.osqp_cleanup(keep)

    # end to end from pinned host memory
    for _ in range(max(1, args.warmup // 2)):
        h, _ = step_e2e(gb.FP32)
        gb.osqp_cleanup(h)
    e2e_ms, _, e2e_stats, hs = timed(step_e2e, gb.FP32, max(1, args.steps // 2))
    for h in hs:
        gb.osqp_cleanup(h)
    e2e_step = maxrank(e2e_ms) / max(1, args.steps // 2)

    # plain FP64 form
    fp64_ms, fp64_infos, fp64_stats, hs = timed(step, gb.FP64, max(1, args.steps // 2))
    for h in hs:
        gb.osqp_cleanup(h)
    fp64_step = maxrank(fp64_ms) / max(1, args.steps // 2)

    extra = {}
    if args.extra and world == 1:
        for wl, forms, seeds, nsteps in EXTRA:
            extra[wl] = measure_config(gb, torch, np, stream, dev, local, wl, forms, seeds, nsteps, policy, args)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm, peak_kind = peaks()
    med = lambda key, arr: statistics.median([i[key] for i in arr])  # noqa: E731
    iters = med("iters", infos)
    solve_ms = med("solve_ms", infos)
    launches = int(sum(i["setup_launches"] + i["solve_launches"] for i in infos))
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(tpath):
        with open(tpath) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and parts[0] == dominant and parts[1] == args.workload:
                    traffic = float(parts[2])
    out = {
        "metric": METRIC,
        "value": replicas.job_throughput(args.steps, world, ms_step * args.steps / 1000.0),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (f64 reductions)",
        "data": "synthetic",
        "config": {"workload": workload_text(args.workload), "name": args.workload, "seed": args.seed, "n": n, "m": m,
                   "nnz_A": int(A.nnz), "nnz_P": int(P.nnz), "precision": "fp32", "rho_policy": "learned" if policy is not None else "ratio",
                   "step": "osqp_setup(device CSR) + osqp_solve + solution to device",
                   "l2": "no flush: each step streams >240 MB of matrices, above the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "status": sorted(set(int(s) for s in stats)),
        "time_to_1e3_s": ms_step / 1000.0,
        "solve_ms": solve_ms,
        "setup_ms": med("setup_ms", infos),
        "admm_iters": iters,
        "pcg_iters": med("pcg_iters", infos),
        "admm_it_per_s": iters / (solve_ms / 1000.0),
        "spmv_gbs": {k: round(v, 1) for k, v in gbs.items()},
        "kernel_ms": {k: round(v, 5) for k, v in k_ms.items()},
        "plain_fp64": {"rho_policy": "ratio", "time_to_1e3_s": fp64_step / 1000.0, "status": sorted(set(int(s) for s in fp64_stats)),
                       "admm_iters": med("iters", fp64_infos), "pcg_iters": med("pcg_iters", fp64_infos),
                       "solve_ms": med("solve_ms", fp64_infos)},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": round(gbs[dominant], 1), "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(gbs[dominant] / hbm, 4),
                     "traffic": traffic,
                     "algorithmic_bytes": algorithmic_bytes(dominant, n_, m_, nnz_pat if dominant == "pcg_kapply" else nnz_a)},
        "e2e": {"value": replicas.job_throughput(1, world, e2e_step / 1000.0), "unit": "solves/s", "ms_per_step": e2e_step,
                "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes)},
        "clocks": clocks,
        "gpu_launches": launches,
        "oracle_error": c1_err,
        "configs": extra,
    }
    if not args.no_cpu_baseline:
        try:
            c = run_cpu_leg(args.workload, args.seed)
            out["cpu_baseline"] = {"value": 1.0 / c["seconds"], "unit": "solves/s", "cores": 1, "kind": "oracle",
                                   "sample": f"one full FP64 direct-LDL' ADMM solve to 1e-3 of the same instance "
                                             f"(Ruiz, factorization, {c['iters']} iterations), single thread",
                                   "seconds": c["seconds"], "status": c["status"]}
        except Exception as e:  # keep the GPU line
            out["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                   "sample": "failed: " + str(e)[:200]}
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def measure_config(gb, torch, np, stream, dev, local, workload, forms, seeds, nsteps, policy, args) -> dict:
    """One more configuration, each form timed like the headline step (set-up
    from device CSR + solve + solution to device, CUDA events on the library's
    stream) over nsteps steps after one warm-up, per seed; with the solution's
    residuals and objective error against the FP64 oracle's tight optimum
    (committed goldens), and the SpMV kernels' time and GB/s."""
    import qpgen
    rec = {"workload": workload_text(workload), "seeds": seeds, "forms": {}}
    for form in forms:
        prec = gb.FP64 if form == "fp64" else gb.FP32
        rows = []
        for seed in seeds:
            qp = qpgen.by_name(workload, seed)
            n, m = qp.n, qp.m
            P, A = qp.P.tocsr(), qp.A.tocsr()
            lo = np.where(np.isinf(qp.l), np.sign(qp.l) * 1e20, qp.l)
            hi = np.where(np.isinf(qp.u), np.sign(qp.u) * 1e20, qp.u)
            d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in
                 {"Prp": P.indptr.astype(np.int64), "Pcol": P.indices.astype(np.int32), "Pval": P.data,
                  "Arp": A.indptr.astype(np.int64), "Acol": A.indices.astype(np.int32), "Aval": A.data,
                  "q": qp.q, "l": lo, "u": hi}.items()}
            xo = torch.empty(n, dtype=torch.float64, device=dev)
            yo = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
            zo = torch.empty(max(m, 1), dtype=torch.float64, device=dev)

            def step():
                s = gb.default_settings(precision=prec, device=local)
                s.cuda_stream = stream.cuda_stream
                if form == "learned_fp32" and policy is not None:
                    s.rho_policy = gb.RHO_LEARNED
                    s.policy_params = policy.ctypes.data
                h = gb.osqp_setup_device(d["Prp"], d["Pcol"], d["Pval"], d["Arp"], d["Acol"], d["Aval"],
                                         d["q"], d["l"], d["u"], n, m, s)
                st = gb.osqp_solve(h)
                gb.gbosqp_get_solution_device(h, xo, yo, zo)
                return h, st

            h, _ = step()
            gb.osqp_cleanup(h)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            hs = [step() for _ in range(nsteps)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / nsteps
            info = gb.osqp_get_info(hs[0][0])
            row = {"seed": seed, "status": int(hs[0][1]), "time_to_1e3_s": ms / 1000.0,
                   "solve_ms": info["solve_ms"], "setup_ms": info["setup_ms"], "admm_iters": info["iters"],
                   "pcg_iters": info["pcg_iters"], "admm_it_per_s": info["iters"] / max(info["solve_ms"] / 1000.0, 1e-12)}
            if seed == seeds[0]:
                na, npat = gb.dims(hs[0][0])[2:4]
                km = {"pcg_kapply": gb.gbosqp_bench_kernel(hs[0][0], gb.K_PCG_KAPPLY, 20),
                      "pcg_direction": gb.gbosqp_bench_kernel(hs[0][0], gb.K_PCG_DIRECTION, 20)}
                s_ = 8 if prec == gb.FP64 else 4
                row["kernel_ms"] = {k: round(v, 5) for k, v in km.items()}
                row["spmv_gbs"] = {"pcg_kapply": round(algorithmic_bytes("pcg_kapply", n, m, npat, s_) / (km["pcg_kapply"] * 1e-3) / 1e9, 1),
                                   "pcg_direction": round(algorithmic_bytes("pcg_direction", n, m, na, s_) / (km["pcg_direction"] * 1e-3) / 1e9, 1)}
            x, y, z = xo.cpu().numpy(), yo[:m].cpu().numpy(), zo[:m].cpu().numpy()
            row.update(solution_errors(qp, x, y, z, info["obj"], golden_optimum(workload, seed)))
            row["eps_prim"], row["eps_dual"] = info["eps_prim"], info["eps_dual"]
            for hh, _ in hs:
                gb.osqp_cleanup(hh)
            rows.append(row)
            del d
        agg = {k: statistics.median([r[k] for r in rows]) for k in ("time_to_1e3_s", "solve_ms", "admm_iters",
                                                                      "pcg_iters", "admm_it_per_s")}
        errs = [r["obj_rel_err"] for r in rows if "obj_rel_err" in r]
        agg["max_obj_rel_err"] = max(errs) if errs else None
        agg["all_within_bound"] = all(r.get("obj_within_bound", True) for r in rows) if errs else None
        own = [r["obj_oracle_1e3_rel_err"] for r in rows if "obj_oracle_1e3_rel_err" in r]
        agg["max_oracle_1e3_obj_rel_err"] = max(own) if own else None
        agg["all_solved"] = all(r["status"] == 1 for r in rows)
        rec["forms"][form] = {"median": agg, "runs": rows}
    return rec


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c = run_cpu_leg(args.workload, args.seed)
    v = 1.0 / c["seconds"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": 1, "warmup": 0,
        "ms_per_step": c["seconds"] * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_text(args.workload), "name": args.workload, "seed": args.seed,
                   "step": "one full FP64 oracle solve (direct LDL' ADMM); one timed step regardless of --steps "
                           "because one solve of the Lasso workload takes about half a minute on one core"},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "one full solve of the same instance, single thread"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "status": c["status"], "iters": c["iters"],
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-leg", action="store_true")
    ap.add_argument("--lean", action="store_true", help="warm-up steps then one step, minimal output (profiling)")
    ap.add_argument("--policy", default="learned", choices=["learned", "ratio"],
                    help="rho rule of the FP32 form (learned: the committed trained policy, if present)")
    ap.add_argument("--policy-file", default=None, help="policy weights to use instead of the committed ones")
    ap.add_argument("--extra", type=int, default=1,
                    help="1: also time the other configurations (random 100x1000 FP64 over 10 seeds, portfolio "
                         "100000x1000 and random 20000x200000 learned FP32 vs plain FP64) and report each "
                         "solution's error against the oracle")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="host: the same kernels driven by a host loop (profilers cannot attribute kernel "
                         "nodes inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.cpu_leg:
        print(json.dumps(cpu_leg(args.workload, args.seed)))
        return
    if args.warmup < 3 and args.impl == "ours" and not args.lean:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
