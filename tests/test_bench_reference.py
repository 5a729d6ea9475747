"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
keeps the JSON-line contract; run on the small random workload so that it
takes seconds (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "random_100x1000", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0.0
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["n_gpus"] == 1
    for key in ("metric", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert key in line, key
    assert line["config"]["name"] == "random_100x1000" and "random QP" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun with several ranks only rank 0 times the oracle and
    prints; the other ranks exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "random_100x1000", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_solution_errors_against_committed_optima():
    """The bench line's error fields on a solution whose distance to the
    optimum is known: the oracle's own eps = 1e-3 solve of a committed
    workload.  Its objective error against f* is within the convexity bound,
    and the same-eps field reproduces the committed record; for a point moved
    away from it (x and z scaled by 1.5) the residuals and the objective error
    grow, and the bound, being rigorous, still holds."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import qpgen
    from oracle import admm
    ref = bench.golden_optimum("random_100x1000", 3)
    assert ref is not None and ref["own_1e3"] is not None
    qp = qpgen.by_name("random_100x1000", 3)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-3, eps_rel=1e-3))
    e = bench.solution_errors(qp, r.x, r.y, r.z, r.obj, ref)
    assert e["obj_within_bound"] and e["obj_bound"] > 0.0
    assert abs(e["obj_oracle_1e3"] - r.obj) <= 1e-9 * max(1.0, abs(r.obj))
    assert abs(e["obj"] - r.obj) <= 1e-9 * max(1.0, abs(r.obj))
    bad = bench.solution_errors(qp, 1.5 * r.x, r.y, 1.5 * r.z, r.obj, ref)
    # residuals grow with the damage, and the bound still holds (it is rigorous)
    assert bad["r_dual"] > e["r_dual"] and bad["obj_within_bound"]
    assert abs(bad["obj"] - ref["obj"]) > abs(e["obj"] - ref["obj"])
