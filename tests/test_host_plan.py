"""Host logic of the SpMV: the warp-stream plan (rows cut into per-warp
ranges, items, split rows and their slots, bundles of long rows), checked on
600 seeded random row-length profiles by a small C++ harness compiled against
the library's plan code, which replays every warp's walk on the host (nvcc
cross-compiles here; no GPU is used)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_plan_and_partition_invariants(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "plan_harness")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(HERE, "plan_harness.cu"),
                           os.path.join(ROOT, "paper_1912_04263_gb300", "csrc", "plan.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
