"""Register and spill budget of the solve kernels, checked at compile time
(no GPU): engine.cu is compiled for sm_103a with ptxas's resource report
into a temporary directory, and every kernel must stay within the register
count its launch bounds allow and spill no more than the known small
amounts below.  The warp-stream SpMV kernels of the PCG loop hold their
next batch of values and columns in registers; what spills is a few words
of live state, about half of it in the rare path that combines the parts
of a row cut between warps (its epilogue works on a local reduction
record), and the checks' compensated FP32 sums and the single-reduction
PCG kernels (four vectors updated per row) need the most.  The FP64
instantiations spill nothing."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_04263_gb300", "csrc")

# kernel name fragment -> largest spill (bytes of stores) allowed
KNOWN_SPILLS = {"k_pcg_kpIfE": 4, "k_pcg_initIfE": 32, "k_check_bIfE": 60, "k_inf_bIfE": 4, "k_spmvIffE": 36,
                "k_sr_kapplyIfE": 48, "k_sr_directionIfE": 104, "k_admm_updateIfE": 8}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


@pytest.fixture(scope="module")
def report():
    with tempfile.TemporaryDirectory() as d:
        cmd = [_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c",
               os.path.join(CSRC, "engine.cu"), "-o", os.path.join(d, "engine.o")]
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    kernels, cur = {}, None
    for line in p.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            kernels[cur] = {}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            kernels[cur]["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            kernels[cur]["regs"] = int(m.group(1))
    assert kernels, p.stderr[-2000:]
    return kernels


def test_every_solve_kernel_was_reported(report):
    names = " ".join(report)
    for k in ["k_pcg_init", "k_pcg_p_t", "k_pcg_kp", "k_pcg_update", "k_admm_update", "k_check_a", "k_check_b",
              "k_check_inf_a", "k_inf_b", "k_rho_apply", "k_output"]:
        assert k in names, k


def test_no_unexpected_spills(report):
    for name, r in report.items():
        allowed = next((v for k, v in KNOWN_SPILLS.items() if k in name), 0)
        assert r.get("spill", 0) <= allowed, (name, r)


def test_register_counts_fit_the_launch_bounds(report):
    """256 threads per CTA and a 65536-register file: the FP32 SpMV
    kernels of the PCG loop are bounded to 4 resident CTAs per SM (64
    registers a thread), the FP32 checks and detection kernels to 3 (80) but
    the check fused with the detection over A to 2 (128), the FP64
    instantiations to 2 (128); nothing may need more than 128."""
    for name, r in report.items():
        regs = r.get("regs", 0)
        assert regs <= 128, (name, r)
        if any(k in name for k in ("k_pcg_p_tIfE", "k_pcg_kpIfE", "k_pcg_initIfE", "k_admm_updateIfE")):
            assert regs <= 64, (name, r)
        if "k_check_inf_a" in name:
            continue
        if any(k in name for k in ("k_check_aIfE", "k_check_bIfE", "k_inf_bIfE")):
            assert regs <= 80, (name, r)
