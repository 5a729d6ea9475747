"""The C-ABI library loads and exports every entry point declared in
include/gbosqp.h; host-only calls behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import qpgen
from oracle import checks, admm
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "gbosqp.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ["osqp_setup", "osqp_solve", "osqp_update_rho", "osqp_get_solution", "osqp_get_info",
                 "osqp_cleanup", "gbosqp_default_settings", "gbosqp_last_error"]:
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_settings_match_the_paper(lib):
    from paper_1912_04263_gb300 import binding as gb
    s = gb.default_settings()
    # Section 3.4 defaults, Table 1 cadence, Section 5.3.4 tolerance rule
    assert s.alpha == 1.6 and s.sigma == 1e-6
    assert s.check_every == 5 and s.rho_every == 10
    assert s.pcg_lambda == 0.15 and s.pcg_eps_min == 1e-7
    assert s.rho0 == 0.1 and s.eps_abs == 1e-3 and s.eps_rel == 1e-3
    # infeasibility tolerances of reading S17; the paper's R = rho I; cold starts
    assert s.eps_prim_inf == 1e-4 and s.eps_dual_inf == 1e-4
    assert s.rho_vector == 0 and s.warm_start == 0


def test_settings_struct_layout_matches_the_header(lib):
    """The ctypes mirror of gbosqp_settings has the header's field order (so
    the binding and the C struct agree byte for byte)."""
    from paper_1912_04263_gb300 import binding as gb
    with open(os.path.join(ROOT, "include", "gbosqp.h")) as f:
        text = f.read()
    body = text[text.index("typedef struct {\n    double alpha;"):]
    body = body[:body.index("} gbosqp_settings;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(?:double|int32_t|void\s*\*|const float\s*\*)\s*\**\s*(\w+)\s*;", body)
    assert [f for f, _ in gb.Settings._fields_] == fields


def test_error_strings_and_null_arguments(lib):
    from paper_1912_04263_gb300 import binding as gb
    assert gb.error_string(gb.SOLVED) == "solved"
    assert gb.error_string(gb.ERR_CSR) == "invalid CSR matrix"
    assert lib.osqp_solve(None) == gb.ERR_INVALID_ARG
    assert lib.gbosqp_default_settings(None) == gb.ERR_INVALID_ARG
    lib.osqp_cleanup(None)
    h = ctypes.c_void_p()
    assert lib.osqp_setup(ctypes.byref(h), None, None, None, None, None, None) == gb.ERR_INVALID_ARG


def test_settings_validation_is_host_side(lib):
    from paper_1912_04263_gb300 import binding as gb
    qp = qpgen.random_qp(5, 7, 0)
    for bad in [dict(alpha=2.0), dict(sigma=0.0), dict(check_every=0), dict(rho_every=7),
                dict(precision=5), dict(rho_policy=gb.RHO_LEARNED), dict(eps_prim_inf=-1e-4),
                dict(eps_dual_inf=float("nan")), dict(eps_dual_inf=float("inf")), dict(warm_start=2),
                dict(rho_vector=-1), dict(rho_min=0.0)]:
        with pytest.raises(gb.GbosqpError) as e:
            gb.Solver(qp, **bad)
        assert e.value.code == gb.ERR_INVALID_ARG, bad


def test_objective_error_bound_holds_on_loose_iterates():
    """The bound used by the GPU parity tests holds for oracle iterates at a
    loose tolerance (exact optimum from brute force)."""
    checked = 0
    for seed in range(8):
        qp = qpgen.tiny_qp(4, 6, seed, n_eq=1, n_inf=1)
        try:
            xs, ys = checks.brute_force(qp)
        except RuntimeError:  # an infeasible draw
            continue
        checked += 1
        fs = admm.objective(qp.P, qp.q, xs)
        r = admm.solve(qp, admm.Settings(eps_abs=1e-2, eps_rel=1e-2, check_every=1))
        v = checks.kkt_violation(qp, r.x, r.z, r.y)
        bound = checks.objective_error_bound(r.x, r.y, v.prim, v.dual, xs, ys)
        assert abs(r.obj - fs) <= bound * (1 + 1e-9) + 1e-12
    assert checked >= 3


def test_binding_constants_match_the_header():
    """Every #define of include/gbosqp.h that the binding mirrors has the same
    value there (error codes, statuses, enumerations, sizes, kernel
    selectors)."""
    from paper_1912_04263_gb300 import binding as gb
    with open(os.path.join(ROOT, "include", "gbosqp.h")) as f:
        text = f.read()
    defs = {}
    for name, val in re.findall(r"^#define\s+GBOSQP_(\w+)\s+\(?(-?[0-9.e]+)\)?", text, flags=re.M):
        defs[name] = float(val) if ("." in val or "e" in val) else int(val)
    pairs = {"OK": gb.OK, "ERR_INVALID_ARG": gb.ERR_INVALID_ARG, "ERR_DIMENSION": gb.ERR_DIMENSION,
             "ERR_CSR": gb.ERR_CSR, "ERR_BOUNDS": gb.ERR_BOUNDS, "ERR_NONFINITE": gb.ERR_NONFINITE,
             "ERR_CUDA": gb.ERR_CUDA, "ERR_OOM": gb.ERR_OOM, "ERR_DEVICE_TIMEOUT": gb.ERR_DEVICE_TIMEOUT,
             "ERR_UNSUPPORTED": gb.ERR_UNSUPPORTED, "ERR_POLICY": gb.ERR_POLICY,
             "SOLVED": gb.SOLVED, "MAX_ITER": gb.MAX_ITER, "NONFINITE": gb.NONFINITE,
             "PRIMAL_INFEASIBLE": gb.PRIMAL_INFEASIBLE, "DUAL_INFEASIBLE": gb.DUAL_INFEASIBLE,
             "FP32": gb.FP32, "FP64": gb.FP64, "RHO_RATIO": gb.RHO_RATIO, "RHO_LEARNED": gb.RHO_LEARNED,
             "RHO_FIXED": gb.RHO_FIXED, "HOST": gb.HOST, "DEVICE": gb.DEVICE, "LOOP_GRAPH": gb.LOOP_GRAPH,
             "LOOP_HOST": gb.LOOP_HOST, "MAT_A": gb.MAT_A, "MAT_PAT": gb.MAT_PAT,
             "CHECK_FIELDS": gb.CHECK_FIELDS, "POLICY_PARAMS": gb.POLICY_PARAMS, "INFINITY": gb.INFINITY,
             "K_PCG_DIRECTION": gb.K_PCG_DIRECTION, "K_PCG_KAPPLY": gb.K_PCG_KAPPLY, "K_PCG_UPDATE": gb.K_PCG_UPDATE,
             "K_PCG_INIT": gb.K_PCG_INIT, "K_ADMM_UPDATE": gb.K_ADMM_UPDATE, "K_CHECK_A": gb.K_CHECK_A,
             "K_CHECK_B": gb.K_CHECK_B, "K_INF_A": gb.K_INF_A, "K_INF_B": gb.K_INF_B,
             "K_PCG_SR_DIRECTION": gb.K_PCG_SR_DIRECTION, "K_PCG_SR_KAPPLY": gb.K_PCG_SR_KAPPLY,
             "PCG_CLASSIC": gb.PCG_CLASSIC, "PCG_SINGLE_REDUCTION": gb.PCG_SINGLE_REDUCTION}
    for name, value in pairs.items():
        assert name in defs, name
        assert defs[name] == value, (name, defs[name], value)
    assert len(gb.CHECK_NAMES) <= gb.CHECK_FIELDS


@pytest.mark.parametrize("struct,cls", [("gbosqp_info", "Info"), ("gbosqp_csr", "Csr")])
def test_info_and_csr_struct_layouts_match_the_header(struct, cls):
    """Field names in declaration order (several per line allowed) equal the
    ctypes mirror's, and the mirror's types have the header's widths."""
    from paper_1912_04263_gb300 import binding as gb
    with open(os.path.join(ROOT, "include", "gbosqp.h")) as f:
        text = f.read()
    body = text[:text.index("} " + struct + ";")]
    body = body[body.rindex("typedef struct {"):]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    widths = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    decl = re.findall(r"(?:const\s+)?(int32_t|int64_t|double)\s*([\w\s,*]+);", body)
    expect_types = []
    for typ, names in decl:
        for nm in names.split(","):
            nm = nm.strip()
            fields.append(nm.lstrip("*").strip())
            expect_types.append(ctypes.c_void_p if nm.startswith("*") else widths[typ])
    mirror = getattr(gb, cls)._fields_
    assert [f for f, _ in mirror] == fields
    for (f, t), e in zip(mirror, expect_types):
        assert ctypes.sizeof(t) == ctypes.sizeof(e), f
