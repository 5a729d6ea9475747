"""Infeasibility detection on the GPU (Section 3.1) against the oracle:
the status of every problem equals the oracle's, and the certificate the
solver returns satisfies eq. (prim_infeas) or eq. (dual_infeas) in the
tested approximate form (unit inf-norm, checked in FP64 on the host)."""
import math

import numpy as np
import pytest

import qpgen
from oracle import admm

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_1912_04263_gb300.binding")

STATUS = {"solved": 1, "max_iter": 2, "primal_infeasible": 4, "dual_infeasible": 5}


def primal_cases():
    return [qpgen.infeasible_primal_qp()] + [qpgen.random_primal_infeasible_qp(20, 40, s) for s in range(4)] + \
        [qpgen.random_primal_infeasible_qp(400, 3000, 11, density=0.05)]


def dual_cases():
    return [qpgen.infeasible_dual_qp()] + [qpgen.random_dual_infeasible_qp(24, 30, 4, s) for s in range(4)] + \
        [qpgen.random_dual_infeasible_qp(500, 2000, 40, 12, density=0.02)]


def check_primal_certificate(qp, y, tol):
    assert np.max(np.abs(y)) == pytest.approx(1.0, rel=1e-12)
    assert np.max(np.abs(qp.A.T @ y)) <= tol
    up_inf, lo_inf = qp.u >= 1e20, qp.l <= -1e20
    assert np.all(y[up_inf] <= 0.0) and np.all(y[lo_inf] >= 0.0)
    pos, neg = y > 0, y < 0
    assert qp.u[pos] @ y[pos] + qp.l[neg] @ y[neg] < 0.0


def check_dual_certificate(qp, x, tol):
    assert np.max(np.abs(x)) == pytest.approx(1.0, rel=1e-12)
    assert qp.q @ x < 0.0
    assert np.max(np.abs(qp.P @ x)) <= tol
    Ax = qp.A @ x
    assert np.all(Ax[qp.u < 1e20] <= tol) and np.all(Ax[qp.l > -1e20] >= -tol)


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
@pytest.mark.parametrize("case", range(6))
def test_primal_infeasible(prec, case):
    qp = primal_cases()[case]
    ref = admm.solve(qp)
    assert ref.status == "primal_infeasible"
    with gb.Solver(qp, precision=prec) as s:
        st = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert st == gb.PRIMAL_INFEASIBLE, (st, info["iters"], ref.iters)
    assert np.all(np.isnan(x)) and np.all(np.isnan(z))
    assert info["obj"] == math.inf
    check_primal_certificate(qp, y, 1e-4 if prec == gb.FP64 else 2e-4)


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
@pytest.mark.parametrize("case", range(6))
def test_dual_infeasible(prec, case):
    qp = dual_cases()[case]
    ref = admm.solve(qp)
    assert ref.status == "dual_infeasible"
    with gb.Solver(qp, precision=prec) as s:
        st = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert st == gb.DUAL_INFEASIBLE, (st, info["iters"], ref.iters)
    assert np.all(np.isnan(y)) and np.all(np.isnan(z))
    assert info["obj"] == -math.inf
    check_dual_certificate(qp, x, 1e-4 if prec == gb.FP64 else 2e-4)


def test_detection_off_runs_to_max_iter_and_launches_fewer_kernels():
    qp = qpgen.random_primal_infeasible_qp(20, 40, 0)
    with gb.Solver(qp, precision=gb.FP64, eps_prim_inf=0.0, eps_dual_inf=0.0, max_iter=200) as s:
        assert s.solve() == gb.MAX_ITER
        off = s.info()
    with gb.Solver(qp, precision=gb.FP64, max_iter=200) as s:
        assert s.solve() == gb.PRIMAL_INFEASIBLE
        on = s.info()
    assert off["iters"] == 200 and on["iters"] < 200
    # each check runs one kernel more: the pass over A takes the detection's
    # rows of A with the check's, and the detection's pass over [P A'] is added
    checks = on["iters"] // 5
    base = 2 + 2 * on["iters"] + 3 * on["pcg_iters"]
    assert on["solve_launches"] == base + 4 * checks
    checks = off["iters"] // 5
    assert off["solve_launches"] == 2 + 2 * off["iters"] + 3 * off["pcg_iters"] + 3 * checks


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
def test_graph_and_host_loop_agree_on_infeasible(prec):
    for qp in (qpgen.random_primal_infeasible_qp(20, 40, 1), qpgen.random_dual_infeasible_qp(24, 30, 4, 1)):
        out = []
        for mode in (gb.LOOP_GRAPH, gb.LOOP_HOST):
            with gb.Solver(qp, precision=prec, loop_mode=mode) as s:
                st = s.solve()
                info = s.info()
                out.append((st, info["iters"], s.solution(), info["solve_launches"]))
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
        for a, b in zip(out[0][2], out[1][2]):
            np.testing.assert_array_equal(a, b)
        # the graph's kernel count (from the iteration counters) is the number
        # of kernels the host-driven loop launched one by one
        assert out[0][3] == out[1][3]


@pytest.mark.parametrize("name", ["random_300x3000", "lasso_50x2000", "portfolio_3000x30", "equality_200x100"])
def test_feasible_families_are_not_flagged_at_tight_tolerance(name):
    """Solvable problems run to 'solved' at 1e-6 in FP64 with detection on."""
    qp = qpgen.by_name(name, 0)
    with gb.Solver(qp, precision=gb.FP64, eps_abs=1e-6, eps_rel=1e-6, pcg_eps_min=1e-13, max_iter=20000) as s:
        st = s.solve()
    assert st == gb.SOLVED
