"""GPU parity on the degenerate problem shapes, against their closed forms
(the same cases pin the oracle on the CPU): a linear program over a box
(P = 0), a problem without constraints (m = 0, empty A, y and z) and scalar
problems (n = 1, one of them an equality).

FP64 solves run at eps 1e-9 with the PCG tolerance floor at 1e-13 (with
m = 0 the adaptive PCG tolerance sits on its floor, which bounds the
accuracy); FP32 solves run at the default 1e-3 and are judged by the
optimality conditions recomputed in FP64 on the host, and by the convexity
bound on the objective error."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm, checks
from qpgen.problems import QP

pytestmark = pytest.mark.gpu

TIGHT = dict(eps_abs=1e-9, eps_rel=1e-9, pcg_eps_min=1e-13, max_iter=20000)


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding


def box_lp(n=30, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n)
    l = -rng.uniform(0.5, 2.0, n)
    u = rng.uniform(0.5, 2.0, n)
    qp = QP(sp.csr_matrix((n, n)), q, sp.identity(n, format="csr"), l, u, name="box_lp")
    return qp, np.where(q > 0, l, u), -q


def free_qp(n=25, seed=1):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    P = sp.csr_matrix(M @ M.T + np.eye(n))
    q = rng.standard_normal(n)
    qp = QP(P, q, sp.csr_matrix((0, n)), np.zeros(0), np.zeros(0), name="free")
    return qp, np.linalg.solve(P.toarray(), -q), np.zeros(0)


def scalar_qp(q0, l0, u0, p=2.0, a=0.5):
    qp = QP(sp.csr_matrix([[p]]), np.array([q0]), sp.csr_matrix([[a]]), np.array([l0]), np.array([u0]))
    x = min(max(-q0 / p, l0 / a), u0 / a)
    return qp, np.array([x]), np.array([-(p * x + q0) / a])


CASES = {"box_lp": box_lp, "free": free_qp,
         "scalar_interior": lambda: scalar_qp(0.5, -1.0, 1.0),
         "scalar_upper": lambda: scalar_qp(-3.0, -1.0, 1.0),
         "scalar_lower": lambda: scalar_qp(8.0, -1.0, 1.0),
         "scalar_equality": lambda: scalar_qp(2.0, 0.7, 0.7)}


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_tight_solve_reaches_the_closed_form(gb, case):
    qp, x_star, y_star = CASES[case]()
    with gb.Solver(qp, precision=gb.FP64, **TIGHT) as s:
        st = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert st == gb.SOLVED, info
    assert y.shape == (qp.m,) and z.shape == (qp.m,)
    scale = max(1.0, float(np.max(np.abs(x_star))))
    assert np.max(np.abs(x - x_star)) <= 1e-6 * scale
    if qp.m:
        assert np.max(np.abs(y - y_star)) <= 1e-6 * max(1.0, float(np.max(np.abs(y_star))))


@pytest.mark.parametrize("case", list(CASES))
def test_fp32_solve_meets_the_optimality_conditions(gb, case):
    qp, x_star, y_star = CASES[case]()
    with gb.Solver(qp, precision=gb.FP32) as s:
        st = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert st == gb.SOLVED, info
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) + 1e-12, (v, info)
    assert v.dual <= info["eps_dual"] * (1 + 1e-6) + 1e-12, (v, info)
    f = admm.objective(qp.P, qp.q, x)
    f_star = admm.objective(qp.P, qp.q, x_star)
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, x_star, y_star)
    assert abs(f - f_star) <= 1.001 * bound + 1e-9 * max(1.0, abs(f_star)), (f, f_star, bound)
