"""Pins of the oracle's infeasibility detection (Section 3.1, eqs.
(prim_infeas) and (dual_infeas)) against facts outside the oracle: hand-made
problems whose certificate direction is known in closed form, and an
independent LP solver (HiGHS through scipy.optimize.linprog) that decides
primal feasibility and the existence of a descent direction of the
recession cone (Farkas' lemma; no GPU)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import qpgen
from oracle import admm


def lp_primal_feasible(qp) -> bool:
    """Is {x : l <= A x <= u} nonempty?  Decided by HiGHS."""
    A = sp.csr_matrix(qp.A)
    fu = qp.u < 1e20
    fl = qp.l > -1e20
    A_ub = sp.vstack([A[fu], -A[fl]], format="csr")
    b_ub = np.concatenate([qp.u[fu], -qp.l[fl]])
    r = linprog(np.zeros(qp.n), A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * qp.n, method="highs")
    assert r.status in (0, 2), r.message
    return r.status == 0


def lp_descent_direction(qp) -> float:
    """min q'd over P d = 0, (A d)_i <= 0 where u_i is finite, (A d)_i >= 0
    where l_i is finite, -1 <= d <= 1: negative iff the (feasible) QP is
    unbounded below.  Decided by HiGHS."""
    A = sp.csr_matrix(qp.A)
    fu = qp.u < 1e20
    fl = qp.l > -1e20
    A_ub = sp.vstack([A[fu], -A[fl]], format="csr")
    r = linprog(qp.q, A_ub=A_ub, b_ub=np.zeros(A_ub.shape[0]), A_eq=sp.csr_matrix(qp.P),
                b_eq=np.zeros(qp.n), bounds=[(-1, 1)] * qp.n, method="highs")
    assert r.status == 0, r.message
    return float(r.fun)


def test_hand_made_primal_certificate_direction():
    """x1 >= 1 and x1 <= 0: every certificate is a positive multiple of
    y = (-1, 1, 0) (A'y = 0 forces y1 = -y2; the infinite bounds fix the
    signs), so the unit-norm certificate is that vector."""
    qp = qpgen.infeasible_primal_qp()
    r = admm.solve(qp)
    assert r.status == "primal_infeasible"
    np.testing.assert_allclose(r.y, [-1.0, 1.0, 0.0], atol=1e-3)
    assert np.all(np.isnan(r.x)) and r.obj == math.inf


def test_hand_made_dual_certificate_direction():
    """min -x1 + x2^2 / 2 with x1 >= 0 unbounded above: the recession
    directions with q'd < 0 and P d = 0 are positive multiples of (1, 0)."""
    qp = qpgen.infeasible_dual_qp()
    r = admm.solve(qp)
    assert r.status == "dual_infeasible"
    np.testing.assert_allclose(r.x, [1.0, 0.0], atol=1e-3)
    assert r.obj == -math.inf


def test_certificate_tests_on_exact_certificates():
    """The two tests accept exact certificates and reject non-certificates."""
    qp = qpgen.infeasible_primal_qp()
    y = admm.primal_infeasibility(qp.A, qp.l, qp.u, np.array([-2.0, 2.0, 0.0]), 1e-4)
    np.testing.assert_array_equal(y, [-1.0, 1.0, 0.0])
    # a component facing an infinite bound is clipped: +5 on row 0 (u = inf)
    y = admm.primal_infeasibility(qp.A, qp.l, qp.u, np.array([5.0, 2.0, 0.0]), 1e-4)
    assert y is None  # clipped to (0, 1, 0): A'y = (1, 0) is not small
    y = admm.primal_infeasibility(qp.A, qp.l, qp.u, np.array([-2.0, 2.0, 0.0]), 1e-4)
    np.testing.assert_array_equal(y, [-1.0, 1.0, 0.0])
    assert admm.primal_infeasibility(qp.A, qp.l, qp.u, np.array([2.0, -2.0, 0.0]), 1e-4) is None
    assert admm.primal_infeasibility(qp.A, qp.l, qp.u, np.zeros(3), 1e-4) is None
    qd = qpgen.infeasible_dual_qp()
    np.testing.assert_array_equal(admm.dual_infeasibility(qd.P, qd.q, qd.A, qd.l, qd.u, np.array([3.0, 0.0]), 1e-4),
                                  [1.0, 0.0])
    assert admm.dual_infeasibility(qd.P, qd.q, qd.A, qd.l, qd.u, np.array([-3.0, 0.0]), 1e-4) is None
    assert admm.dual_infeasibility(qd.P, qd.q, qd.A, qd.l, qd.u, np.array([0.0, 1.0]), 1e-4) is None


@pytest.mark.parametrize("seed", range(4))
def test_random_primal_infeasible_matches_lp(seed):
    qp = qpgen.random_primal_infeasible_qp(20, 40, seed)
    assert not lp_primal_feasible(qp)
    for solver in (admm.solve, admm.solve_pcg):
        r = solver(qp)
        assert r.status == "primal_infeasible", (solver.__name__, r.status, r.iters)
        y = r.y
        assert np.max(np.abs(y)) == pytest.approx(1.0)
        assert np.max(np.abs(qp.A.T @ y)) <= 1e-4
        pos, neg = y > 0, y < 0
        assert qp.u[pos] @ y[pos] + qp.l[neg] @ y[neg] < 0.0


@pytest.mark.parametrize("seed", range(4))
def test_random_dual_infeasible_matches_lp(seed):
    qp = qpgen.random_dual_infeasible_qp(24, 30, 4, seed)
    assert lp_primal_feasible(qp)
    assert lp_descent_direction(qp) < -1e-3
    for solver in (admm.solve, admm.solve_pcg):
        r = solver(qp)
        assert r.status == "dual_infeasible", (solver.__name__, r.status, r.iters)
        x = r.x
        assert np.max(np.abs(x)) == pytest.approx(1.0)
        assert qp.q @ x < 0.0
        assert np.max(np.abs(qp.P @ x)) <= 1e-4


@pytest.mark.parametrize("seed", range(6))
def test_feasible_bounded_problems_are_not_flagged(seed):
    """Solvable problems (LP-confirmed) reach 'solved', never an infeasibility
    status, also at tight tolerances where iterates differ by tiny steps."""
    for qp in (qpgen.random_qp(30, 60, seed), qpgen.tiny_qp(4, 7, seed, n_eq=1, n_inf=2),
               qpgen.lasso_qp(8, 40, seed)):
        assert lp_primal_feasible(qp)
        for eps in (1e-3, 1e-7):
            r = admm.solve(qp, admm.Settings(eps_abs=eps, eps_rel=eps, max_iter=20000))
            assert r.status == "solved", (qp.name, eps, r.status)


def test_printed_margin_would_flag_a_solvable_problem():
    """With the margin as printed (support < +eps) a solvable problem with
    duplicated equality rows has a dy that passes both tests (A'dy = 0 and
    support 0 < eps): the reading with -eps rejects it, and the solve of
    that problem ends 'solved'."""
    qp = qpgen.equality_qp(6, 4, 3)
    A = sp.vstack([qp.A, qp.A], format="csr")  # duplicated rows: null(A') nontrivial
    dup = qpgen.QP(qp.P, qp.q, A, np.concatenate([qp.l, qp.l]), np.concatenate([qp.u, qp.u]))
    y_drift = np.concatenate([np.ones(4), -np.ones(4)])
    pos, neg = y_drift > 0, y_drift < 0
    support = dup.u[pos] @ y_drift[pos] + dup.l[neg] @ y_drift[neg]
    assert abs(support) < 1e-12 and np.max(np.abs(dup.A.T @ y_drift)) < 1e-12  # printed form: accept
    assert admm.primal_infeasibility(dup.A, dup.l, dup.u, y_drift, 1e-4) is None
    assert admm.solve(dup).status == "solved"
