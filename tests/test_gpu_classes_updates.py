"""GPU parity on the other problem classes of the paper's benchmark set
(Control, Huber, SVM; Section 6.1) and for the parametric updates (new q,
new bounds, warm-started sequences as in model predictive control), against
the oracle.  The reference solutions use the oracle's direct solver with
OSQP's rho vector (eq. (rho_vec)), which reaches the same optimum as the
scalar rho of the GPU path in far fewer iterations on equality-heavy
problems."""
import functools

import numpy as np
import pytest

import qpgen
from oracle import admm, checks

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_1912_04263_gb300.binding")

CLASSES = ["control_20x10_T20", "huber_50x500", "svm_50x500"]


def tight(qp):
    return admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=200000, rho_vector=True))


@functools.lru_cache(maxsize=None)
def named(name):
    qp = qpgen.by_name(name, 0)
    return qp, tight(qp)


def assert_solution(qp, ref, x, y, z, info, obj_rel=None):
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) + 1e-12, (v, info)
    assert v.dual <= info["eps_dual"] * (1 + 1e-6) + 1e-12, (v, info)
    assert v.box <= 1e-6 * max(1.0, float(np.max(np.abs(z))))
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, ref.x, ref.y)
    f = admm.objective(qp.P, qp.q, x)
    assert abs(f - ref.obj) <= 1.001 * bound + 1e-9 * max(1.0, abs(ref.obj)), (f, ref.obj, bound)
    if obj_rel is not None:
        assert abs(f - ref.obj) <= obj_rel * max(1.0, abs(ref.obj)), (f, ref.obj)


def solve(s):
    st = s.solve()
    x, y, z = s.solution()
    return st, x, y, z, s.info()


@pytest.mark.parametrize("name", CLASSES)
@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
def test_classes_match_oracle(name, prec):
    qp, ref = named(name)
    assert ref.status == "solved"
    with gb.Solver(qp, precision=prec, max_iter=20000) as s:
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED, info
    assert_solution(qp, ref, x, y, z, info)


@pytest.mark.parametrize("name", ["huber_1000x20000", "svm_1000x20000"])
def test_larger_classes_fp32(name):
    """Members of the two classes with 3M nonzeros (61000 and 21000
    variables), FP32 path, against the oracle."""
    qp = qpgen.by_name(name, 0)
    ref = admm.solve(qp, admm.Settings(eps_abs=1e-7, eps_rel=1e-7, max_iter=100000, rho_vector=True))
    with gb.Solver(qp, precision=gb.FP32) as s:
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED, info
    assert_solution(qp, ref, x, y, z, info)


@pytest.mark.parametrize("name", ["huber_50x500", "svm_50x500"])
def test_classes_fp64_tight(name):
    qp, ref = named(name)
    with gb.Solver(qp, precision=gb.FP64, eps_abs=1e-6, eps_rel=1e-6, pcg_eps_min=1e-13, max_iter=40000) as s:
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED, info
    assert_solution(qp, ref, x, y, z, info, obj_rel=1e-6)


def perturbed(qp, seed, dq=0.0, dl=0.0, du=0.0):
    r = np.random.default_rng(seed)
    q = qp.q + dq * r.standard_normal(qp.n)
    fin_l, fin_u = np.isfinite(qp.l), np.isfinite(qp.u)
    l = np.where(fin_l, qp.l - dl * r.random(qp.m), qp.l)
    u = np.where(fin_u, qp.u + du * r.random(qp.m), qp.u)
    return qpgen.QP(qp.P, q, qp.A, l, u, name=qp.name + "_upd")


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
def test_update_lin_cost_matches_oracle_of_new_problem(prec):
    qp = qpgen.by_name("random_300x3000", 0)
    new = perturbed(qp, 1, dq=0.5)
    ref = tight(new)
    with gb.Solver(qp, precision=prec) as s:
        assert s.solve() == gb.SOLVED
        s.update_lin_cost(new.q)
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED
    assert_solution(new, ref, x, y, z, info)


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
@pytest.mark.parametrize("sides", ["both", "lower", "upper"])
def test_update_bounds_matches_oracle_of_new_problem(prec, sides):
    qp = qpgen.by_name("lasso_50x2000", 0)
    new = perturbed(qp, 2, dl=0.3 if sides != "upper" else 0.0, du=0.3 if sides != "lower" else 0.0)
    ref = tight(new)
    with gb.Solver(qp, precision=prec) as s:
        assert s.solve() == gb.SOLVED
        s.update_bounds(new.l if sides != "upper" else None, new.u if sides != "lower" else None)
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED
    assert_solution(new, ref, x, y, z, info)


def test_warm_started_mpc_sequence():
    """A receding-horizon sequence: the initial state changes between solves
    (the first nx equality rows), the next solve starts from the previous
    iterates (warm_start = 1), needs fewer iterations than a cold solve, and
    matches the oracle of each problem."""
    nx = 10
    qp = qpgen.control_qp(nx, 5, 10, 3)
    x0 = qp.meta["x_init"]
    with gb.Solver(qp, precision=gb.FP64, warm_start=1, max_iter=20000) as s, \
            gb.Solver(qp, precision=gb.FP64, max_iter=20000) as cold:
        assert s.solve() == gb.SOLVED
        warm_iters, cold_iters = [], []
        for k in range(1, 5):
            xk = x0 * (1.0 - 0.05 * k)
            l, u = qp.l.copy(), qp.u.copy()
            l[:nx] = u[:nx] = -xk
            step = qpgen.QP(qp.P, qp.q, qp.A, l, u)
            s.update_bounds(l, u)
            cold.update_bounds(l, u)
            st, x, y, z, info = solve(s)
            assert st == gb.SOLVED
            assert_solution(step, tight(step), x, y, z, info)
            assert cold.solve() == gb.SOLVED
            warm_iters.append(info["iters"])
            cold_iters.append(cold.info()["iters"])
    assert sum(warm_iters) < sum(cold_iters), (warm_iters, cold_iters)


def test_invalid_updates_leave_the_problem_unchanged():
    qp = qpgen.by_name("random_100x1000", 0)
    with gb.Solver(qp, precision=gb.FP64) as s:
        assert s.solve() == gb.SOLVED
        x0 = s.solution()[0]
        q = qp.q.copy()
        q[3] = np.nan
        with pytest.raises(gb.GbosqpError) as e:
            s.update_lin_cost(q)
        assert e.value.code == gb.ERR_NONFINITE
        l = qp.l.copy()
        l[5] = qp.u[5] + 1.0
        with pytest.raises(gb.GbosqpError) as e:
            s.update_bounds(l, None)
        assert e.value.code == gb.ERR_BOUNDS
        u = qp.u.copy()
        u[7] = -np.inf
        with pytest.raises(gb.GbosqpError) as e:
            s.update_bounds(None, u)
        assert e.value.code == gb.ERR_BOUNDS
        assert s.solve() == gb.SOLVED
        assert np.array_equal(s.solution()[0], x0)


def test_update_with_the_same_data_changes_nothing_but_rounding():
    """Re-sending the set-up's q, l, u rescales them in one step instead of
    the set-up's incremental passes: the problem is the same up to rounding
    (the iteration count may differ), so tight solves agree."""
    qp = qpgen.by_name("portfolio_3000x30", 0)
    kw = dict(precision=gb.FP64, eps_abs=1e-9, eps_rel=1e-9, pcg_eps_min=1e-14, max_iter=100000)
    with gb.Solver(qp, **kw) as s:
        assert s.solve() == gb.SOLVED
        x0 = s.solution()[0]
        s.update_lin_cost(qp.q)
        s.update_bounds(qp.l, qp.u)
        assert s.solve() == gb.SOLVED
        x1 = s.solution()[0]
    assert np.max(np.abs(x1 - x0)) <= 1e-6 * max(1.0, np.max(np.abs(x0)))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", ["control_20x10_T20", "lasso_50x2000"])
def test_rho_vector_trajectory_matches_oracle(name):
    """R = rho diag(rs) of eq. (rho_vec): 20 iterations of the GPU take the
    PCG steps of the FP64 CPU restatement with the same R and reach the same
    iterates."""
    qp = qpgen.by_name(name, 0)
    K = 20
    ref = admm.solve_pcg(qp, admm.Settings(rho_vector=True), max_iter=K)
    with gb.Solver(qp, precision=gb.FP64, loop_mode=gb.LOOP_HOST, rho_vector=1) as s:
        gb.gbosqp_set_iterates(s.h, np.zeros(qp.n), np.zeros(qp.m), np.zeros(qp.m), np.zeros(qp.n), 0.1)
        st, per = gb.gbosqp_admm_iterations(s.h, K)
        x, z, y, xt, rho = gb.gbosqp_get_iterates(s.h)
    xs, zs, ys, xts = ref.scaled_state
    assert per.tolist() == ref.pcg_per_iter[:K]
    assert relmax(x, xs) <= 1e-6 and relmax(z, zs) <= 1e-6 and relmax(y, ys) <= 1e-6


@pytest.mark.parametrize("prec", [gb.FP64, gb.FP32])
@pytest.mark.parametrize("name", ["control_20x10_T20", "huber_50x500", "lasso_50x2000", "equality_200x100"])
def test_rho_vector_solves_match_oracle(prec, name):
    """(On the equality class every row gets 1e3 rho, which makes PCG
    ill-conditioned enough that FP64 trajectories of the CPU restatement and
    the GPU drift apart by a PCG step; the solutions are compared.)"""
    qp, ref = named(name)
    with gb.Solver(qp, precision=prec, rho_vector=1, max_iter=20000) as s:
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED, info
    assert_solution(qp, ref, x, y, z, info)
    if name.startswith("control"):
        with gb.Solver(qp, precision=prec, max_iter=20000) as s:
            s.solve()
            assert info["iters"] < s.info()["iters"]


def test_rho_vector_follows_bound_updates():
    """Turning inequality rows into equalities by osqp_update_bounds moves
    them to the 1e3 rho class.  Pinning 50 rows of the 100 x 1000 random QP
    at the midpoints of their boxes is infeasible (HiGHS agrees) and is
    reported so; pinning them at A x of a feasible point solves and matches
    the oracle of the new problem."""
    qp = qpgen.by_name("random_100x1000", 0)
    l, u = qp.l.copy(), qp.u.copy()
    l[:50] = u[:50] = 0.5 * (qp.l[:50] + qp.u[:50])
    with gb.Solver(qp, precision=gb.FP64, rho_vector=1, max_iter=20000) as s:
        s.solve()
        x_feas = s.solution()[0]
        s.update_bounds(l, u)
        assert s.solve() == gb.PRIMAL_INFEASIBLE
        ax = qp.A @ x_feas
        l2, u2 = qp.l.copy(), qp.u.copy()
        l2[:50] = u2[:50] = np.clip(ax[:50], qp.l[:50], qp.u[:50])
        new = qpgen.QP(qp.P, qp.q, qp.A, l2, u2)
        s.update_bounds(l2, u2)
        st, x, y, z, info = solve(s)
    assert st == gb.SOLVED
    assert_solution(new, tight(new), x, y, z, info)
