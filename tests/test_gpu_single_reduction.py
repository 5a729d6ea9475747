"""GPU parity of the single-reduction PCG (pcg_variant = PCG_SINGLE_REDUCTION):
the device's two-kernel step against the FP64 restatement
oracle.admm.pcg_single_reduction (the Chronopoulos-Gear rearrangement of
Algorithm 3, pinned on the CPU against Algorithm 3 itself), the ADMM
trajectory against oracle.admm.solve_pcg with the same variant, and solves
against the oracle's optimum.

Tolerances as in test_gpu_parity: FP64 iterates 1e-9 for a few PCG steps,
identical PCG step counts along an ADMM trajectory with iterates to 1e-6;
solutions by the optimality conditions and the convexity bound."""
import functools
import os

import numpy as np
import pytest

import qpgen
from oracle import admm, checks

pytestmark = pytest.mark.gpu

SMALL = ["random_100x1000", "lasso_50x2000", "portfolio_3000x30", "random_300x3000"]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding


@functools.lru_cache(maxsize=None)
def problem(name):
    return qpgen.by_name(name, 0)


@functools.lru_cache(maxsize=None)
def scaled(name):
    qp = problem(name)
    return admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, 10)


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("name", SMALL)
def test_sr_pcg_steps_match_restatement(gb, name):
    qp, sc = problem(name), scaled(name)
    rng = np.random.default_rng(31)
    b = rng.standard_normal(qp.n)
    x0 = 0.1 * rng.standard_normal(qp.n)
    rho = 0.3
    Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, 1e-6, rho)
    K = lambda v: admm.reduced_kkt_apply(sc.P, sc.A, 1e-6, rho, v)  # noqa: E731
    with gb.Solver(qp, precision=gb.FP64, pcg_variant=gb.PCG_SINGLE_REDUCTION) as s:
        for k in (1, 2, 5):
            ref = admm.pcg_single_reduction(K, b, x0, Minv, 0.0, k)
            x, it, rn = gb.gbosqp_pcg(s.h, rho, b, x0, 0.0, k)
            assert it == ref.iters == k
            assert relmax(x, ref.x) <= 1e-9, k
            assert abs(rn - ref.r_norm) <= 1e-9 * max(ref.r_norm, 1.0)
        # the stopping rule on the device's own trajectory (as for Algorithm 3)
        x, it, rn = gb.gbosqp_pcg(s.h, rho, b, x0, 1e-4, 200)
        assert 0 < it < 200 and rn <= 1e-4
        _, it1, rn1 = gb.gbosqp_pcg(s.h, rho, b, x0, 0.0, it - 1)
        assert it1 == it - 1 and rn1 > 1e-4


@pytest.mark.parametrize("name", ["random_100x1000", "lasso_50x2000", "random_300x3000"])
def test_sr_admm_trajectory_matches_restatement(gb, name):
    """20 iterations of Algorithm 1 with the single-reduction PCG: the same
    PCG step count in every iteration as the FP64 restatement, and the same
    iterates."""
    qp = problem(name)
    ref = admm.solve_pcg(qp, admm.Settings(pcg_variant="single_reduction"), max_iter=20)
    with gb.Solver(qp, precision=gb.FP64, loop_mode=gb.LOOP_HOST, pcg_variant=gb.PCG_SINGLE_REDUCTION) as s:
        gb.gbosqp_set_iterates(s.h, np.zeros(qp.n), np.zeros(qp.m), np.zeros(qp.m), np.zeros(qp.n), 0.1)
        st, per = gb.gbosqp_admm_iterations(s.h, 20)
        x, z, y, xt, rho = gb.gbosqp_get_iterates(s.h)
    assert per.tolist() == ref.pcg_per_iter[:20]
    xs, zs, ys, _ = ref.scaled_state
    assert relmax(x, xs) <= 1e-6 and relmax(z, zs) <= 1e-6 and relmax(y, ys) <= 1e-6
    assert abs(rho - ref.rho) <= 1e-6 * ref.rho


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", [0, 1])
def test_sr_solve_matches_oracle(gb, name, prec):
    qp = problem(name)
    kw = dict(precision=prec, pcg_variant=gb.PCG_SINGLE_REDUCTION)
    pol = os.path.join(os.path.dirname(gb.__file__), "policy", "rho_policy.bin")
    if prec == gb.FP32 and os.path.exists(pol):
        kw.update(rho_policy=gb.RHO_LEARNED, policy_params=gb.load_policy(pol))
    with gb.Solver(qp, **kw) as s:
        status = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert status == gb.SOLVED, info
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) + 1e-12 and v.dual <= info["eps_dual"] * (1 + 1e-6) + 1e-12
    ref = admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=100000))
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, ref.x, ref.y)
    f = admm.objective(qp.P, qp.q, x)
    assert abs(f - ref.obj) <= 1.001 * bound + 1e-9 * max(1.0, abs(ref.obj))


def test_sr_graph_and_host_loop_are_identical(gb):
    qp = problem("lasso_50x2000")
    out = []
    for mode in (gb.LOOP_GRAPH, gb.LOOP_HOST):
        with gb.Solver(qp, precision=gb.FP32, loop_mode=mode, pcg_variant=gb.PCG_SINGLE_REDUCTION) as s:
            s.solve()
            out.append((s.solution(), s.info()))
    (x1, y1, z1), i1 = out[0]
    (x2, y2, z2), i2 = out[1]
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2) and np.array_equal(z1, z2)
    assert i1["iters"] == i2["iters"] and i1["pcg_iters"] == i2["pcg_iters"]
