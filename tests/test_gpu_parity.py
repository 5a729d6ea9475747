"""GPU parity: every step of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C ABI.

Tolerances:
* FP64 path: element-wise relative 1e-12 for set-up and SpMV (sums of at most
  a few thousand terms), 1e-9 for a few PCG steps, identical PCG step counts
  along an ADMM trajectory.
* FP32 path: a matrix value rounded to FP32 differs by at most 2^-24
  relatively; an FP32 row sum of L products differs from the exact one by
  at most about (L + 2) 2^-24 times the sum of |a_ij x_j| (the standard
  recursive-summation bound), which the SpMV test uses row by row.
* Solutions: residuals within the solver's own eps_prim / eps_dual rule
  recomputed in FP64 on the unscaled data; objective within the convexity
  bound |f - f*| <= max(||y||_1, ||y*||_1) ||r_prim|| + ||r_dual|| ||x - x*||_1,
  and within 1e-3 relative where the oracle's own 1e-3 solve achieves it.
"""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import admm, checks

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24

SMALL = ["random_100x1000", "lasso_50x2000", "portfolio_3000x30", "random_300x3000", "portfolio_8000x50"]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding


@functools.lru_cache(maxsize=None)
def problem(name, seed=0):
    return qpgen.by_name(name, seed)


@functools.lru_cache(maxsize=None)
def scaled_ref(name):
    qp = problem(name)
    return admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, 10)


@functools.lru_cache(maxsize=None)
def tight_ref(name):
    qp = problem(name)
    return admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=100000))


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def fp32_row_bound(M, x):
    """(L_i + 2) 2^-24 sum_j |M_ij x_j| per row, plus the rounding of x."""
    L = np.diff(M.indptr)
    return (L + 4) * U32 * (abs(M) @ np.abs(x)) + 1e-30


# ----------------------------------------------------------------- set-up --

@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", [0, 1])
def test_setup_equilibration_matches_oracle(gb, name, prec):
    """Algorithm 2 on the device: D, E, c and the scaled matrices."""
    qp, sc = problem(name), scaled_ref(name)
    with gb.Solver(qp, precision=prec) as s:
        D, E, c = gb.gbosqp_get_scaling(s.h)
        A = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_A)
        PAt = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_PAT)
    assert relmax(D, sc.D) <= 1e-12 and relmax(E, sc.E) <= 1e-12 and abs(c - sc.c) <= 1e-12 * sc.c
    ref_pat = sp.hstack([sc.P, sc.A.T]).tocsr()
    ref_pat.sort_indices()
    for got, ref in [(A, sc.A), (PAt, ref_pat)]:
        assert np.array_equal(got.indptr, ref.indptr) and np.array_equal(got.indices, ref.indices)
        tol = 1e-12 if prec == 1 else 1.01 * U32
        assert np.all(np.abs(got.data - ref.data) <= tol * np.abs(ref.data) + 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_setup_from_upper_triangle_equals_full(gb, prec):
    qp = problem("random_100x1000")
    with gb.Solver(qp, precision=prec, P_is_upper=True) as s1, gb.Solver(qp, precision=prec) as s2:
        a = gb.gbosqp_get_scaled_csr(s1.h, gb.MAT_PAT)
        b = gb.gbosqp_get_scaled_csr(s2.h, gb.MAT_PAT)
        assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
        assert np.array_equal(a.data, b.data)


# ------------------------------------------------------------------- SpMV --

def _spmv_case(gb, s, M, which, x, prec, fp64acc):
    y = gb.gbosqp_spmv(s.h, which, x, fp64acc)
    if prec == 1:
        xr = x
    else:
        xr = x.astype(np.float32).astype(np.float64)
    ref = M @ xr
    if prec == 1:
        bound = 1e-12 * (abs(M) @ np.abs(xr)) + 1e-300
    elif fp64acc:  # FP32 products (one rounding each) summed in FP64
        bound = 1.01 * U32 * (abs(M) @ np.abs(xr)) + 1e-300
    else:
        bound = fp32_row_bound(M, xr) + U32 * np.abs(ref)
    assert np.all(np.abs(y - ref) <= bound), float(np.max(np.abs(y - ref) / bound))


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", [0, 1])
def test_spmv_matches_oracle(gb, name, prec):
    qp = problem(name)
    rng = np.random.default_rng(1)
    with gb.Solver(qp, precision=prec) as s:
        A = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_A)
        PAt = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_PAT)
        for fp64acc in (False, True):
            _spmv_case(gb, s, A, gb.MAT_A, rng.standard_normal(qp.n), prec, fp64acc)
            _spmv_case(gb, s, PAt, gb.MAT_PAT, rng.standard_normal(qp.n + qp.m), prec, fp64acc)


@pytest.mark.parametrize("prec", [0, 1])
def test_spmv_edge_row_lengths(gb, prec):
    """Empty rows, rows at and around the 2048-nonzero item capacity, and long
    rows split into pieces (A) or long columns (A' rows in [P A'])."""
    lens = [0, 1, 31, 32, 33, 2047, 2048, 2049, 4096, 4097, 10000, 50000, 0, 3] + [5] * 3000 + [0] * 7
    qp = qpgen.rowlen_qp(lens, 60000, 3)
    rng = np.random.default_rng(2)
    with gb.Solver(qp, precision=prec, scaling_iters=0) as s:
        A = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_A)
        PAt = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_PAT)
        assert np.array_equal(np.diff(A.indptr), np.array(lens))
        for fp64acc in (False, True):
            _spmv_case(gb, s, A, gb.MAT_A, rng.standard_normal(qp.n), prec, fp64acc)
            _spmv_case(gb, s, PAt, gb.MAT_PAT, rng.standard_normal(qp.n + qp.m), prec, fp64acc)


# -------------------------------------------------------------------- PCG --

@pytest.mark.parametrize("name", SMALL)
def test_pcg_fp64_matches_algorithm3(gb, name):
    qp, sc = problem(name), scaled_ref(name)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(qp.n)
    x0 = 0.1 * rng.standard_normal(qp.n)
    rho = 0.3
    Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, 1e-6, rho)
    K = lambda v: admm.reduced_kkt_apply(sc.P, sc.A, 1e-6, rho, v)  # noqa: E731
    with gb.Solver(qp, precision=gb.FP64) as s:
        for k in (1, 2, 5):
            ref = admm.pcg(K, b, x0, Minv, 0.0, k)
            x, it, rn = gb.gbosqp_pcg(s.h, rho, b, x0, 0.0, k)
            assert it == ref.iters == k
            assert relmax(x, ref.x) <= 1e-9, k
            assert abs(rn - ref.r_norm) <= 1e-9 * max(ref.r_norm, 1.0)
        # stopping rule ||r||_inf <= eps (reading S3), checked on the
        # device's own trajectory: it stops at the first step whose residual
        # is within eps (the run one step shorter ends above eps), and the
        # iterate it returns has a true residual K x - b, recomputed here in
        # FP64, within eps up to the drift of the recurrence (10^-10 of
        # ||K||_inf ||x||_inf + ||b||_inf).  Iterates are compared step by
        # step only over the first steps above: on the ill-conditioned
        # problems two FP64 CG runs with different summation orders drift
        # apart after a few tens of steps, and ||r||_inf, not being monotone,
        # can then first cross eps at a different step.
        Kn = float(np.max(np.abs(sc.P).sum(axis=1) + 1e-6 + rho * (abs(sc.A).T @ (abs(sc.A) @ np.ones(qp.n)))))
        for eps in (0.05 * ref.r_norm, 1e-4):
            x, it, rn = gb.gbosqp_pcg(s.h, rho, b, x0, eps, 200)
            assert 0 < it < 200 and rn <= eps
            _, it1, rn1 = gb.gbosqp_pcg(s.h, rho, b, x0, 0.0, it - 1)
            assert it1 == it - 1 and rn1 > eps
            true_r = np.max(np.abs(K(x) - b))
            assert true_r <= eps + 1e-10 * (Kn * np.max(np.abs(x)) + np.max(np.abs(b))), (eps, it, true_r)


@pytest.mark.parametrize("name", SMALL)
def test_pcg_fp32_first_steps(gb, name):
    qp, sc = problem(name), scaled_ref(name)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(qp.n)
    rho = 0.3
    Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, 1e-6, rho)
    K = lambda v: admm.reduced_kkt_apply(sc.P, sc.A, 1e-6, rho, v)  # noqa: E731
    with gb.Solver(qp, precision=gb.FP32) as s:
        for k in (1, 2, 3):
            ref = admm.pcg(K, b, np.zeros(qp.n), Minv, 0.0, k)
            x, it, _ = gb.gbosqp_pcg(s.h, rho, b, np.zeros(qp.n), 0.0, k)
            assert it == k
            assert relmax(x, ref.x) <= 2e-4, k


def test_pcg_zero_steps_and_exact_start(gb):
    qp = problem("random_100x1000")
    sc = scaled_ref("random_100x1000")
    with gb.Solver(qp, precision=gb.FP64) as s:
        b = np.ones(qp.n)
        x, it, rn = gb.gbosqp_pcg(s.h, 0.5, b, np.zeros(qp.n), 0.0, 0)
        assert it == 0 and np.all(x == 0.0) and abs(rn - 1.0) <= 1e-15
        K = (sc.P + 1e-6 * sp.identity(qp.n) + 0.5 * (sc.A.T @ sc.A)).toarray()
        xs = np.linalg.solve(K, b)
        x, it, rn = gb.gbosqp_pcg(s.h, 0.5, b, xs, 1e-8, 50)
        assert it == 0 and rn <= 1e-8


# ------------------------------------------------------- ADMM trajectory --

# The portfolio problems are ill-conditioned enough that a PCG step count
# (the first crossing of a non-monotone ||r||_inf below eps) changes with the
# summation order: the 3000-asset one is followed for 3 iterations, the
# 8000-asset one (whose first PCG solve already takes 10 steps) not at all.
@pytest.mark.parametrize("name", [n for n in SMALL if n != "portfolio_8000x50"])
def test_admm_trajectory_fp64_matches_cpu_restatement(gb, name):
    """20 iterations of Algorithm 1 with PCG, checks and rho updates: the GPU
    takes the same number of PCG steps in every iteration as the FP64 CPU
    restatement of Section 5.3, and reaches the same iterates."""
    qp = problem(name)
    K = 3 if name.startswith("portfolio") else 20
    ref = admm.solve_pcg(qp, admm.Settings(), max_iter=K)
    with gb.Solver(qp, precision=gb.FP64, loop_mode=gb.LOOP_HOST) as s:
        gb.gbosqp_set_iterates(s.h, np.zeros(qp.n), np.zeros(qp.m), np.zeros(qp.m), np.zeros(qp.n), 0.1)
        st, per = gb.gbosqp_admm_iterations(s.h, K)
        x, z, y, xt, rho = gb.gbosqp_get_iterates(s.h)
    assert per.tolist() == ref.pcg_per_iter[:K]
    xs, zs, ys, xts = ref.scaled_state
    assert relmax(x, xs) <= 1e-6 and relmax(z, zs) <= 1e-6 and relmax(y, ys) <= 1e-6
    assert abs(rho - ref.rho) <= 1e-6 * ref.rho


@pytest.mark.parametrize("name", SMALL)
def test_check_matches_oracle_residuals(gb, name):
    """The termination check (Section 3.1, readings S1-S2) at a mid-solve
    state against the oracle's residual functions on the same state."""
    qp, sc = problem(name), scaled_ref(name)
    ref = admm.solve_pcg(qp, admm.Settings(), max_iter=7)
    xs, zs, ys, xts = ref.scaled_state
    with gb.Solver(qp, precision=gb.FP64, loop_mode=gb.LOOP_HOST) as s:
        gb.gbosqp_set_iterates(s.h, xs, zs, ys, xts, 0.1)
        c = gb.gbosqp_check(s.h)
    xu, zu, yu = admm.unscale(sc, xs, zs, ys)
    ru = admm.residuals(qp.P, qp.q, qp.A, xu, zu, yu)
    rs = admm.residuals(sc.P, sc.q, sc.A, xs, zs, ys)
    for got, want in [(c["r_prim"], ru.r_prim), (c["r_dual"], ru.r_dual), (c["eps_prim"], ru.eps_prim),
                      (c["eps_dual"], ru.eps_dual), (c["r_prim_s"], rs.r_prim), (c["r_dual_s"], rs.r_dual),
                      (c["norm_Ax_s"], rs.norm_Ax), (c["norm_z_s"], rs.norm_z), (c["norm_Px_s"], rs.norm_Px),
                      (c["norm_Aty_s"], rs.norm_Aty), (c["norm_q_s"], rs.norm_q),
                      (c["obj"], admm.objective(qp.P, qp.q, xu))]:
        assert abs(got - want) <= 1e-9 * max(abs(want), 1e-3), (got, want)


@pytest.mark.parametrize("name", SMALL)
def test_check_fp32_matches_fp64_definition(gb, name):
    """FP32 handle: the termination check forms FP32 products and adds them
    with FP64 accuracy (compensated FP32 lane sums combined in FP64, reading
    S13).  Against the FP64 definitions of Section 3.1 evaluated on the same
    FP32 data (the scaled matrices as the device holds them, read back
    exactly, q_bar and the iterates rounded to FP32, the device's D, E, c),
    every quantity agrees within the rounding of the products: 2^-24 of
    |a_ij x_j| each, taken as 2^-23 of the row's sum of |a_ij x_j|."""
    qp = problem(name)
    ref = admm.solve_pcg(qp, admm.Settings(), max_iter=7)
    f32 = lambda v: np.asarray(v, np.float32).astype(np.float64)  # noqa: E731
    xs, zs, ys, xts = (f32(v) for v in ref.scaled_state)
    with gb.Solver(qp, precision=gb.FP32, loop_mode=gb.LOOP_HOST) as s:
        gb.gbosqp_set_iterates(s.h, xs, zs, ys, xts, 0.1)
        c = gb.gbosqp_check(s.h)
        A = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_A)
        PAt = gb.gbosqp_get_scaled_csr(s.h, gb.MAT_PAT)
        D, E, cost = gb.gbosqp_get_scaling(s.h)
    n = qp.n
    P, At = PAt[:, :n], PAt[:, n:]
    qb = f32(scaled_ref(name).q)
    ax, px, aty = A @ xs, P @ xs, At @ ys
    eA = 2.0 ** -23 * (abs(A) @ np.abs(xs))
    eP, eT = 2.0 ** -23 * (abs(P) @ np.abs(xs)), 2.0 ** -23 * (abs(At) @ np.abs(ys))
    rd = px + qb + aty
    mx = lambda v: float(np.max(np.abs(v))) if len(v) else 0.0  # noqa: E731
    ci = 1.0 / cost
    want = {
        "r_prim_s": (mx(ax - zs), mx(eA)), "norm_Ax_s": (mx(ax), mx(eA)), "norm_z_s": (mx(zs), 0.0),
        "r_dual_s": (mx(rd), mx(eP + eT)), "norm_Px_s": (mx(px), mx(eP)), "norm_Aty_s": (mx(aty), mx(eT)),
        "r_prim": (mx((ax - zs) / E), mx(eA / E)), "r_dual": (mx(rd / D) * ci, mx((eP + eT) / D) * ci),
        "obj": ((0.5 * xs @ px + qb @ xs) * ci, 0.5 * np.abs(xs) @ eP * ci),
    }
    nAx, nz = mx(ax / E), mx(zs / E)
    nPx, nAty, nq = mx(px / D) * ci, mx(aty / D) * ci, mx(qb / D) * ci
    want["eps_prim"] = (1e-3 + 1e-3 * max(nAx, nz), 1e-3 * mx(eA / E))
    want["eps_dual"] = (1e-3 + 1e-3 * max(nPx, nAty, nq), 1e-3 * (mx((eP + eT) / D) * ci + 2.0 ** -23 * nq))
    for k, (w, tol) in want.items():
        assert abs(c[k] - w) <= tol + 1e-12 * max(abs(w), 1e-3), (k, c[k], w, tol)


# -------------------------------------------------------------- solutions --

def _assert_solution(gb, qp, name, x, y, z, info, obj_rel=None):
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-6) + 1e-12, (v, info)
    assert v.dual <= info["eps_dual"] * (1 + 1e-6) + 1e-12, (v, info)
    assert v.box <= 1e-6 * max(1.0, float(np.max(np.abs(z))))
    ref = tight_ref(name)
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, ref.x, ref.y)
    f = admm.objective(qp.P, qp.q, x)
    assert abs(f - ref.obj) <= 1.001 * bound + 1e-9 * max(1.0, abs(ref.obj)), (f, ref.obj, bound)
    if obj_rel is not None:
        assert abs(f - ref.obj) <= obj_rel * max(1.0, abs(ref.obj)), (f, ref.obj)
    assert abs(info["obj"] - f) <= 1e-6 * max(1.0, abs(f))


@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_matches_oracle(gb, name, prec):
    qp = problem(name)
    with gb.Solver(qp, precision=prec) as s:
        status = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert status == gb.SOLVED, info
    # 1e-3 relative where the oracle's own 1e-3 solve gets there
    own = admm.solve(qp)
    tight = tight_ref(name)
    ok = abs(own.obj - tight.obj) <= 1e-3 * max(1.0, abs(tight.obj))
    _assert_solution(gb, qp, name, x, y, z, info, obj_rel=1e-3 if ok else None)
    # against the oracle's own solve at the same eps: both objectives lie
    # within their convexity bounds of f*, so within the sum of the bounds of
    # each other
    v, vo = checks.kkt_violation(qp, x, z, y), checks.kkt_violation(qp, own.x, own.z, own.y)
    b_gpu = checks.objective_error_bound(x, y, v.prim, v.dual, tight.x, tight.y)
    b_own = checks.objective_error_bound(own.x, own.y, vo.prim, vo.dual, tight.x, tight.y)
    f = admm.objective(qp.P, qp.q, x)
    assert abs(f - own.obj) <= 1.001 * (b_gpu + b_own) + 1e-9 * max(1.0, abs(own.obj)), (f, own.obj, b_gpu, b_own)


@pytest.mark.parametrize("name", ["random_100x1000", "lasso_50x2000", "random_300x3000"])
def test_solve_fp64_tight(gb, name):
    """FP64 path at eps_abs = eps_rel = 1e-6: residuals within the rule and
    objective within 1e-6 relative of the oracle."""
    qp = problem(name)
    with gb.Solver(qp, precision=gb.FP64, eps_abs=1e-6, eps_rel=1e-6, max_iter=20000) as s:
        status = s.solve()
        x, y, z = s.solution()
        info = s.info()
    assert status == gb.SOLVED, info
    _assert_solution(gb, qp, name, x, y, z, info, obj_rel=1e-6)


def test_graph_and_host_loop_are_identical(gb):
    qp = problem("lasso_50x2000")
    out = []
    for mode in (gb.LOOP_GRAPH, gb.LOOP_HOST):
        with gb.Solver(qp, precision=gb.FP32, loop_mode=mode) as s:
            s.solve()
            out.append((s.solution(), s.info()))
    (x1, y1, z1), i1 = out[0]
    (x2, y2, z2), i2 = out[1]
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2) and np.array_equal(z1, z2)
    assert i1["iters"] == i2["iters"] and i1["pcg_iters"] == i2["pcg_iters"]


def test_repeated_solves_are_bitwise_identical(gb):
    qp = problem("portfolio_8000x50")
    with gb.Solver(qp, precision=gb.FP32) as s:
        s.solve()
        a = s.solution()
        s.solve()
        b = s.solution()
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("seed,n,m,neq,ninf", [(0, 3, 5, 0, 0), (1, 4, 7, 1, 2), (2, 5, 8, 2, 3), (4, 5, 6, 1, 1)])
def test_brute_force_tiny(gb, seed, n, m, neq, ninf):
    qp = qpgen.tiny_qp(n, m, seed, n_eq=neq, n_inf=ninf)
    xb, yb = checks.brute_force(qp)
    # the PCG tolerance floor (1e-7 in Section 5.3.4) is lowered for a 1e-10 solve
    with gb.Solver(qp, precision=gb.FP64, eps_abs=1e-10, eps_rel=1e-10, max_iter=50000, pcg_eps_min=1e-14) as s:
        assert s.solve() == gb.SOLVED
        x, y, z = s.solution()
    assert np.max(np.abs(x - xb)) <= 1e-7
    assert np.max(np.abs(y - yb)) <= 1e-6


@pytest.mark.parametrize("seed,scale_a", [(0, False), (1, True)])
def test_box_closed_form(gb, seed, scale_a):
    qp = qpgen.box_qp(3000, seed, with_inf=True, scale_a=scale_a)
    xs, zs, ys = checks.box_qp_solution(qp.P.diagonal(), qp.q, qp.A.diagonal(), qp.l, qp.u)
    with gb.Solver(qp, precision=gb.FP64, eps_abs=1e-9, eps_rel=1e-9, max_iter=20000, pcg_eps_min=1e-13) as s:
        assert s.solve() == gb.SOLVED
        x, y, z = s.solution()
    assert np.max(np.abs(x - xs)) <= 1e-7
    assert np.max(np.abs(y - ys)) <= 1e-6


def test_update_rho_and_warm_start(gb):
    qp = problem("random_300x3000")
    with gb.Solver(qp, precision=gb.FP64, rho_policy=gb.RHO_FIXED) as s:
        s.update_rho(0.7)
        assert s.solve() == gb.SOLVED
        assert s.info()["rho"] == 0.7
        x, y, z = s.solution()
        it1 = s.info()["iters"]
        s.warm_start(x, y)
        assert s.solve() == gb.SOLVED
        assert s.info()["iters"] <= max(5, it1 // 4)


def test_device_resident_inputs_equal_host_inputs(gb):
    torch = pytest.importorskip("torch")
    qp = problem("lasso_50x2000")
    dev = torch.device("cuda:0")
    P, A = qp.P.tocsr(), qp.A.tocsr()
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    l = np.where(np.isinf(qp.l), np.sign(qp.l) * 1e20, qp.l)
    u = np.where(np.isinf(qp.u), np.sign(qp.u) * 1e20, qp.u)
    args = [t(P.indptr, torch.int64), t(P.indices, torch.int32), t(P.data, torch.float64),
            t(A.indptr, torch.int64), t(A.indices, torch.int32), t(A.data, torch.float64),
            t(qp.q, torch.float64), t(l, torch.float64), t(u, torch.float64)]
    torch.cuda.synchronize()
    h = gb.osqp_setup_device(*args, qp.n, qp.m)
    try:
        assert gb.osqp_solve(h) == gb.SOLVED
        xd = gb.osqp_get_solution(h)[0]
    finally:
        gb.osqp_cleanup(h)
    with gb.Solver(qp) as s:
        s.solve()
        xh = s.solution()[0]
    assert np.array_equal(xd, xh)


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "range", "bounds", "nan", "lower_in_upper"])
def test_invalid_inputs_are_rejected_on_device(gb, case):
    """Validation runs in device kernels; each defect gives its error code."""
    qp = qpgen.random_qp(20, 30, 1)
    l, u = qp.l.copy(), qp.u.copy()
    P_is_upper = case == "lower_in_upper"
    hp = gb._HostCsr(sp.tril(qp.P, format="csr") if P_is_upper else qp.P)
    ha = gb._HostCsr(qp.A)
    col = ha.col.copy()
    val = ha.val.copy()
    r = int(np.argmax(np.diff(ha.rowptr)))
    a0, a1 = int(ha.rowptr[r]), int(ha.rowptr[r + 1])
    code = gb.ERR_CSR
    if case == "unsorted":
        col[a0:a1] = col[a0:a1][::-1].copy()
    elif case == "duplicate":
        col[a0 + 1] = col[a0]
    elif case == "range":
        col[a0] = qp.n + 3
    elif case == "bounds":
        l[3] = u[3] + 1.0
        code = gb.ERR_BOUNDS
    elif case == "nan":
        val[a0] = np.nan
        code = gb.ERR_NONFINITE
    ha.c.colind = col.ctypes.data
    ha.c.val = val.ctypes.data
    s = gb.default_settings()
    s.P_is_upper = 1 if P_is_upper else 0
    q = np.ascontiguousarray(qp.q)
    h = gb.ctypes.c_void_p()
    rc = gb.lib().osqp_setup(gb.ctypes.byref(h), gb.ctypes.byref(hp.c), gb.ctypes.byref(ha.c), q.ctypes.data,
                             l.ctypes.data, u.ctypes.data, gb.ctypes.byref(s))
    assert rc == code, (case, rc, gb.lib().gbosqp_setup_error())
    assert not h.value


def test_dimension_mismatch_is_rejected(gb):
    qp = qpgen.random_qp(20, 30, 1)
    with pytest.raises(gb.GbosqpError) as e:
        gb.osqp_setup(qp.P, qp.A[:, :10], qp.q, qp.l, qp.u)
    assert e.value.code == gb.ERR_DIMENSION


def test_max_iter_status(gb):
    qp = problem("portfolio_3000x30")
    with gb.Solver(qp, max_iter=10) as s:
        assert s.solve() == gb.MAX_ITER
        assert s.info()["iters"] == 10


@pytest.mark.parametrize("seed", range(10))
def test_random_100x1000_fp64_ten_seeds(gb, seed):
    """The plain-method FP64 workload (n = 100, m = 1000) on seeds 0-9:
    residuals within the rule; objective within 1e-3 of the tight oracle
    where the oracle's own 1e-3 solve gets there, else within the
    convexity bound."""
    qp = qpgen.random_qp(100, 1000, seed)
    ref = admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=100000))
    own = admm.solve(qp)
    with gb.Solver(qp, precision=gb.FP64) as s:
        assert s.solve() == gb.SOLVED
        x, y, z = s.solution()
        info = s.info()
    v = checks.kkt_violation(qp, x, z, y)
    assert v.prim <= info["eps_prim"] * (1 + 1e-9) and v.dual <= info["eps_dual"] * (1 + 1e-9)
    f = admm.objective(qp.P, qp.q, x)
    bound = checks.objective_error_bound(x, y, v.prim, v.dual, ref.x, ref.y)
    assert abs(f - ref.obj) <= 1.001 * bound + 1e-12
    if abs(own.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)):
        assert abs(f - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj))
