"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(no GPU).  Each test checks the oracle against something other than itself:
values printed in the paper, closed forms, brute force, a textbook dense
solve, invariants.  A few tests plant a mistake in the oracle and check that
a pin catches it."""
import numpy as np
import pytest
import scipy.sparse as sp

import qpgen
from oracle import admm, checks, formats, ldl, mlp
from tests.conftest import read_golden


# ---------------------------------------------------------------- formats --

def test_worked_example_formats():
    """COO / CSR / CSC arrays of the 4x5 example (Section 4.3)."""
    g = read_golden("worked_example_4x5.txt")
    M = np.array([g[f"matrix_row{i}"] for i in range(4)])
    v, ri, ci = formats.coo_from_dense(M)
    assert v.tolist() == g["coo_value"]
    assert ri.tolist() == g["coo_row_index"]
    assert ci.tolist() == g["coo_column_index"]
    v, rp, ci = formats.csr_from_dense(M)
    assert v.tolist() == g["csr_value"]
    assert rp.tolist() == g["csr_row_pointer"]
    assert ci.tolist() == g["csr_column_index"]
    cv, cr, cp = formats.csc_from_dense(M)
    assert cv.tolist() == g["csc_value"]
    assert cr.tolist() == g["csc_row_index"]
    assert cp.tolist() == g["csc_column_pointer"]
    # CSC of A read as CSR of A' (Section 4.3.3)
    tv, tp, tc = formats.csr_of_transpose(4, 5, v, rp, ci)
    assert tv.tolist() == g["csc_value"]
    assert tp.tolist() == g["csc_column_pointer"]
    assert tc.tolist() == g["csc_row_index"]
    # RowIndex recovered from RowPointer (Section 5.4.3)
    assert formats.row_index_from_row_pointer(rp).tolist() == g["coo_row_index"]


def test_transpose_matches_scipy_on_random():
    A = qpgen.problems.sparse_normal(3, "t", 37, 23, 0.2)
    tv, tp, tc = formats.csr_of_transpose(37, 23, A.data, A.indptr, A.indices)
    T = A.T.tocsr()
    T.sort_indices()
    assert np.array_equal(tp, T.indptr)
    assert np.array_equal(tc, T.indices)
    assert np.array_equal(tv, T.data)


# -------------------------------------------------------------------- LDL --

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kkt_ldl_matches_dense_solve(seed):
    qp = qpgen.random_qp(30, 60, seed)
    F = ldl.KKTFactor(qp.P, qp.A, 1e-6, 0.37)
    K = F.K.toarray()
    rhs = np.random.default_rng(seed).standard_normal(90)
    sol = F.solve(rhs)
    ref = np.linalg.solve(K, rhs)
    assert np.max(np.abs(sol - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))


def test_ldl_factor_reconstructs_matrix():
    qp = qpgen.lasso_qp(8, 40, 0)
    F = ldl.KKTFactor(qp.P, qp.A, 1e-6, 0.1)
    f = F.ldl
    n = f.n
    L = sp.csc_matrix((f.Lx[:f.nnzL], f.Li[:f.nnzL], f.Lp), shape=(n, n)).toarray() + np.eye(n)
    Kp = F.K.toarray()[np.ix_(f.perm, f.perm)]
    assert np.max(np.abs(L @ np.diag(f.D[:n]) @ L.T - Kp)) <= 1e-10 * np.max(np.abs(Kp))


# ------------------------------------------------ solutions: brute force --

@pytest.mark.parametrize("seed,n,m,neq,ninf", [(0, 3, 5, 0, 0), (1, 4, 7, 1, 2), (2, 5, 8, 2, 3),
                                               (3, 2, 6, 0, 4), (4, 5, 6, 1, 1)])
def test_oracle_matches_brute_force(seed, n, m, neq, ninf):
    qp = qpgen.tiny_qp(n, m, seed, n_eq=neq, n_inf=ninf)
    xb, yb = checks.brute_force(qp)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-11, eps_rel=1e-11, max_iter=50000, check_every=1))
    assert r.status == "solved"
    assert np.max(np.abs(r.x - xb)) <= 1e-8
    assert np.max(np.abs(r.y - yb)) <= 1e-7


@pytest.mark.parametrize("seed,scale_a", [(0, False), (1, True), (2, True)])
def test_oracle_matches_box_closed_form(seed, scale_a):
    qp = qpgen.box_qp(40, seed, with_inf=True, scale_a=scale_a)
    pd = qp.P.diagonal()
    a = qp.A.diagonal()
    xs, zs, ys = checks.box_qp_solution(pd, qp.q, a, qp.l, qp.u)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-11, eps_rel=1e-11, max_iter=50000, check_every=1))
    assert np.max(np.abs(r.x - xs)) <= 1e-8
    assert np.max(np.abs(r.y - ys)) <= 1e-7
    r2 = admm.solve_pcg(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=20000))
    assert np.max(np.abs(r2.x - xs)) <= 1e-6


def test_unconstrained_reduces_to_linear_solve():
    qp = qpgen.random_qp(25, 40, 5)
    qp.l[:] = -np.inf
    qp.u[:] = np.inf
    x_ref = np.linalg.solve(qp.P.toarray(), -qp.q)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-11, eps_rel=1e-11, max_iter=50000, check_every=1))
    assert np.max(np.abs(r.x - x_ref)) <= 1e-8 * max(1, np.max(np.abs(x_ref)))
    assert np.max(np.abs(r.y)) <= 1e-8


def test_equality_only_reduces_to_kkt_solve():
    qp = qpgen.equality_qp(30, 12, 2)
    n, m = qp.n, qp.m
    K = np.block([[qp.P.toarray(), qp.A.toarray().T], [qp.A.toarray(), np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([-qp.q, qp.l]))
    r = admm.solve(qp, admm.Settings(eps_abs=1e-11, eps_rel=1e-11, max_iter=50000, check_every=1))
    assert np.max(np.abs(r.x - sol[:n])) <= 1e-7 * max(1, np.max(np.abs(sol[:n])))
    assert np.max(np.abs(r.y - sol[n:])) <= 1e-6 * max(1, np.max(np.abs(sol[n:])))


def test_kkt_conditions_and_gap_on_tight_solution():
    qp = qpgen.random_qp(100, 1000, 0)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-10, eps_rel=1e-10, max_iter=50000, check_every=5))
    v = checks.kkt_violation(qp, r.x, r.z, r.y)
    # box feasibility holds exactly in scaled space; unscaling costs an ulp
    assert v.prim <= 1e-8 and v.dual <= 1e-8 and v.box <= 1e-14 and v.compl <= 1e-8
    assert abs(checks.duality_gap(qp, r.x, r.y)) <= 1e-7


# ------------------------------------------------------------------- PCG --

def _dense_reduced(P, A, sigma, rho):
    return P.toarray() + sigma * np.eye(P.shape[0]) + rho * (A.T @ A).toarray()


def test_pcg_equals_dense_solve_and_terminates_in_n_steps():
    qp = qpgen.random_qp(30, 90, 7)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u)
    sigma, rho = 1e-6, 0.3
    K = _dense_reduced(sc.P, sc.A, sigma, rho)
    b = np.random.default_rng(1).standard_normal(30)
    Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, sigma, rho)
    out = admm.pcg(lambda v: admm.reduced_kkt_apply(sc.P, sc.A, sigma, rho, v), b, np.zeros(30),
                   Minv, 1e-12, 200, keep_directions=True)
    assert out.iters <= 30
    ref = np.linalg.solve(K, b)
    assert np.max(np.abs(out.x - ref)) <= 1e-9 * max(1, np.max(np.abs(ref)))
    # conjugacy p_i' K p_j = 0 for i != j (Section 4.1.1); in floating point
    # it decays once the residual is small, so the first 15 directions
    ps = [p for p, _ in out.directions][:15]
    Kps = [kp for _, kp in out.directions][:15]
    for i in range(len(ps)):
        for j in range(i):
            assert abs(ps[i] @ Kps[j]) <= 1e-11 * np.sqrt((ps[i] @ Kps[i]) * (ps[j] @ Kps[j]))


def test_reduced_kkt_matches_full_kkt():
    """Eliminating nu from eq. (kkt) gives eq. (kkt_red): both give the same
    x~ and z~ (Section 4)."""
    qp = qpgen.random_qp(20, 50, 3)
    sigma, rho = 1e-6, 0.5
    x = np.random.default_rng(0).standard_normal(20)
    z = np.random.default_rng(1).standard_normal(50)
    y = np.random.default_rng(2).standard_normal(50)
    F = ldl.KKTFactor(qp.P, qp.A, sigma, rho)
    sol = F.solve(np.concatenate([sigma * x - qp.q, z - y / rho]))
    xt_full = sol[:20]
    zt_full = z + (sol[20:] - y) / rho
    K = _dense_reduced(qp.P, qp.A, sigma, rho)
    xt_red = np.linalg.solve(K, admm.reduced_kkt_rhs(qp.q, qp.A, sigma, rho, x, z, y))
    assert np.max(np.abs(xt_full - xt_red)) <= 1e-9
    assert np.max(np.abs(zt_full - qp.A @ xt_red)) <= 1e-9


def test_jacobi_diag_identity():
    qp = qpgen.random_qp(15, 40, 4)
    d = admm.jacobi_diag(qp.P, qp.A, 1e-6, 2.0)
    dense = np.diag(_dense_reduced(qp.P, qp.A, 1e-6, 2.0))
    assert np.max(np.abs(d - dense)) <= 1e-12 * np.max(np.abs(dense))


# ------------------------------------------------------------------ Ruiz --

def test_ruiz_definitions_and_equilibration():
    qp = qpgen.random_qp(40, 120, 9)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, iters=60)
    D, E, c = sc.D, sc.E, sc.c
    # scaled data equal their definitions (Section 3.3)
    assert np.allclose(sc.P.toarray(), c * np.diag(D) @ qp.P.toarray() @ np.diag(D), rtol=1e-12, atol=1e-14)
    assert np.allclose(sc.A.toarray(), np.diag(E) @ qp.A.toarray() @ np.diag(D), rtol=1e-12, atol=1e-14)
    assert np.allclose(sc.q, c * D * qp.q, rtol=1e-12)
    assert np.allclose(sc.l, E * qp.l) and np.allclose(sc.u, E * qp.u)
    # after many passes Algorithm 2 is at its fixed point: delta = 1, i.e.
    # the columns of [[P_bar, A_bar'],[A_bar, 0]] have unit inf-norm, and
    # gamma = 1, i.e. max(mean column norm of P_bar, ||q_bar||) = 1
    M = sp.bmat([[sc.P, sc.A.T], [sc.A, None]]).toarray()
    cn = np.max(np.abs(M), axis=0)
    assert np.max(np.abs(cn - 1.0)) <= 1e-9
    gam = max(np.mean(np.max(np.abs(sc.P.toarray()), axis=0)), np.max(np.abs(sc.q)))
    assert abs(gam - 1.0) <= 1e-9
    # unscale(scale(v)) = v
    xb = np.random.default_rng(0).standard_normal(40)
    x, z, y = admm.unscale(sc, xb, sc.A @ xb, np.ones(120))
    assert np.allclose(x / D, xb) and np.allclose(z * E, sc.A @ xb) and np.allclose(y * c / E, 1.0)


def test_ruiz_scaled_problem_has_same_solution():
    """The scaled QP's optimum divided by c equals the original optimum; the
    optima are found by brute force, independently of ADMM."""
    qp = qpgen.tiny_qp(4, 6, 11, n_eq=1, n_inf=1)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, iters=10)
    scaled = qpgen.QP(sc.P, sc.q, sc.A, sc.l, sc.u)
    x, _ = checks.brute_force(qp)
    xb, _ = checks.brute_force(scaled)
    f = admm.objective(qp.P, qp.q, x)
    fb = admm.objective(sc.P, sc.q, xb)
    assert abs(fb / sc.c - f) <= 1e-10 * max(1, abs(f))
    assert np.allclose(sc.D * xb, x, atol=1e-10)


# ---------------------------------------------------- PCG-ADMM vs direct --

@pytest.mark.parametrize("name", ["random_100x1000", "lasso_50x2000", "random_300x3000"])
def test_pcg_admm_reaches_direct_solution(name):
    qp = qpgen.by_name(name, 0)
    tight = admm.solve(qp, admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=50000))
    r = admm.solve_pcg(qp, admm.Settings(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000))
    assert r.status == "solved"
    assert abs(r.obj - tight.obj) <= 1e-5 * max(1.0, abs(tight.obj))


# --------------------------------------------------------------- planted --

def test_planted_wrong_dual_sign_is_caught(monkeypatch):
    """A sign error in the dual update (Algorithm 1, step 7) must break the
    brute-force pin."""
    qp = qpgen.tiny_qp(3, 5, 0)
    xb, _ = checks.brute_force(qp)

    def bad_update(xt, zt, x, z, y, alpha, rho, l, u):
        x_new = alpha * xt + (1.0 - alpha) * x
        zr = alpha * zt + (1.0 - alpha) * z
        z_new = admm.project_box(zr + y / rho, l, u)
        return x_new, z_new, y - rho * (zr - z_new)

    monkeypatch.setattr(admm, "admm_update", bad_update)
    r = admm.solve(qp, admm.Settings(eps_abs=1e-11, eps_rel=1e-11, max_iter=3000, check_every=1))
    assert not (r.status == "solved" and np.max(np.abs(r.x - xb)) <= 1e-8)


def test_planted_dropped_sigma_term_is_caught(monkeypatch):
    """Dropping sigma x from the matrix-free K-apply must break the dense-solve
    pin of PCG."""
    qp = qpgen.random_qp(10, 5, 1)  # m < n: A'A is singular, sigma matters
    sigma, rho = 1e-1, 0.3
    K = _dense_reduced(qp.P * 0.0, qp.A, sigma, rho)
    b = np.ones(10)

    def bad_apply(P, A, s, r, x):
        return P @ x + A.T @ (r * (A @ x))

    out = admm.pcg(lambda v: bad_apply(qp.P * 0.0, qp.A, sigma, rho, v), b, np.zeros(10),
                   np.ones(10), 1e-12, 100)
    assert np.max(np.abs(out.x - np.linalg.solve(K, b))) > 1e-6


def test_planted_transposed_scaling_is_caught():
    """Using D where E belongs (A_bar = D A E) must break the Ruiz definition
    pin."""
    qp = qpgen.random_qp(12, 12, 2)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, iters=5)
    wrong = np.diag(sc.D) @ qp.A.toarray() @ np.diag(sc.E)
    assert not np.allclose(sc.A.toarray(), wrong, rtol=1e-6)


# ------------------------------------------------------------------- MLP --

def _mlp_params(seed=0):
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal(s) * (0.5 if k.startswith("W") else 0.1)
            for k, s in mlp.PARAM_SHAPES.items()}


def test_mlp_gradients_match_finite_differences():
    p = _mlp_params(0)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((16, 4))
    T = rng.standard_normal((16, 2))
    W = np.ones((16, 2))
    W[::3, 1] = 0.0
    _, g = mlp.grads(p, X, T, W)
    h = 1e-6
    for k, v in p.items():
        flat = v.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 17)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss_fn(p, X, T, W)
            flat[idx] = old - h
            lm = mlp.loss_fn(p, X, T, W)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_bf16_round_known_values():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.0e38, -2.5, 0.1])
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to even (1.0);
    # 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    expect = np.array([1.0, 1.0, 1.0078125, 2.0**127 * 226 / 128, -2.5, 0.10009765625])
    got = mlp.bf16_round(vals)
    assert np.allclose(got, expect, rtol=1e-7)


# -------------------------------------------------------------- inputs ---

def test_generators_are_deterministic_and_shaped():
    a = qpgen.random_qp(100, 1000, 0)
    b = qpgen.random_qp(100, 1000, 0)
    c = qpgen.random_qp(100, 1000, 1)
    assert np.array_equal(a.A.data, b.A.data) and np.array_equal(a.A.indices, b.A.indices)
    assert not np.array_equal(a.q, c.q)
    dens = a.A.nnz / (1000 * 100)
    assert abs(dens - 0.15) < 0.01
    assert np.all(a.l <= 0) and np.all(a.u >= 0)
    assert abs(a.P - a.P.T).max() == 0.0
    las = qpgen.lasso_qp(20, 300, 0)
    assert las.n == 20 + 300 + 20 and las.m == 300 + 40
    por = qpgen.portfolio_qp(200, 5, 0)
    assert por.n == 205 and por.m == 5 + 1 + 200


def test_bf16_gradient_variant_reduces_to_exact_without_rounding(monkeypatch):
    """With BF16 rounding replaced by the identity, the BF16-emulating
    forward/backward equals the exact one (which finite differences pin)."""
    p = _mlp_params(3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((20, 4))
    T = rng.standard_normal((20, 2))
    W = np.ones((20, 2))
    monkeypatch.setattr(mlp, "bf16_round", lambda a: np.asarray(a, np.float64))
    l1, g1, _ = mlp.grads_bf16(p, X, T, W)
    l2, g2 = mlp.grads(p, X, T, W)
    assert abs(l1 - l2) <= 1e-14 * max(1.0, abs(l2))
    for k in g2:
        assert np.allclose(g1[k], g2[k], rtol=1e-12, atol=1e-14)


# ------------------------------------------------- dense Schur-complement solve --

def test_schur_matrix_is_p_plus_sigma_plus_atra():
    """oracle.dense.schur_matrix against the dense product written out."""
    from oracle import dense
    rng = np.random.default_rng(11)
    qp = qpgen.random_qp(40, 300, 2)
    r = rng.uniform(0.1, 10.0, qp.m)
    S = dense.schur_matrix(qp.P, qp.A, 1e-3, r)
    Ad = qp.A.toarray()
    ref = qp.P.toarray() + 1e-3 * np.eye(qp.n) + Ad.T @ (r[:, None] * Ad)
    assert np.max(np.abs(S - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_dense_schur_solve_equals_sparse_ldl():
    """Both factors solve eq. (kkt) for the same right-hand side to 1e-10, on
    a mid-size random QP after Ruiz scaling, for a scalar rho and a rho
    vector."""
    from oracle import dense, ldl
    qp = qpgen.by_name("random_300x3000", 0)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, 10)
    rng = np.random.default_rng(12)
    rhs = rng.standard_normal(qp.n + qp.m)
    for rho in (0.1, admm.rho_vector(0.1, sc.l, sc.u, True), 7.0):
        a = ldl.KKTFactor(sc.P, sc.A, 1e-6, rho).solve(rhs)
        F = dense.DenseSchurFactor(sc.P, sc.A, 1e-6, rho)
        b = F.solve(rhs)
        assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(a))
        assert F.max_rel_residual <= 1e-12


def test_oracle_solve_same_with_either_factor():
    """The direct ADMM takes the same path with either factor: the same
    iteration count and rho history, and iterates equal to 1e-8."""
    qp = qpgen.by_name("random_300x3000", 0)
    a = admm.solve(qp, admm.Settings(kkt="sparse"))
    b = admm.solve(qp, admm.Settings(kkt="dense"))
    assert a.status == b.status == "solved" and a.iters == b.iters
    assert np.allclose(a.rho_history, b.rho_history, rtol=1e-12)
    assert np.max(np.abs(a.x - b.x)) <= 1e-8 * max(1.0, np.max(np.abs(a.x)))
    assert abs(a.obj - b.obj) <= 1e-9 * max(1.0, abs(a.obj))


# ------------------------------------------------ single-reduction PCG --

@pytest.mark.parametrize("name", ["random_100x1000", "lasso_50x2000", "portfolio_3000x30"])
def test_single_reduction_pcg_has_the_iterates_of_algorithm3(name):
    """In exact arithmetic the single-reduction rearrangement produces the
    iterates of Algorithm 3: in FP64 the first 5 steps agree to 1e-10 and the
    residual norms likewise, on the reduced KKT systems of three families."""
    qp = qpgen.by_name(name, 0)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, 10)
    rng = np.random.default_rng(21)
    b = rng.standard_normal(qp.n)
    x0 = 0.1 * rng.standard_normal(qp.n)
    for rho in (0.1, 4.0):
        Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, 1e-6, rho)
        K = lambda v: admm.reduced_kkt_apply(sc.P, sc.A, 1e-6, rho, v)  # noqa: E731
        for k in range(1, 6):
            a = admm.pcg(K, b, x0, Minv, 0.0, k)
            g = admm.pcg_single_reduction(K, b, x0, Minv, 0.0, k)
            assert a.iters == g.iters == k
            assert np.max(np.abs(a.x - g.x)) <= 1e-10 * max(1.0, np.max(np.abs(a.x))), (rho, k)
            assert abs(a.r_norm - g.r_norm) <= 1e-10 * max(1.0, a.r_norm)


def test_single_reduction_pcg_solves_and_stops_like_algorithm3():
    """Run to a tolerance: the same number of steps on a well-conditioned
    system, the stopping rule ||r||_inf <= eps on both, and a solution equal
    to the dense solve within what that residual allows; a zero step budget
    or an exact start returns at once."""
    qp = qpgen.by_name("random_100x1000", 0)
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, 10)
    rho = 0.5
    Minv = 1.0 / admm.jacobi_diag(sc.P, sc.A, 1e-6, rho)
    K = lambda v: admm.reduced_kkt_apply(sc.P, sc.A, 1e-6, rho, v)  # noqa: E731
    b = np.random.default_rng(22).standard_normal(qp.n)
    Kd = (sc.P + 1e-6 * sp.identity(qp.n) + rho * (sc.A.T @ sc.A)).toarray()
    xs = np.linalg.solve(Kd, b)
    a = admm.pcg(K, b, np.zeros(qp.n), Minv, 1e-8, 500)
    g = admm.pcg_single_reduction(K, b, np.zeros(qp.n), Minv, 1e-8, 500)
    assert g.r_norm <= 1e-8 and a.r_norm <= 1e-8 and g.iters == a.iters
    assert np.max(np.abs(g.x - xs)) <= 1e-8 * np.max(np.abs(np.linalg.inv(Kd)).sum(axis=1))
    assert admm.pcg_single_reduction(K, b, np.zeros(qp.n), Minv, 0.0, 0).iters == 0
    assert admm.pcg_single_reduction(K, b, xs, Minv, 1e-8, 50).iters == 0


def test_single_reduction_admm_follows_the_classic_path():
    """Algorithm 1 with either PCG takes the same PCG step counts for 20
    iterations on a small random QP and reaches the same iterates."""
    qp = qpgen.by_name("random_100x1000", 0)
    a = admm.solve_pcg(qp, admm.Settings(), max_iter=20)
    g = admm.solve_pcg(qp, admm.Settings(pcg_variant="single_reduction"), max_iter=20)
    assert a.pcg_per_iter == g.pcg_per_iter
    for u, v in zip(a.scaled_state, g.scaled_state):
        assert np.max(np.abs(u - v)) <= 1e-8 * max(1.0, np.max(np.abs(u)))
