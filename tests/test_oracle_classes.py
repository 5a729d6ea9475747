"""The QP encodings of the Control, Huber and SVM classes (Section 6.1)
checked against the problems as the paper states them: at the oracle's
solution the QP objective equals the original objective (Huber penalty,
hinge loss, quadratic control cost) and the dynamics hold (no GPU)."""
import numpy as np
import pytest

import qpgen
from oracle import admm

TIGHT = admm.Settings(eps_abs=1e-9, eps_rel=1e-9, max_iter=200000, rho_vector=True)


def huber(t, M=1.0):
    a = np.abs(t)
    return np.where(a <= M, t * t, M * (2.0 * a - M))


@pytest.mark.parametrize("seed", [0, 1])
def test_huber_encoding(seed):
    n, m = 30, 200
    qp = qpgen.huber_qp(n, m, seed)
    r = admm.solve(qp, TIGHT)
    assert r.status == "solved"
    x = r.x[:n]
    Ad = qp.A[:m, :n]
    b = qp.l[:m]
    f_orig = float(np.sum(huber(Ad @ x - b)))
    assert r.obj == pytest.approx(f_orig, rel=1e-6)
    # the Huber objective is minimised: no better x nearby
    g = np.random.default_rng(seed).standard_normal(n) * 1e-3
    assert float(np.sum(huber(Ad @ (x + g) - b))) >= f_orig - 1e-8


@pytest.mark.parametrize("seed", [0, 1])
def test_svm_encoding(seed):
    n, m = 20, 120
    qp = qpgen.svm_qp(n, m, seed)
    r = admm.solve(qp, TIGHT)
    assert r.status == "solved"
    x = r.x[:n]
    B = qp.A[:m, :n]  # rows b_i a_i'
    f_orig = float(x @ x + np.sum(np.maximum(0.0, B @ x + 1.0)))
    assert r.obj == pytest.approx(f_orig, rel=1e-6)


@pytest.mark.parametrize("seed", [0, 1])
def test_control_encoding(seed):
    nx, nu, T = 6, 3, 8
    qp = qpgen.control_qp(nx, nu, T, seed)
    r = admm.solve(qp, TIGHT)
    assert r.status == "solved"
    X = r.x[:(T + 1) * nx].reshape(T + 1, nx)
    U = r.x[(T + 1) * nx:].reshape(T, nu)
    np.testing.assert_allclose(X[0], qp.meta["x_init"], atol=1e-6)
    Qd = qp.P.diagonal()[:nx] / 2.0
    Rd = qp.P.diagonal()[(T + 1) * nx:][:nu] / 2.0
    f_orig = float(sum(X[t] @ (Qd * X[t]) for t in range(T + 1)) + sum(U[t] @ (Rd * U[t]) for t in range(T)))
    assert r.obj == pytest.approx(f_orig, rel=1e-6, abs=1e-9)
    # dynamics: the equality rows give x_{t+1} = A x_t + B u_t; check them as
    # rows of the constraint matrix evaluated at the solution
    eq = qp.l == qp.u
    assert np.max(np.abs((qp.A @ r.x)[eq] - qp.l[eq])) <= 1e-6
    assert np.all(np.abs(X) <= (1.0 + 1.0) + 1e-6)


def test_class_generators_are_deterministic():
    for f in (lambda: qpgen.control_qp(5, 2, 4, 9), lambda: qpgen.huber_qp(10, 40, 9), lambda: qpgen.svm_qp(10, 40, 9)):
        a, b = f(), f()
        assert (a.P != b.P).nnz == 0 and (a.A != b.A).nnz == 0
        assert np.array_equal(a.q, b.q) and np.array_equal(a.l, b.l) and np.array_equal(a.u, b.u)


def test_reduced_kkt_with_rho_vector_matches_full_kkt():
    """With R = diag(rho_i) of eq. (rho_vec) (1e3 rho on equality rows),
    eliminating nu from eq. (kkt) gives (P + sigma I + A'RA) x~ =
    sigma x - q + A'(R z - y): both give the same x~ and z~, and the
    matrix-free apply and the Jacobi diagonal equal their dense forms."""
    qp = qpgen.control_qp(4, 2, 5, 1)
    n, m = qp.n, qp.m
    sigma = 1e-6
    rv = admm.rho_vector(0.3, qp.l, qp.u, True)
    assert set(np.unique(rv)) == {0.3, 300.0}
    r = np.random.default_rng(0)
    x, z, y = r.standard_normal(n), r.standard_normal(m), r.standard_normal(m)
    from oracle import ldl
    F = ldl.KKTFactor(qp.P, qp.A, sigma, rv)
    sol = F.solve(np.concatenate([sigma * x - qp.q, z - y / rv]))
    Ad = qp.A.toarray()
    K = qp.P.toarray() + sigma * np.eye(n) + Ad.T @ np.diag(rv) @ Ad
    xt = np.linalg.solve(K, admm.reduced_kkt_rhs(qp.q, qp.A, sigma, rv, x, z, y))
    assert np.max(np.abs(sol[:n] - xt)) <= 1e-8 * max(1.0, np.max(np.abs(xt)))
    assert np.max(np.abs(z + (sol[n:] - y) / rv - Ad @ xt)) <= 1e-8 * max(1.0, np.max(np.abs(xt)))
    v = r.standard_normal(n)
    np.testing.assert_allclose(admm.reduced_kkt_apply(qp.P, qp.A, sigma, rv, v), K @ v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(admm.jacobi_diag(qp.P, qp.A, sigma, rv), np.diag(K), rtol=1e-13)


def test_pcg_form_with_rho_vector_reaches_direct_solution():
    qp = qpgen.control_qp(10, 5, 10, 2)
    ref = admm.solve(qp, TIGHT)
    r = admm.solve_pcg(qp, admm.Settings(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, rho_vector=True,
                                         pcg_eps_min=1e-12))
    assert r.status == "solved"
    assert abs(r.obj - ref.obj) <= 1e-5 * max(1.0, abs(ref.obj))
    scalar = admm.solve_pcg(qp, admm.Settings(eps_abs=1e-6, eps_rel=1e-6, max_iter=20000, pcg_eps_min=1e-12))
    assert r.iters < scalar.iters  # the point of eq. (rho_vec) on equality-heavy problems
