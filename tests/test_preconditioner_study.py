"""Why the PCG keeps the Jacobi preconditioner (no GPU): on the ADMM state
after 20 iterations of the oracle's PCG form, a damped Neumann polynomial
in D^-1 K on top of Jacobi (degree 1-3, damping 1 / lambda_max(D^-1 K))
needs at least as many applications of K, counting those inside the
preconditioner and the warm start's residual, as Jacobi alone to reach the
same tolerance.  In exact arithmetic CG's iterate is already the best one in
the Krylov space of D^-1 K, so a polynomial preconditioner can only save
reductions, and the device path has no separate reduction passes to save."""
import numpy as np
import pytest

import qpgen
from oracle import admm


def _pcg_count(apply_K, b, x0, prec, eps, max_iter=2000):
    x = x0.copy()
    r = apply_K(x) - b
    applies = 1
    y = prec(r)
    p = -y
    ry = r @ y
    k = 0
    while np.max(np.abs(r)) > eps and k < max_iter:
        Kp = apply_K(p)
        applies += 1
        a = ry / (p @ Kp)
        x += a * p
        r += a * Kp
        y = prec(r)
        ry_new = r @ y
        p = -y + (ry_new / ry) * p
        ry = ry_new
        k += 1
    assert np.max(np.abs(r)) <= eps
    return applies


@pytest.mark.parametrize("name", ["random_300x3000", "lasso_50x2000", "portfolio_3000x30"])
def test_polynomial_preconditioning_costs_more_kkt_applies(name):
    qp = qpgen.by_name(name, 0)
    s = admm.Settings()
    r = admm.solve_pcg(qp, s, max_iter=20)
    x, z, y, xt = r.scaled_state
    sc = admm.ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, s.scaling_iters)
    rho = r.rho

    def K(v):
        return admm.reduced_kkt_apply(sc.P, sc.A, s.sigma, rho, v)

    b = admm.reduced_kkt_rhs(sc.q, sc.A, s.sigma, rho, x, z, y)
    dinv = 1.0 / admm.jacobi_diag(sc.P, sc.A, s.sigma, rho)
    v = np.random.default_rng(0).standard_normal(b.size)
    for _ in range(30):  # power iteration: lambda_max of D^-1 K
        v = dinv * K(v)
        lam = np.linalg.norm(v)
        v /= lam
    w = 1.0 / lam
    res0 = np.max(np.abs(K(xt) - b))
    for rel in (1e-2, 1e-4):
        eps = rel * res0
        jacobi = _pcg_count(K, b, xt, lambda t: dinv * t, eps)
        for degree in (1, 2, 3):
            inner = [0]

            def prec(t, d=degree):
                acc = dinv * t
                term = acc.copy()
                for _ in range(d):
                    term = term - w * dinv * K(term)
                    inner[0] += 1
                    acc = acc + term
                return w * acc

            outer = _pcg_count(K, b, xt, prec, eps)
            assert outer + inner[0] >= jacobi, (name, rel, degree, outer + inner[0], jacobi)
