"""Pins of the oracle on the degenerate problem shapes (no GPU): a linear
program (P = 0), a problem without constraints (m = 0) and a scalar problem
(n = 1), each against its closed form, for the direct-solve ADMM and for the
PCG form of Algorithm 3.

With r_prim = 0 (no constraints) the adaptive PCG tolerance of Section 5.3.4,
lambda sqrt(||r_prim|| ||r_dual||), falls to its floor eps_min, which then
bounds the attainable accuracy; the PCG cases set eps_min below the
requested tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm
from qpgen.problems import QP


def _tight(eps=1e-10, eps_min=1e-13):
    s = admm.Settings(eps_abs=eps, eps_rel=eps, max_iter=100000, check_every=1)
    s.pcg_eps_min = eps_min
    return s


def _box_lp(n, seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n)
    l = -rng.uniform(0.5, 2.0, n)
    u = rng.uniform(0.5, 2.0, n)
    return QP(sp.csr_matrix((n, n)), q, sp.identity(n, format="csr"), l, u, name="box_lp")


@pytest.mark.parametrize("form", ["direct", "pcg"])
def test_box_lp_reaches_the_vertex(form):
    """min q'x over l <= x <= u: x_i = l_i where q_i > 0 and u_i where
    q_i < 0; dual feasibility q + y = 0 gives y = -q."""
    qp = _box_lp(30, 0)
    solve = admm.solve if form == "direct" else admm.solve_pcg
    r = solve(qp, _tight(1e-9))
    assert r.status == "solved"
    x_star = np.where(qp.q > 0, qp.l, qp.u)
    assert np.max(np.abs(r.x - x_star)) <= 1e-7
    assert np.max(np.abs(r.y + qp.q)) <= 1e-7
    assert r.obj == pytest.approx(float(qp.q @ x_star), abs=1e-6)


@pytest.mark.parametrize("form", ["direct", "pcg"])
def test_no_constraints_is_a_linear_solve(form):
    rng = np.random.default_rng(1)
    n = 25
    M = rng.standard_normal((n, n))
    P = sp.csr_matrix(M @ M.T + np.eye(n))
    q = rng.standard_normal(n)
    qp = QP(P, q, sp.csr_matrix((0, n)), np.zeros(0), np.zeros(0), name="free")
    solve = admm.solve if form == "direct" else admm.solve_pcg
    r = solve(qp, _tight(1e-10))
    assert r.status == "solved"
    assert r.y.shape == (0,) and r.z.shape == (0,)
    x_star = np.linalg.solve(P.toarray(), -q)
    assert np.max(np.abs(r.x - x_star)) <= 1e-8 * max(1.0, np.max(np.abs(x_star)))


@pytest.mark.parametrize("q0,l0,u0", [(-3.0, -1.0, 1.0), (0.5, -1.0, 1.0), (8.0, -1.0, 1.0), (2.0, 0.7, 0.7)])
def test_scalar_problem(q0, l0, u0):
    """min p x^2 / 2 + q x subject to l <= a x <= u, with p = 2 and a = 0.5:
    x = clip(-q / p, l / a, u / a), y = -(p x + q) / a."""
    p, a = 2.0, 0.5
    qp = QP(sp.csr_matrix([[p]]), np.array([q0]), sp.csr_matrix([[a]]), np.array([l0]), np.array([u0]))
    x_star = min(max(-q0 / p, l0 / a), u0 / a)
    y_star = -(p * x_star + q0) / a
    for solve in (admm.solve, admm.solve_pcg):
        r = solve(qp, _tight(1e-11))
        assert r.status == "solved"
        assert abs(r.x[0] - x_star) <= 1e-9 and abs(r.y[0] - y_star) <= 1e-8
