"""Solution checks that do not run ADMM.  TEST INFRASTRUCTURE.

* ``kkt_violation``   the optimality conditions of Section 2.1,
                      eqs. (prim_feas)-(compl_slack), for a candidate (x, z, y)
* ``duality_gap``     x'Px + q'x + u'y_+ + l'y_-, zero at a primal-dual solution
                      (Lagrangian duality of the QP eq. (qp))
* ``brute_force``     the unique solution of a tiny strictly convex QP found
                      by enumerating every active set {at l, at u, free}
* ``box_qp_solution`` the closed form for diagonal P and A = diag(a), a > 0
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class KKTViolation:
    prim: float          # ||Ax - z||_inf                      (prim_feas)
    dual: float          # ||Px + q + A'y||_inf                (dual_feas)
    box: float           # max violation of l <= z <= u        (box_constr)
    compl: float         # max |min(y,0)(z-l)|, |max(y,0)(z-u)| (compl_slack);
                         # |min(y,0)| where l = -inf, |max(y,0)| where u = +inf


def kkt_violation(qp, x, z, y) -> KKTViolation:
    P, q, A, l, u = qp.P, qp.q, qp.A, qp.l, qp.u
    prim = float(np.max(np.abs(A @ x - z), initial=0.0))
    dual = float(np.max(np.abs(P @ x + q + A.T @ y), initial=0.0))
    box = float(max(np.max(l - z, initial=0.0), np.max(z - u, initial=0.0), 0.0))
    yneg = np.minimum(y, 0.0)
    ypos = np.maximum(y, 0.0)
    # with an infinite bound eq. (compl_slack) can only hold with a zero
    # multiplier on that side, so the violation there is the multiplier
    with np.errstate(invalid="ignore"):
        cl = np.where(np.isinf(l), yneg, yneg * (z - l))
        cu = np.where(np.isinf(u), ypos, ypos * (z - u))
    compl = float(max(np.max(np.abs(cl), initial=0.0), np.max(np.abs(cu), initial=0.0)))
    return KKTViolation(prim, dual, box, compl)


def objective_error_bound(x, y, r_prim, r_dual, x_star, y_star) -> float:
    """Bound on |f(x) - f*| for an iterate whose (z, y) satisfy the box and
    complementarity conditions exactly (as ADMM's projection step ensures),
    from convexity: f(x) - f* >= -||y*||_1 ||Ax - z||_inf and
    f(x) - f* <= ||Px + q + A'y||_inf ||x - x*||_1 + ||y||_1 ||Ax - z||_inf."""
    return float(max(np.sum(np.abs(y_star)), np.sum(np.abs(y))) * r_prim
                 + r_dual * np.sum(np.abs(np.asarray(x) - np.asarray(x_star))))


def duality_gap(qp, x, y) -> float:
    """Primal objective minus the dual objective at y, evaluated where the
    dual residual is dropped: x'Px + q'x + u'y_+ + l'y_-.  Infinite bounds
    paired with a zero multiplier contribute nothing."""
    P, q, l, u = qp.P, qp.q, qp.l, qp.u
    ypos = np.maximum(y, 0.0)
    yneg = np.minimum(y, 0.0)
    su = float(np.sum(np.where(ypos != 0.0, u * ypos, 0.0)))
    sl = float(np.sum(np.where(yneg != 0.0, l * yneg, 0.0)))
    return float(x @ (P @ x) + q @ x) + su + sl


def brute_force(qp, tol: float = 1e-9):
    """Solve a tiny QP with P > 0 by trying every active set.

    Each constraint is at its lower bound, at its upper bound, or free
    (rows with l = u are always active, multiplier of either sign).  For an
    active set S the equality-constrained KKT system
        [[P, A_S'], [A_S, 0]] [x; y_S] = [-q; b_S]
    is solved densely; the set is accepted when l <= Ax <= u and the
    multipliers have the signs of eq. (compl_slack): y_i <= 0 at a lower
    bound, y_i >= 0 at an upper bound.  Returns (x, y)."""
    P = np.asarray(sp.csr_matrix(qp.P).todense())
    A = np.asarray(sp.csr_matrix(qp.A).todense())
    q, l, u = qp.q, qp.l, qp.u
    n, m = P.shape[0], A.shape[0]
    choices = []
    for i in range(m):
        if l[i] == u[i]:
            choices.append(("E",))
        else:
            opts = ["F"]
            if np.isfinite(l[i]):
                opts.append("L")
            if np.isfinite(u[i]):
                opts.append("U")
            choices.append(tuple(opts))
    best = None
    for assign in itertools.product(*choices):
        S = [i for i in range(m) if assign[i] != "F"]
        b = np.array([l[i] if assign[i] in ("L", "E") else u[i] for i in S])
        k = len(S)
        K = np.zeros((n + k, n + k))
        K[:n, :n] = P
        if k:
            K[:n, n:] = A[S].T
            K[n:, :n] = A[S]
        rhs = np.concatenate([-q, b])
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        if not np.allclose(K @ sol, rhs, atol=1e-10, rtol=1e-10):
            continue
        x = sol[:n]
        y = np.zeros(m)
        y[S] = sol[n:]
        Ax = A @ x
        if np.any(Ax < l - tol) or np.any(Ax > u + tol):
            continue
        ok = True
        for i in S:
            if assign[i] == "L" and y[i] > tol:
                ok = False
            if assign[i] == "U" and y[i] < -tol:
                ok = False
        if ok:
            best = (x, y)
            break
    if best is None:
        raise RuntimeError("no active set satisfies the optimality conditions")
    return best


def box_qp_solution(pdiag, q, a, l, u):
    """min 1/2 sum p_i x_i^2 + q'x  s.t.  l_i <= a_i x_i <= u_i  (a_i > 0):
    x_i = clip(-q_i / p_i, l_i / a_i, u_i / a_i) and, from dual feasibility
    p_i x_i + q_i + a_i y_i = 0, y_i = -(p_i x_i + q_i) / a_i."""
    x = np.minimum(np.maximum(-q / pdiag, l / a), u / a)
    y = -(pdiag * x + q) / a
    return x, a * x, y
