"""FP64 CPU restatement of the paper's ADMM QP method.  TEST INFRASTRUCTURE.

Two solvers share the step functions below:

* ``solve``      Algorithm 1 (OSQP) with the direct LDL' solve of the KKT
                 system eq. (kkt) (Section 3.2): the ground-truth solution.
* ``solve_pcg``  Algorithm 1 with the reduced KKT system eq. (kkt_red_sc)
                 solved by warm-started Jacobi-PCG (Algorithm 3) with the
                 residual-based tolerance of Section 5.3.4, R = rho I,
                 termination checked every 5 and rho adapted every 10
                 iterations (Table 1): the GPU algorithm, run on the CPU in
                 FP64, for trajectory-level comparison.

Readings of points the paper leaves open (each is listed with its reason in
the design notes):
  S1  eps_prim = eps_abs + eps_rel max(||Ax||, ||z||),
      eps_dual = eps_abs + eps_rel max(||Px||, ||A'y||, ||q||), inf-norms of
      unscaled quantities (OSQP's rule, reference Stellato 2020).
  S2  rho <- rho sqrt((||r_p|| / max(||Ax||, ||z||)) /
                      (||r_d|| / max(||Px||, ||A'y||, ||q||)))
      on scaled quantities, clamped to [1e-6, 1e6]; a zero normaliser or a
      zero dual residual means no update.
  S3  PCG stops when ||r||_inf <= eps (absolute test, inf-norm).
  S4  Ruiz: a fixed number of passes; the scaling is applied incrementally
      so that P_bar = c D P D holds after every pass; a norm below 1e-4 is
      taken as 1 and a norm above 1e4 as 1e4 (for D, E and the cost scale).
  S5  before the first termination check the PCG tolerance is
      max(lambda ||q_bar||_inf, eps_min).
  S6  cold start x = z = y = 0, rho_0 = 0.1.
  S7  PCG step length alpha = r'y / p'Kp (Algorithm 3 prints a minus sign
      that contradicts Section 4.1.1 and the cited Nocedal & Wright).
  S17 infeasibility tests (Section 3.1, approximate forms of eqs.
      (prim_infeas) and (dual_infeas)) run at every termination check that
      does not find convergence, on dx = x^k - x^(k-1), dy = y^k - y^(k-1)
      (unscaled).  Each candidate is scaled to unit inf-norm first: the
      printed absolute form holds for every converging sequence, whose
      differences go to zero.  The strict inequalities of the certificates
      are tested with the margin on the safe side (< -eps, not < eps), so a
      solvable problem whose iterates drift along a null direction is not
      reported infeasible.  dy is projected first onto the cone on which
      the support function of [l, u] is finite (a component that faces an
      infinite bound is clipped to zero).  eps_pinf = eps_dinf = 1e-4.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .ldl import KKTFactor

MIN_SCALING = 1e-4
MAX_SCALING = 1e4
RHO_MIN = 1e-6
RHO_MAX = 1e6


@dataclass
class Settings:
    sigma: float = 1e-6          # Section 3.4 default
    alpha: float = 1.6           # Section 3.4 default
    rho0: float = 0.1
    eps_abs: float = 1e-3
    eps_rel: float = 1e-3
    max_iter: int = 4000
    scaling_iters: int = 10
    check_every: int = 5         # Table 1 (cuOSQP)
    rho_every: int = 10          # Section 5.3.3
    adaptive_rho: bool = True
    rho_vector: bool = False     # eq. (rho_vec): 1e3 rho on equality rows
    refactor_ratio: float = 5.0  # direct solver only: refactor on a 5x change
    kkt: str = "auto"            # direct solver: "sparse" LDL' of eq. (kkt), "dense" Schur
                                 # complement (oracle/dense.py), "auto": dense for n >= 2000, m >= 4n
    pcg_lambda: float = 0.15     # Section 5.3.4
    pcg_eps_min: float = 1e-7    # Section 5.3.4
    max_cg_iter: int = 50
    pcg_variant: str = "classic"  # solve_pcg: "classic" Algorithm 3 or "single_reduction"
    eps_prim_inf: float = 1e-4   # S17
    eps_dual_inf: float = 1e-4   # S17


def norm_inf(v) -> float:
    v = np.asarray(v)
    return float(np.max(np.abs(v))) if v.size else 0.0


# --------------------------------------------------------------------------
# Ruiz equilibration, Algorithm 2
# --------------------------------------------------------------------------

def limit_scaling(v):
    """Norms below 1e-4 are replaced by 1, norms above 1e4 by 1e4 (S4)."""
    v = np.asarray(v, np.float64)
    out = np.where(v < MIN_SCALING, 1.0, v)
    return np.minimum(out, MAX_SCALING)


def col_inf_norms(M: sp.spmatrix) -> np.ndarray:
    M = sp.csc_matrix(M)
    out = np.zeros(M.shape[1])
    for j in range(M.shape[1]):
        seg = M.data[M.indptr[j]:M.indptr[j + 1]]
        if seg.size:
            out[j] = np.max(np.abs(seg))
    return out


def row_inf_norms(M: sp.spmatrix) -> np.ndarray:
    return col_inf_norms(sp.csr_matrix(M).T)


@dataclass
class Scaling:
    D: np.ndarray
    E: np.ndarray
    c: float
    P: sp.csr_matrix
    q: np.ndarray
    A: sp.csr_matrix
    l: np.ndarray
    u: np.ndarray


def ruiz(P, q, A, l, u, iters: int = 10) -> Scaling:
    """Algorithm 2: D, E, c such that P_bar = c D P D, q_bar = c D q,
    A_bar = E A D, l_bar = E l, u_bar = E u."""
    P = sp.csr_matrix(P, dtype=np.float64)
    A = sp.csr_matrix(A, dtype=np.float64)
    n, m = P.shape[0], A.shape[0]
    D = np.ones(n)
    E = np.ones(m)
    c = 1.0
    Pb, qb, Ab = P.copy(), np.asarray(q, np.float64).copy(), A.copy()
    for _ in range(iters):
        # column inf-norms of M = [[P_bar, A_bar'], [A_bar, 0]]
        norm_x = np.maximum(col_inf_norms(Pb), col_inf_norms(Ab)) if n else np.zeros(0)
        norm_z = row_inf_norms(Ab) if m else np.zeros(0)
        dx = 1.0 / np.sqrt(limit_scaling(norm_x))
        dz = 1.0 / np.sqrt(limit_scaling(norm_z))
        D = D * dx
        E = E * dz
        Pb = sp.csr_matrix(sp.diags(dx) @ Pb @ sp.diags(dx))
        qb = dx * qb
        Ab = sp.csr_matrix(sp.diags(dz) @ Ab @ sp.diags(dx))
        # cost scaling
        mean_p = float(np.mean(col_inf_norms(Pb))) if n else 0.0
        gamma = 1.0 / float(limit_scaling(max(mean_p, norm_inf(qb))))
        Pb = Pb * gamma
        qb = qb * gamma
        c = c * gamma
    lb = np.where(np.isinf(l), l, E * l)
    ub = np.where(np.isinf(u), u, E * u)
    return Scaling(D, E, c, Pb, qb, Ab, lb, ub)


def unscale(sc: Scaling, x_bar, z_bar, y_bar):
    """x = D x_bar, z = E^{-1} z_bar, y = E y_bar / c (Section 3.3)."""
    return sc.D * x_bar, z_bar / sc.E, sc.E * y_bar / sc.c


# --------------------------------------------------------------------------
# ADMM pieces, Algorithm 1 and Section 3.1
# --------------------------------------------------------------------------

def project_box(v, l, u):
    """Euclidean projection onto [l, u]: min(max(v, l), u) (Section 3)."""
    return np.minimum(np.maximum(v, l), u)


def admm_update(xt, zt, x, z, y, alpha, rho, l, u):
    """Steps 5-7 of Algorithm 1 (relaxation, projection, dual update)."""
    x_new = alpha * xt + (1.0 - alpha) * x
    zr = alpha * zt + (1.0 - alpha) * z
    z_new = project_box(zr + y / rho, l, u)
    y_new = y + rho * (zr - z_new)
    return x_new, z_new, y_new


@dataclass
class Residuals:
    r_prim: float
    r_dual: float
    eps_prim: float
    eps_dual: float
    norm_Ax: float
    norm_z: float
    norm_Px: float
    norm_Aty: float
    norm_q: float

    def converged(self) -> bool:
        return self.r_prim <= self.eps_prim and self.r_dual <= self.eps_dual


def residuals(P, q, A, x, z, y, eps_abs=1e-3, eps_rel=1e-3) -> Residuals:
    """r_prim = Ax - z, r_dual = Px + q + A'y (Section 3.1), inf-norms, and
    the tolerances of reading S1."""
    Ax = A @ x
    Px = P @ x
    Aty = A.T @ y
    rp = norm_inf(Ax - z)
    rd = norm_inf(Px + q + Aty)
    nAx, nz, nPx, nAty, nq = norm_inf(Ax), norm_inf(z), norm_inf(Px), norm_inf(Aty), norm_inf(q)
    return Residuals(rp, rd, eps_abs + eps_rel * max(nAx, nz),
                     eps_abs + eps_rel * max(nPx, nAty, nq), nAx, nz, nPx, nAty, nq)


def rho_ratio_rule(rho: float, scaled: Residuals) -> float:
    """Reading S2 of the residual-ratio rule (Section 3.4)."""
    prim_norm = max(scaled.norm_Ax, scaled.norm_z)
    dual_norm = max(scaled.norm_Px, scaled.norm_Aty, scaled.norm_q)
    if prim_norm <= 0.0 or dual_norm <= 0.0 or scaled.r_dual <= 0.0:
        return rho
    ratio = (scaled.r_prim / prim_norm) / (scaled.r_dual / dual_norm)
    if not math.isfinite(ratio):
        return rho
    return float(min(max(rho * math.sqrt(ratio), RHO_MIN), RHO_MAX))


def rho_vector(rho: float, l, u, use_vector: bool):
    """R = rho I, or OSQP's eq. (rho_vec): 1e3 rho on rows with l_i = u_i."""
    if not use_vector:
        return np.full(len(l), rho)
    return np.where(l == u, 1e3 * rho, rho)


def objective(P, q, x) -> float:
    return float(0.5 * x @ (P @ x) + q @ x)


# --------------------------------------------------------------------------
# Infeasibility detection, Section 3.1 (reading S17)
# --------------------------------------------------------------------------

INF_BOUND = 1e20  # a bound with |v| >= 1e20 is infinite


def primal_infeasibility(A, l, u, dy, eps):
    """Approximate certificate test of eq. (prim_infeas) on dy.

    dy is clipped to the cone where the support function
    u'(y)_+ + l'(y)_- of the box [l, u] is finite (y_i <= 0 where u_i is
    infinite, y_i >= 0 where l_i is infinite), scaled to unit inf-norm, and
    accepted when ||A'y||_inf <= eps and u'(y)_+ + l'(y)_- < -eps.
    Returns the scaled certificate, or None."""
    l = np.asarray(l, np.float64)
    u = np.asarray(u, np.float64)
    y = np.array(dy, np.float64, copy=True)
    u_inf = u >= INF_BOUND
    l_inf = l <= -INF_BOUND
    y[u_inf] = np.minimum(y[u_inf], 0.0)
    y[l_inf] = np.maximum(y[l_inf], 0.0)
    nrm = norm_inf(y)
    if not (nrm > 0.0 and math.isfinite(nrm)):
        return None
    y /= nrm
    pos, neg = y > 0.0, y < 0.0
    support = float(u[pos] @ y[pos] + l[neg] @ y[neg])
    if support < -eps and norm_inf(A.T @ y) <= eps:
        return y
    return None


def dual_infeasibility(P, q, A, l, u, dx, eps):
    """Approximate certificate test of eq. (dual_infeas) on dx.

    dx is scaled to unit inf-norm and accepted when ||P x||_inf <= eps,
    q'x < -eps, and (A x)_i <= eps on rows with a finite upper bound and
    (A x)_i >= -eps on rows with a finite lower bound.  Returns the scaled
    certificate, or None."""
    x = np.array(dx, np.float64, copy=True)
    nrm = norm_inf(x)
    if not (nrm > 0.0 and math.isfinite(nrm)):
        return None
    x /= nrm
    if not float(q @ x) < -eps:
        return None
    if norm_inf(P @ x) > eps:
        return None
    Ax = A @ x
    l = np.asarray(l, np.float64)
    u = np.asarray(u, np.float64)
    if np.any(Ax[u < INF_BOUND] > eps) or np.any(Ax[l > -INF_BOUND] < -eps):
        return None
    return x


def infeasibility(qp, dx, dy, s: "Settings"):
    """Primal test first, then dual; returns (status, certificate) or None."""
    if s.eps_prim_inf > 0.0:
        y = primal_infeasibility(qp.A, qp.l, qp.u, dy, s.eps_prim_inf)
        if y is not None:
            return "primal_infeasible", y
    if s.eps_dual_inf > 0.0:
        x = dual_infeasibility(qp.P, qp.q, qp.A, qp.l, qp.u, dx, s.eps_dual_inf)
        if x is not None:
            return "dual_infeasible", x
    return None


def _certificate_result(qp, found, k, res, rho, **kw):
    """Result for an infeasible problem: the certificate in y (primal) or x
    (dual), NaN elsewhere; objective +inf (primal) or -inf (dual)."""
    status, cert = found
    nan_n, nan_m = np.full(qp.n, np.nan), np.full(qp.m, np.nan)
    if status == "primal_infeasible":
        return Result(nan_n, nan_m, cert, status, k, math.inf, res, rho, **kw)
    return Result(cert, nan_m, nan_m, status, k, -math.inf, res, rho, **kw)


# --------------------------------------------------------------------------
# Reduced KKT system and PCG, Section 4 and Section 5.3
# --------------------------------------------------------------------------

def reduced_kkt_apply(P, A, sigma, rho, x):
    """(P + sigma I + A'RA) x with R = rho I (rho a scalar) or R = diag(rho)
    (rho a vector, eq. (rho_vec)), evaluated matrix-free as
    z = R A x; r = P x + sigma x + A' z (Section 5.3)."""
    z = rho * (A @ x)
    return P @ x + sigma * x + A.T @ z


def reduced_kkt_rhs(q, A, sigma, rho, x, z, y):
    """sigma x - q + A'(R z - y), the right-hand side of eq. (kkt_red_sc)
    (of eq. (kkt_red) for a vector R)."""
    return sigma * x - q + A.T @ (rho * z - y)


def jacobi_diag(P, A, sigma, rho):
    """diag(P) + sigma 1 + diag(A'RA), with diag(A'RA)_i = rho ||A_:,i||_2^2
    for R = rho I (Section 5.3.1) and sum_j rho_j A_ji^2 for R = diag(rho)."""
    A = sp.csc_matrix(A)
    colsq = np.zeros(A.shape[1])
    rv = np.broadcast_to(np.asarray(rho, np.float64), (A.shape[0],))
    for j in range(A.shape[1]):
        seg = A.data[A.indptr[j]:A.indptr[j + 1]]
        if np.ndim(rho) == 0:
            colsq[j] = float(seg @ seg)
        else:
            colsq[j] = float((seg * rv[A.indices[A.indptr[j]:A.indptr[j + 1]]]) @ seg)
    if np.ndim(rho) != 0:
        return sp.csr_matrix(P).diagonal() + sigma + colsq
    return sp.csr_matrix(P).diagonal() + sigma + rho * colsq


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    r_norm: float
    directions: list = field(default_factory=list)


def pcg(apply_K, b, x0, Minv, eps, max_iter, relative=False, keep_directions=False) -> PCGResult:
    """Algorithm 3 (Nocedal & Wright Alg. 5.3) with the inf-norm stopping test
    of Section 5.3.4: stop when ||r|| <= eps (or eps ||b|| if relative).

    Step length (reading S7): alpha = r'y / p'Kp.  Algorithm 3 as printed
    carries a minus sign here, which with p^0 = -y^0 makes every step go
    uphill; Section 4.1.1 gives alpha = -r'p / p'Kp, and r'p = -r'y holds
    for every PCG direction, so both the cited Alg. 5.3 and Section 4.1.1
    give the positive step used here."""
    x = np.array(x0, np.float64, copy=True)
    r = apply_K(x) - b
    yv = Minv * r
    p = -yv
    ry = float(r @ yv)
    tol = eps * norm_inf(b) if relative else eps
    k = 0
    dirs = []
    while norm_inf(r) > tol and k < max_iter:
        Kp = apply_K(p)
        pKp = float(p @ Kp)
        if not pKp > 0.0:
            break
        if keep_directions:
            dirs.append((p.copy(), Kp.copy()))
        a = ry / pKp
        x = x + a * p
        r = r + a * Kp
        yv = Minv * r
        ry_new = float(r @ yv)
        beta = ry_new / ry if ry != 0.0 else 0.0
        p = -yv + beta * p
        ry = ry_new
        k += 1
    return PCGResult(x, k, norm_inf(r), dirs)


def pcg_single_reduction(apply_K, b, x0, Minv, eps, max_iter) -> PCGResult:
    """Algorithm 3 rearranged so that both inner products of a step come from
    one reduction (Chronopoulos & Gear, "s-step iterative methods for
    symmetric linear systems", 1989): besides r and y = M^-1 r the method
    carries w = K y and s = K p, and per step computes gamma = r'y and
    delta = w'y of the same vectors.  With beta_i = gamma_i / gamma_(i-1) and
    alpha_i = gamma_i / (delta_i - beta_i gamma_i / alpha_(i-1)) (alpha_0 =
    gamma_0 / delta_0, beta_0 = 0) the recurrences

        p_i = -y_i + beta_i p_(i-1),   s_i = -w_i + beta_i s_(i-1),
        x_(i+1) = x_i + alpha_i p_i,   r_(i+1) = r_i + alpha_i s_i,
        y_(i+1) = M^-1 r_(i+1),        w_(i+1) = K y_(i+1)

    give the iterates of Algorithm 3 (same sign conventions as pcg(): r = Kx
    - b, step length of reading S7) in exact arithmetic, at one product with
    K per step (K y instead of K p; s = K p follows by recurrence).  The
    stopping test ||r||_inf <= eps of Section 5.3.4 is taken on r_(i+1) as
    soon as it is formed."""
    x = np.array(x0, np.float64, copy=True)
    r = apply_K(x) - b
    yv = Minv * r
    k = 0
    if not norm_inf(r) > eps or max_iter <= 0:
        return PCGResult(x, 0, norm_inf(r), [])
    w = apply_K(yv)
    gamma, delta = float(r @ yv), float(w @ yv)
    p = np.zeros_like(x)
    sv = np.zeros_like(x)
    alpha_prev, gamma_prev = 0.0, 0.0
    while True:
        if k == 0:
            beta = 0.0
            den = delta
        else:
            beta = gamma / gamma_prev if gamma_prev != 0.0 else 0.0
            den = delta - beta * gamma / alpha_prev
        if not den > 0.0:
            break
        alpha = gamma / den
        p = -yv + beta * p
        sv = -w + beta * sv
        x = x + alpha * p
        r = r + alpha * sv
        yv = Minv * r
        k += 1
        if not norm_inf(r) > eps or k >= max_iter:
            break
        w = apply_K(yv)
        gamma_prev, alpha_prev = gamma, alpha
        gamma, delta = float(r @ yv), float(w @ yv)
    return PCGResult(x, k, norm_inf(r), [])


def pcg_tolerance(r_prim_scaled, r_dual_scaled, lam=0.15, eps_min=1e-7) -> float:
    """eps = max(lambda sqrt(||r_prim_bar|| ||r_dual_bar||), eps_min)
    (Section 5.3.4)."""
    return max(lam * math.sqrt(r_prim_scaled * r_dual_scaled), eps_min)


# --------------------------------------------------------------------------
# Solvers
# --------------------------------------------------------------------------

@dataclass
class Result:
    x: np.ndarray
    z: np.ndarray
    y: np.ndarray
    status: str
    iters: int
    obj: float
    res: Residuals
    rho: float
    pcg_iters: int = 0
    pcg_per_iter: list = field(default_factory=list)
    rho_history: list = field(default_factory=list)
    kkt_rel_residual: float = 0.0
    scaled_state: tuple = ()


def kkt_factor(P, A, sigma, rv, kind: str = "auto"):
    """The factor the direct ADMM solves eq. (kkt) with: the sparse LDL' of
    the whole quasi-definite matrix, or the dense Cholesky of its Schur
    complement on the variables (many constraints, few variables)."""
    n, m = P.shape[0], A.shape[0]
    if kind == "dense" or (kind == "auto" and n >= 2000 and m >= 4 * n):
        from .dense import DenseSchurFactor
        return DenseSchurFactor(P, A, sigma, rv)
    return KKTFactor(P, A, sigma, rv)


def _prepare(qp, s: Settings):
    sc = ruiz(qp.P, qp.q, qp.A, qp.l, qp.u, s.scaling_iters)
    return sc


def solve(qp, settings: Settings | None = None, x0=None, y0=None) -> Result:
    """Algorithm 1 with the exact LDL' solve of eq. (kkt) (OSQP on the CPU)."""
    s = settings or Settings()
    sc = _prepare(qp, s)
    n, m = qp.n, qp.m
    x = np.zeros(n) if x0 is None else np.asarray(x0, np.float64) / sc.D
    y = np.zeros(m) if y0 is None else sc.c * np.asarray(y0, np.float64) / sc.E
    z = sc.A @ x if x0 is not None else np.zeros(m)
    rho = s.rho0
    rv = rho_vector(rho, sc.l, sc.u, s.rho_vector)
    F = kkt_factor(sc.P, sc.A, s.sigma, rv, s.kkt)
    status = "max_iter"
    res = None
    hist = [rho]
    k = 0
    max_rel = 0.0
    for k in range(1, s.max_iter + 1):
        sol = F.solve(np.concatenate([s.sigma * x - sc.q, z - y / rv]))
        xt, nu = sol[:n], sol[n:]
        zt = z + (nu - y) / rv
        x_prev, y_prev = x, y
        x, z, y = admm_update(xt, zt, x, z, y, s.alpha, rv, sc.l, sc.u)
        need_check = (k % s.check_every == 0) or (s.adaptive_rho and k % s.rho_every == 0)
        if need_check:
            xu, zu, yu = unscale(sc, x, z, y)
            res = residuals(qp.P, qp.q, qp.A, xu, zu, yu, s.eps_abs, s.eps_rel)
            if k % s.check_every == 0 and res.converged():
                status = "solved"
                break
            if k % s.check_every == 0:
                xp, _, yp = unscale(sc, x_prev, z, y_prev)
                found = infeasibility(qp, xu - xp, yu - yp, s)
                if found is not None:
                    return _certificate_result(qp, found, k, res, rho, rho_history=hist,
                                               kkt_rel_residual=max(max_rel, F.max_rel_residual))
            if s.adaptive_rho and k % s.rho_every == 0:
                res_s = residuals(sc.P, sc.q, sc.A, x, z, y)
                new_rho = rho_ratio_rule(rho, res_s)
                if new_rho > s.refactor_ratio * rho or new_rho < rho / s.refactor_ratio:
                    max_rel = max(max_rel, F.max_rel_residual)
                    rho = new_rho
                    rv = rho_vector(rho, sc.l, sc.u, s.rho_vector)
                    F = kkt_factor(sc.P, sc.A, s.sigma, rv, s.kkt)
                    hist.append(rho)
    xu, zu, yu = unscale(sc, x, z, y)
    res = residuals(qp.P, qp.q, qp.A, xu, zu, yu, s.eps_abs, s.eps_rel)
    max_rel = max(max_rel, F.max_rel_residual)
    return Result(xu, zu, yu, status, k, objective(qp.P, qp.q, xu), res, rho,
                  rho_history=hist, kkt_rel_residual=max_rel, scaled_state=(x, z, y))


def solve_pcg(qp, settings: Settings | None = None, max_iter: int | None = None) -> Result:
    """Algorithm 1 with the reduced KKT system eq. (kkt_red_sc) solved by
    warm-started Jacobi-PCG, as in Section 5.3 and Table 1, in FP64."""
    s = settings or Settings()
    sc = _prepare(qp, s)
    n, m = qp.n, qp.m
    P, q, A = sc.P, sc.q, sc.A
    x = np.zeros(n)
    z = np.zeros(m)
    y = np.zeros(m)
    xt = np.zeros(n)
    rho = s.rho0
    rv = rho_vector(rho, sc.l, sc.u, s.rho_vector) if s.rho_vector else rho
    Minv = 1.0 / jacobi_diag(P, A, s.sigma, rv)
    eps = max(s.pcg_lambda * norm_inf(q), s.pcg_eps_min)
    status = "max_iter"
    total_cg = 0
    per_iter = []
    hist = [rho]
    limit = s.max_iter if max_iter is None else max_iter
    k = 0
    for k in range(1, limit + 1):
        b = reduced_kkt_rhs(q, A, s.sigma, rv, x, z, y)
        method = pcg_single_reduction if s.pcg_variant == "single_reduction" else pcg
        out = method(lambda v: reduced_kkt_apply(P, A, s.sigma, rv, v), b, xt, Minv, eps, s.max_cg_iter)
        xt = out.x
        total_cg += out.iters
        per_iter.append(out.iters)
        zt = A @ xt
        x_prev, y_prev = x, y
        x, z, y = admm_update(xt, zt, x, z, y, s.alpha, rv, sc.l, sc.u)
        if k % s.check_every == 0:
            xu, zu, yu = unscale(sc, x, z, y)
            res = residuals(qp.P, qp.q, qp.A, xu, zu, yu, s.eps_abs, s.eps_rel)
            res_s = residuals(P, q, A, x, z, y)
            if res.converged():
                status = "solved"
                break
            xp, _, yp = unscale(sc, x_prev, z, y_prev)
            found = infeasibility(qp, xu - xp, yu - yp, s)
            if found is not None:
                return _certificate_result(qp, found, k, res, rho, pcg_iters=total_cg, pcg_per_iter=per_iter,
                                           rho_history=hist)
            eps = pcg_tolerance(res_s.r_prim, res_s.r_dual, s.pcg_lambda, s.pcg_eps_min)
            if s.adaptive_rho and k % s.rho_every == 0:
                rho = rho_ratio_rule(rho, res_s)
                rv = rho_vector(rho, sc.l, sc.u, s.rho_vector) if s.rho_vector else rho
                Minv = 1.0 / jacobi_diag(P, A, s.sigma, rv)
                hist.append(rho)
    xu, zu, yu = unscale(sc, x, z, y)
    res = residuals(qp.P, qp.q, qp.A, xu, zu, yu, s.eps_abs, s.eps_rel)
    return Result(xu, zu, yu, status, k, objective(qp.P, qp.q, xu), res, rho,
                  pcg_iters=total_cg, pcg_per_iter=per_iter, rho_history=hist,
                  scaled_state=(x, z, y, xt))
