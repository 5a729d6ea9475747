"""Seeded synthetic QPs:  minimize 1/2 x'Px + q'x  subject to  l <= Ax <= u.

The classes follow the problem classes the paper benchmarks on (Section 6.1:
Random, Lasso, Portfolio, Equality); the benchmark instances themselves are
not used.  Sizes and distributions follow the workloads this solver is
measured on:

* random_qp    P = M M' + 1e-2 I with M n x n Bernoulli(density) N(0,1);
               A m x n Bernoulli(density) N(0,1); q ~ N(0,1);
               l = -U[0,1], u = U[0,1].
* lasso_qp     variables (x, y, t):  min y'y + lam 1't
               s.t. y = D x - b,  -t <= x <= t.
               D is m_samples x n_features Bernoulli(density) N(0,1);
               x_true has half zeros and the rest N(0, 1/n_features);
               b = D x_true + N(0, noise_var); lam = 0.2 ||D'b||_inf.
* portfolio_qp variables (x, y):  min x'Dx + y'y - mu'x / gamma
               s.t. y = F'x,  1'x = 1,  x >= 0.
               F is n x k Bernoulli(density) N(0,1); D = diag(U[0, sqrt(k)]);
               mu ~ N(0,1).
* control_qp   states x_0..x_T (nx each), inputs u_0..u_{T-1} (nu each):
               min x_T'Q_T x_T + sum_t x_t'Q x_t + u_t'R u_t
               s.t. x_0 = x_init, x_{t+1} = A x_t + B u_t, |x_t| <= xbar,
               |u_t| <= ubar.  A = I + Bernoulli(density) N(0, 0.0025), B
               Bernoulli(density) N(0,1), Q = diag of Bernoulli(0.7) U[0,10],
               Q_T = Q, R = 0.1 I, xbar = 1 + U[0,1], ubar = 0.5 + U[0,1],
               x_init = 0.25 U[-1,1] xbar.
* huber_qp     Huber fitting of b ~ A x with threshold M = 1 as the QP
               min u'u + 2M 1'(r + s)  s.t.  A x - u - r + s = b, r, s >= 0
               (the Huber penalty of a residual a'x - b splits into a
               quadratic part u and linear parts r, s).  A m x n
               Bernoulli(density) N(0,1); x_true ~ N(0, 1/n); b = A x_true +
               e with e ~ N(0, 1/4) and 5% of the entries U[0, 10] outliers.
* svm_qp       hinge-loss support vector machine, min x'x + lam 1't
               s.t. t >= diag(b) A x + 1, t >= 0; labels b = +1 on the first
               half of the m points, -1 on the rest; features Bernoulli(density)
               with values N(+1/n, 1/n) for b = +1 and N(-1/n, 1/n) for
               b = -1; lam = 1.

In N(a, b) the second argument is the variance.  P is returned as the full
symmetric matrix in CSR with sorted column indices; infinite bounds are
+-inf.  Nothing here performs solver arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .rng import Stream, bernoulli_pattern

INF = np.inf


@dataclass
class QP:
    P: sp.csr_matrix
    q: np.ndarray
    A: sp.csr_matrix
    l: np.ndarray
    u: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.P.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    def nnz(self) -> int:
        return int(self.P.nnz + self.A.nnz)


def _csr(rows, cols, vals, shape) -> sp.csr_matrix:
    """CSR from entries already in row-major order (no duplicates)."""
    nrows = shape[0]
    counts = np.bincount(rows, minlength=nrows) if rows.size else np.zeros(nrows, np.int64)
    indptr = np.zeros(nrows + 1, np.int64)
    np.cumsum(counts, out=indptr[1:])
    M = sp.csr_matrix((np.asarray(vals, np.float64), cols.astype(np.int32), indptr), shape=shape)
    M.has_sorted_indices = True
    return M


def _clean(M) -> sp.csr_matrix:
    M = sp.csr_matrix(M, dtype=np.float64)
    M.sum_duplicates()
    M.eliminate_zeros()
    M.sort_indices()
    return M


def sparse_normal(seed: int, tag: str, nrows: int, ncols: int, density: float) -> sp.csr_matrix:
    rows, cols = bernoulli_pattern(Stream(seed, tag + ".pattern"), nrows, ncols, density)
    vals = Stream(seed, tag + ".values").normal(rows.size)
    return _csr(rows, cols, vals, (nrows, ncols))


def random_qp(n: int, m: int, seed: int, p_density: float = 0.15, a_density: float = 0.15,
              p_reg: float = 1e-2) -> QP:
    M = sparse_normal(seed, "random/M", n, n, p_density)
    P = _clean(M @ M.T + p_reg * sp.identity(n, format="csr"))
    A = sparse_normal(seed, "random/A", m, n, a_density)
    q = Stream(seed, "random/q").normal(n)
    l = -Stream(seed, "random/l").uniform(m)
    u = Stream(seed, "random/u").uniform(m)
    return QP(P, q, A, l, u, name=f"random_n{n}_m{m}_s{seed}",
              meta=dict(kind="random", n=n, m=m, seed=seed, p_density=p_density, a_density=a_density))


def lasso_qp(n_features: int = 1000, m_samples: int = 100000, seed: int = 0, density: float = 0.15,
             noise_var: float = 1e-2) -> QP:
    nf, ms = n_features, m_samples
    D = sparse_normal(seed, "lasso/D", ms, nf, density)
    perm = Stream(seed, "lasso/support").permutation(nf)
    x_true = np.zeros(nf)
    nz = perm[nf // 2:]
    x_true[nz] = Stream(seed, "lasso/x_true").normal(nz.size, 0.0, np.sqrt(1.0 / nf))
    b = D @ x_true + Stream(seed, "lasso/noise").normal(ms, 0.0, np.sqrt(noise_var))
    lam = 0.2 * np.max(np.abs(D.T @ b)) if ms else 0.0
    In = sp.identity(nf, format="csr")
    Im = sp.identity(ms, format="csr")
    P = _clean(sp.block_diag([sp.csr_matrix((nf, nf)), 2.0 * Im, sp.csr_matrix((nf, nf))], format="csr"))
    q = np.concatenate([np.zeros(nf), np.zeros(ms), lam * np.ones(nf)])
    A = _clean(sp.bmat([[D, -Im, None], [In, None, -In], [In, None, In]], format="csr"))
    l = np.concatenate([b, -INF * np.ones(nf), np.zeros(nf)])
    u = np.concatenate([b, np.zeros(nf), INF * np.ones(nf)])
    return QP(P, q, A, l, u, name=f"lasso_f{nf}_s{ms}_s{seed}",
              meta=dict(kind="lasso", n_features=nf, m_samples=ms, seed=seed, lam=lam))


def portfolio_qp(n_assets: int = 100000, k_factors: int = 1000, seed: int = 0, density: float = 0.5,
                 gamma: float = 1.0) -> QP:
    na, k = n_assets, k_factors
    F = sparse_normal(seed, "portfolio/F", na, k, density)
    Dd = Stream(seed, "portfolio/D").uniform(na) * np.sqrt(k)
    mu = Stream(seed, "portfolio/mu").normal(na)
    P = _clean(sp.block_diag([sp.diags(2.0 * Dd), 2.0 * sp.identity(k)], format="csr"))
    q = np.concatenate([-mu / gamma, np.zeros(k)])
    A = _clean(sp.bmat([[F.T.tocsr(), -sp.identity(k)],
                        [sp.csr_matrix(np.ones((1, na))), None],
                        [sp.identity(na), None]], format="csr"))
    l = np.concatenate([np.zeros(k), [1.0], np.zeros(na)])
    u = np.concatenate([np.zeros(k), [1.0], INF * np.ones(na)])
    return QP(P, q, A, l, u, name=f"portfolio_n{na}_k{k}_s{seed}",
              meta=dict(kind="portfolio", n_assets=na, k_factors=k, seed=seed))


def equality_qp(n: int, m: int, seed: int, density: float = 0.15) -> QP:
    """Equality class (l = u): P = M M' + 1e-2 I, A random, b = A x0 feasible."""
    M = sparse_normal(seed, "equality/M", n, n, density)
    P = _clean(M @ M.T + 1e-2 * sp.identity(n, format="csr"))
    A = sparse_normal(seed, "equality/A", m, n, density)
    x0 = Stream(seed, "equality/x0").normal(n)
    b = A @ x0
    q = Stream(seed, "equality/q").normal(n)
    return QP(P, q, A, b.copy(), b.copy(), name=f"equality_n{n}_m{m}_s{seed}",
              meta=dict(kind="equality", n=n, m=m, seed=seed))


def box_qp(n: int, seed: int, with_inf: bool = True, scale_a: bool = False) -> QP:
    """Diagonal P and A = diag(a) (A = I unless scale_a): a QP with a closed-form
    solution.  Some bounds are infinite when with_inf."""
    s = Stream(seed, "box/pdiag")
    pd = 0.5 + 2.0 * s.uniform(n)
    q = Stream(seed, "box/q").normal(n, 0.0, 4.0)
    a = (0.5 + 1.5 * Stream(seed, "box/a").uniform(n)) if scale_a else np.ones(n)
    lo = -Stream(seed, "box/l").uniform(n) - 0.1
    hi = Stream(seed, "box/u").uniform(n) + 0.1
    if with_inf:
        sel = Stream(seed, "box/inf").uniform(n)
        lo[sel < 0.2] = -INF
        hi[(sel >= 0.2) & (sel < 0.4)] = INF
        both = sel >= 0.9
        lo[both] = -INF
        hi[both] = INF
    P = _clean(sp.diags(pd))
    A = _clean(sp.diags(a))
    return QP(P, q, A, lo, hi, name=f"box_n{n}_s{seed}", meta=dict(kind="box", seed=seed))


def tiny_qp(n: int, m: int, seed: int, n_eq: int = 0, n_inf: int = 0) -> QP:
    """Small dense strictly convex QP (P > 0) for brute-force active-set checks.
    The first n_eq constraints are equalities; n_inf bounds are infinite."""
    Md = Stream(seed, "tiny/M").normal(n * n).reshape(n, n)
    P = Md @ Md.T + 0.5 * np.eye(n)
    P = 0.5 * (P + P.T)
    A = Stream(seed, "tiny/A").normal(m * n).reshape(m, n)
    q = Stream(seed, "tiny/q").normal(n, 0.0, 4.0)
    c = Stream(seed, "tiny/c").normal(m, 0.0, 0.25)
    w = 0.2 + Stream(seed, "tiny/w").uniform(m)
    l = c - w
    u = c + w
    l[:n_eq] = c[:n_eq]
    u[:n_eq] = c[:n_eq]
    if n_inf:
        idx = Stream(seed, "tiny/inf").permutation(m - n_eq)[:n_inf] + n_eq
        for j, i in enumerate(idx):
            if j % 2 == 0:
                l[i] = -INF
            else:
                u[i] = INF
    return QP(_clean(sp.csr_matrix(P)), q, _clean(sp.csr_matrix(A)), l, u,
              name=f"tiny_n{n}_m{m}_s{seed}", meta=dict(kind="tiny", seed=seed))


def rowlen_qp(row_lengths, n: int, seed: int, zero_p_every: int = 3) -> QP:
    """A with prescribed row lengths (distinct uniform columns, N(0,1)
    values) and a diagonal P that is zero on every zero_p_every-th entry
    (empty rows of P).  For exercising SpMV work splitting: empty rows, rows
    at and around the per-item capacity, and very long rows."""
    rows, cols = [], []
    st = Stream(seed, "rowlen/cols")
    for i, L in enumerate(row_lengths):
        L = int(min(L, n))
        if L:
            # distinct uniform columns: first occurrences of uniform draws
            k = 2 * L + 16
            while True:
                idx = np.floor(st.uniform(k) * n).astype(np.int64)
                _, first = np.unique(idx, return_index=True)
                if first.size >= L:
                    break
                k *= 2
            c = np.sort(idx[np.sort(first)[:L]])
            rows.append(np.full(L, i, np.int64))
            cols.append(c.astype(np.int64))
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = Stream(seed, "rowlen/vals").normal(rows.size)
    m = len(row_lengths)
    A = _csr(rows, cols, vals, (m, n))
    pd = 0.5 + Stream(seed, "rowlen/pd").uniform(n)
    if zero_p_every:
        pd[::zero_p_every] = 0.0
    P = _clean(sp.diags(pd))
    q = Stream(seed, "rowlen/q").normal(n)
    l = -Stream(seed, "rowlen/l").uniform(m) - 0.1
    u = Stream(seed, "rowlen/u").uniform(m) + 0.1
    return QP(P, q, A, l, u, name=f"rowlen_m{m}_n{n}_s{seed}", meta=dict(kind="rowlen", seed=seed))


def infeasible_primal_qp() -> QP:
    """x1 >= 1 and x1 <= 0 (plus a harmless second variable)."""
    P = _clean(sp.identity(2))
    A = _clean(sp.csr_matrix(np.array([[1.0, 0.0], [1.0, 0.0], [0.0, 1.0]])))
    return QP(P, np.zeros(2), A, np.array([1.0, -INF, -1.0]), np.array([INF, 0.0, 1.0]),
              name="infeasible_primal")


def infeasible_dual_qp() -> QP:
    """min -x1 with x1 unbounded above (P = 0 on x1)."""
    P = _clean(sp.csr_matrix(np.array([[0.0, 0.0], [0.0, 1.0]])))
    A = _clean(sp.csr_matrix(np.array([[1.0, 0.0], [0.0, 1.0]])))
    return QP(P, np.array([-1.0, 0.0]), A, np.array([0.0, -1.0]), np.array([INF, 1.0]),
              name="infeasible_dual")


def random_primal_infeasible_qp(n: int, m: int, seed: int, density: float = 0.3) -> QP:
    """random_qp(n, m) plus three rows that contradict each other: a1'x >= 1,
    a2'x >= 1 and (a1 + a2)'x <= 1.5 with a1, a2 N(0,1) dense rows (only the
    combination y = (-1, -1, 1) of the three rows exposes it)."""
    base = random_qp(n, m, seed, p_density=density, a_density=density)
    a = Stream(seed, "pinf/a").normal(2 * n).reshape(2, n)
    extra = np.vstack([a[0], a[1], a[0] + a[1]])
    A = _clean(sp.vstack([base.A, sp.csr_matrix(extra)], format="csr"))
    l = np.concatenate([base.l, [1.0, 1.0, -INF]])
    u = np.concatenate([base.u, [INF, INF, 1.5]])
    return QP(base.P, base.q, A, l, u, name=f"pinf_n{n}_m{m}_s{seed}",
              meta=dict(kind="primal_infeasible", n=n, m=m, seed=seed))


def random_dual_infeasible_qp(n: int, m: int, k: int, seed: int, density: float = 0.3) -> QP:
    """Unbounded QP: variables (x1, x2) with x2 of size k absent from P
    (P = blkdiag(M M' + 1e-2 I, 0)), q2 < 0 on x2, and x2 entering only
    rows with an infinite upper bound through nonnegative coefficients; the
    m rows in x1 alone have l = -U[0,1], u = U[0,1]."""
    n1 = n - k
    M = sparse_normal(seed, "dinf/M", n1, n1, density)
    P1 = M @ M.T + 1e-2 * sp.identity(n1, format="csr")
    P = _clean(sp.block_diag([P1, sp.csr_matrix((k, k))], format="csr"))
    A1 = sparse_normal(seed, "dinf/A1", m, n1, density)
    B1 = sparse_normal(seed, "dinf/B1", k, n1, density)
    B2 = sp.diags(0.5 + Stream(seed, "dinf/B2").uniform(k))
    A = _clean(sp.bmat([[A1, None], [B1, B2]], format="csr"))
    q = np.concatenate([Stream(seed, "dinf/q1").normal(n1), -0.5 - Stream(seed, "dinf/q2").uniform(k)])
    l = np.concatenate([-Stream(seed, "dinf/l").uniform(m), -1.0 - Stream(seed, "dinf/lb").uniform(k)])
    u = np.concatenate([Stream(seed, "dinf/u").uniform(m), INF * np.ones(k)])
    return QP(P, q, A, l, u, name=f"dinf_n{n}_m{m}_k{k}_s{seed}",
              meta=dict(kind="dual_infeasible", n=n, m=m, k=k, seed=seed))


def control_qp(nx: int, nu: int, T: int, seed: int, density: float = 0.3) -> QP:
    st = lambda tag: Stream(seed, "control/" + tag)  # noqa: E731
    Ad = sp.identity(nx, format="csr") + sparse_normal(seed, "control/A", nx, nx, density) * 0.05
    Bd = sparse_normal(seed, "control/B", nx, nu, density)
    qd = st("Q").uniform(nx) * 10.0
    qd[st("Qmask").uniform(nx) > 0.7] = 0.0
    xbar = 1.0 + st("xbar").uniform(nx)
    ubar = 0.5 + st("ubar").uniform(nu)
    x0 = 0.25 * (2.0 * st("x0").uniform(nx) - 1.0) * xbar
    nX, nU = (T + 1) * nx, T * nu
    # objective: 2 Q on x_0..x_T (Q_T = Q), 2 R on u (the 1/2 x'Px convention)
    P = _clean(sp.block_diag([sp.diags(np.tile(2.0 * qd, T + 1)), sp.diags(np.full(nU, 0.2))], format="csr"))
    # dynamics rows: -x_0 = -x_init; A x_t + B u_t - x_{t+1} = 0
    Ax = sp.kron(sp.eye(T + 1), -sp.eye(nx)) + sp.kron(sp.eye(T + 1, k=-1), Ad)
    Bu = sp.kron(sp.vstack([sp.csr_matrix((1, T)), sp.eye(T)]), Bd)
    Aeq = sp.hstack([Ax, Bu])
    Aineq = sp.identity(nX + nU, format="csr")
    A = _clean(sp.vstack([Aeq, Aineq], format="csr"))
    leq = np.concatenate([-x0, np.zeros(T * nx)])
    lineq = np.concatenate([np.tile(-xbar, T + 1), np.tile(-ubar, T)])
    uineq = np.concatenate([np.tile(xbar, T + 1), np.tile(ubar, T)])
    return QP(P, np.zeros(nX + nU), A, np.concatenate([leq, lineq]), np.concatenate([leq, uineq]),
              name=f"control_nx{nx}_nu{nu}_T{T}_s{seed}",
              meta=dict(kind="control", nx=nx, nu=nu, T=T, seed=seed, x_init=x0))


def huber_qp(n: int, m: int, seed: int, density: float = 0.15, M: float = 1.0) -> QP:
    Ad = sparse_normal(seed, "huber/A", m, n, density)
    x_true = Stream(seed, "huber/x").normal(n, 0.0, np.sqrt(1.0 / n))
    e = Stream(seed, "huber/noise").normal(m, 0.0, 0.5)
    out = Stream(seed, "huber/outlier").uniform(m) < 0.05
    e[out] = 10.0 * Stream(seed, "huber/outval").uniform(m)[out]
    b = Ad @ x_true + e
    Im = sp.identity(m, format="csr")
    P = _clean(sp.block_diag([sp.csr_matrix((n, n)), 2.0 * Im, sp.csr_matrix((2 * m, 2 * m))], format="csr"))
    q = np.concatenate([np.zeros(n + m), 2.0 * M * np.ones(2 * m)])
    A = _clean(sp.bmat([[Ad, -Im, -Im, Im], [None, None, Im, None], [None, None, None, Im]], format="csr"))
    l = np.concatenate([b, np.zeros(2 * m)])
    u = np.concatenate([b, INF * np.ones(2 * m)])
    return QP(P, q, A, l, u, name=f"huber_n{n}_m{m}_s{seed}", meta=dict(kind="huber", n=n, m=m, seed=seed))


def svm_qp(n: int, m: int, seed: int, density: float = 0.15, lam: float = 1.0) -> QP:
    half = m // 2
    b = np.concatenate([np.ones(half), -np.ones(m - half)])
    rows, cols = bernoulli_pattern(Stream(seed, "svm/pattern"), m, n, density)
    vals = Stream(seed, "svm/values").normal(rows.size, 0.0, np.sqrt(1.0 / n)) + b[rows] / n
    F = _csr(rows, cols, vals, (m, n))
    Im = sp.identity(m, format="csr")
    P = _clean(sp.block_diag([2.0 * sp.identity(n), sp.csr_matrix((m, m))], format="csr"))
    q = np.concatenate([np.zeros(n), lam * np.ones(m)])
    A = _clean(sp.bmat([[sp.diags(b) @ F, -Im], [None, Im]], format="csr"))
    l = np.concatenate([-INF * np.ones(m), np.zeros(m)])
    u = np.concatenate([-np.ones(m), INF * np.ones(m)])
    return QP(P, q, A, l, u, name=f"svm_n{n}_m{m}_s{seed}", meta=dict(kind="svm", n=n, m=m, seed=seed))


def by_name(name: str, seed: int = 0) -> QP:
    """The named workloads: full-size (C0..C4) and small versions of the same
    families used for oracle-backed parity."""
    table = {
        "random_100x1000": lambda s: random_qp(100, 1000, s),
        "lasso_1000x100000": lambda s: lasso_qp(1000, 100000, s),
        "portfolio_100000x1000": lambda s: portfolio_qp(100000, 1000, s),
        "random_20000x200000": lambda s: random_qp(20000, 200000, s, p_density=5e-4, a_density=0.01),
        "random_5000x50000": lambda s: random_qp(5000, 50000, s),  # held-out workload of the learned policy
        # small members of the same families
        "lasso_50x2000": lambda s: lasso_qp(50, 2000, s),
        "lasso_100x5000": lambda s: lasso_qp(100, 5000, s),
        "portfolio_3000x30": lambda s: portfolio_qp(3000, 30, s),
        "portfolio_8000x50": lambda s: portfolio_qp(8000, 50, s),
        "random_300x3000": lambda s: random_qp(300, 3000, s),
        "random_2000x20000": lambda s: random_qp(2000, 20000, s, p_density=5e-3, a_density=0.01),
        "equality_200x100": lambda s: equality_qp(200, 100, s),
        "control_20x10_T20": lambda s: control_qp(20, 10, 20, s),
        "huber_50x500": lambda s: huber_qp(50, 500, s),
        "svm_50x500": lambda s: svm_qp(50, 500, s),
        # larger members of the same three classes (GPU parity at size)
        "huber_1000x20000": lambda s: huber_qp(1000, 20000, s),
        "svm_1000x20000": lambda s: svm_qp(1000, 20000, s),
    }
    return table[name](seed)
