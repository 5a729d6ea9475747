"""The synthetic inputs follow their stated recipe (no GPU): Bernoulli
patterns at the stated density with independent entries, N(0, 1) values,
the Lasso regularisation weight lambda = 0.2 ||D'b||_inf and block layout,
the portfolio's uniform risk weights on [0, sqrt(k)] and budget row, the
random class's bounds and regularised P, and the size of the benchmark's
Lasso workload.  Tolerances are five standard deviations of each
statistic."""
import numpy as np
import scipy.sparse as sp

import qpgen
from qpgen.problems import INF


def _pattern_stats(M, p):
    M = sp.csr_matrix(M)
    rows, cols = M.shape
    N = rows * cols
    dens = M.nnz / N
    assert abs(dens - p) <= 5 * np.sqrt(p * (1 - p) / N), (dens, p)
    per_row = np.diff(M.indptr)
    var = cols * p * (1 - p)  # Binomial(cols, p) per row when entries are independent
    assert abs(per_row.var() - var) <= 5 * var * np.sqrt(2.0 / rows), (per_row.var(), var)
    v = M.data
    assert abs(v.mean()) <= 5 / np.sqrt(v.size)
    assert abs(v.var() - 1.0) <= 5 * np.sqrt(2.0 / v.size)


def test_random_class():
    n, m = 200, 2000
    qp = qpgen.random_qp(n, m, 3)
    _pattern_stats(qp.A, 0.15)
    assert np.all((-qp.l >= 0) & (-qp.l < 1)) and np.all((qp.u >= 0) & (qp.u < 1))
    for v in (-qp.l, qp.u):  # U[0, 1)
        assert abs(v.mean() - 0.5) <= 5 / np.sqrt(12 * m)
    assert abs(qp.q.mean()) <= 5 / np.sqrt(n) and abs(qp.q.var() - 1) <= 5 * np.sqrt(2 / n)
    # P = M M' + 1e-2 I: symmetric, and P - 1e-2 I is positive semidefinite
    Pd = qp.P.toarray()
    assert np.array_equal(Pd, Pd.T)
    assert np.linalg.eigvalsh(Pd - 1e-2 * np.eye(n)).min() >= -1e-9 * np.abs(Pd).max()


def test_lasso_class():
    nf, ms = 50, 2000
    qp = qpgen.lasso_qp(nf, ms, 2)
    D = qp.A[:ms, :nf]
    _pattern_stats(D, 0.15)
    b = qp.l[:ms]
    assert np.array_equal(qp.l[:ms], qp.u[:ms])  # D x - y = b
    lam = 0.2 * np.max(np.abs(D.T @ b))
    assert np.isclose(qp.meta["lam"], lam, rtol=1e-14)
    assert np.array_equal(qp.q, np.concatenate([np.zeros(nf + ms), lam * np.ones(nf)]))
    # blocks: [D -I 0; I 0 -I; I 0 I], P = blkdiag(0, 2 I, 0)
    A = qp.A.toarray()
    assert np.array_equal(A[:ms, nf:nf + ms], -np.eye(ms))
    assert np.array_equal(A[ms:ms + nf, :nf], np.eye(nf)) and np.array_equal(A[ms:ms + nf, nf + ms:], -np.eye(nf))
    assert np.array_equal(A[ms + nf:, :nf], np.eye(nf)) and np.array_equal(A[ms + nf:, nf + ms:], np.eye(nf))
    assert np.array_equal(qp.P.diagonal(), np.concatenate([np.zeros(nf), 2 * np.ones(ms), np.zeros(nf)]))
    assert qp.P.nnz == ms
    assert np.all(qp.l[ms:ms + nf] <= -INF) and np.all(qp.u[ms:ms + nf] == 0)
    assert np.all(qp.l[ms + nf:] == 0) and np.all(qp.u[ms + nf:] >= INF)


def test_portfolio_class():
    na, k = 3000, 30
    qp = qpgen.portfolio_qp(na, k, 5)
    F = qp.A[:k, :na].T
    _pattern_stats(F, 0.5)
    d = qp.P.diagonal()[:na] / 2.0  # risk weights: U[0, sqrt(k))
    a = np.sqrt(k)
    assert d.min() >= 0 and d.max() < a
    assert abs(d.mean() - a / 2) <= 5 * a / np.sqrt(12 * na)
    assert np.array_equal(qp.P.diagonal()[na:], 2 * np.ones(k)) and qp.P.nnz == na + k
    A = qp.A.tocsr()
    assert np.array_equal(A[:k, na:].toarray(), -np.eye(k))
    assert np.array_equal(A[k].toarray().ravel(), np.concatenate([np.ones(na), np.zeros(k)]))
    assert qp.l[k] == 1 and qp.u[k] == 1
    assert np.array_equal(A[k + 1:, :na].toarray(), np.eye(na))
    assert np.all(qp.l[k + 1:] == 0) and np.all(qp.u[k + 1:] >= INF)
    assert np.all(qp.l[:k] == 0) and np.all(qp.u[:k] == 0)


def test_benchmark_lasso_workload_size():
    """The measured workload: D 100000 x 1000 at 15%, n = m = 102000,
    nnz(A) = nnz(D) + 100000 + 2000 (about 15.1M), nnz(P) = 100000."""
    qp = qpgen.by_name("lasso_1000x100000", 0)
    assert qp.n == 102000 and qp.m == 102000
    nnz_d = qp.A.nnz - 102000
    assert abs(nnz_d / 1e8 - 0.15) <= 5 * np.sqrt(0.15 * 0.85 / 1e8)
    assert qp.P.nnz == 100000
