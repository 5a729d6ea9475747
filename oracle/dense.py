"""Dense Schur-complement solve of the ADMM linear step.  TEST INFRASTRUCTURE.

For problems with few variables and many constraints (the 20000 x 200000
random QP) the sparse LDL' of the full KKT matrix fills its trailing block
completely and takes hours in scalar code.  There the oracle eliminates the
constraint block of eq. (kkt) (Section 3.2) by hand instead:

    [[P + sigma I, A'      ], [x~], = [b1],   =>   S x~ = b1 + A' R b2,
     [A,          -R^{-1}  ]] [nu ]   [b2]          nu = R (A x~ - b2),

with S = P + sigma I + A' R A (eq. (kkt_red_sc), the reduced system the
paper's PCG solves), formed densely by a plain C loop (oracle/schur.c) and
factored by LAPACK's Cholesky (S is positive definite: P is positive
semidefinite, sigma > 0, R > 0).  Like the sparse factor, every solve
applies two steps of iterative refinement against the full KKT matrix and
records the relative residual it reaches.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "schur.c")
_LIB = os.path.join(_HERE, "_schur.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile schur.c into oracle/_schur.so (OpenMP when the compiler has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.schur_form.argtypes = [ctypes.c_int32, ctypes.c_int32, i64p, i32p, f64p, f64p, i64p, i32p, f64p,
                                   ctypes.c_double, f64p]
        lib.schur_form.restype = None
        _lib = lib
    return _lib


def schur_matrix(P: sp.spmatrix, A: sp.spmatrix, sigma: float, r) -> np.ndarray:
    """S = P + sigma I + A' diag(r) A, dense."""
    P = sp.csr_matrix(P, dtype=np.float64)
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    n, m = P.shape[0], A.shape[0]
    rv = np.ascontiguousarray(np.broadcast_to(np.asarray(r, np.float64), (m,)))
    S = np.empty((n, n), np.float64)
    _load().schur_form(n, m, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                       rv, P.indptr.astype(np.int64), P.indices.astype(np.int32), P.data, float(sigma), S)
    return S


class DenseSchurFactor:
    """Solves with [[P + sigma I, A'], [A, -diag(1/rho)]] through the
    Cholesky factor of its Schur complement S (see the module docstring)."""

    def __init__(self, P: sp.csr_matrix, A: sp.csr_matrix, sigma: float, rho):
        n, m = P.shape[0], A.shape[0]
        self.n, self.m = n, m
        self.r = np.broadcast_to(np.asarray(rho, np.float64), (m,)).copy()
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.At = self.A.T.tocsr()
        self.K = sp.bmat([[P + sigma * sp.identity(n), A.T],
                          [A, sp.diags(-1.0 / self.r) if m else None]], format="csr")
        L, lower = la.cho_factor(schur_matrix(P, A, sigma, self.r), lower=True, overwrite_a=True,
                                 check_finite=False)
        # kept in Fortran order: LAPACK's solve would otherwise get a transposed
        # copy of the whole factor on every call
        self.cho = (np.asfortranarray(L), lower)
        self.max_rel_residual = 0.0

    def _solve_once(self, rhs: np.ndarray) -> np.ndarray:
        b1, b2 = rhs[:self.n], rhs[self.n:]
        x = la.cho_solve(self.cho, b1 + self.At @ (self.r * b2), check_finite=False)
        nu = self.r * (self.A @ x - b2)
        return np.concatenate([x, nu])

    def solve(self, rhs: np.ndarray, refine: int = 2) -> np.ndarray:
        sol = self._solve_once(rhs)
        for _ in range(refine):
            sol = sol + self._solve_once(rhs - self.K @ sol)
        scale = max(np.max(np.abs(rhs)) if rhs.size else 0.0, 1e-300)
        rel = float(np.max(np.abs(rhs - self.K @ sol)) / scale) if rhs.size else 0.0
        self.max_rel_residual = max(self.max_rel_residual, rel)
        return sol
