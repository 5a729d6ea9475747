"""ctypes front end of the oracle's sparse LDL' (ldl.c).  TEST INFRASTRUCTURE.

``KKTFactor`` factors the quasi-definite KKT matrix of the ADMM linear step
(paper Section 3.2, eq. (kkt)):

    [[P + sigma I,  A'      ],     [x~ ]   [sigma x - q     ]
     [A,           -R^{-1}  ]]  *  [nu ] = [z - R^{-1} y    ]

after a symmetric permutation that orders the nodes by ascending static
degree (number of off-diagonal entries in their KKT row), so that
low-degree constraint rows and variables are eliminated first and the dense
part of the factor, if any, lands in the trailing block.  The solve applies
two steps of iterative refinement against the unpermuted matrix and records
the relative residual it reaches.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldl.c")
_LIB = os.path.join(_HERE, "_ldl.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ldl.c into oracle/_ldl.so with the host C compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.ldl_symbolic.argtypes = [ctypes.c_int32, i64p, i32p, i32p, i64p]
        lib.ldl_symbolic.restype = None
        lib.ldl_numeric.argtypes = [ctypes.c_int32, i64p, i32p, f64p, i64p, i32p, i32p, f64p, f64p]
        lib.ldl_numeric.restype = ctypes.c_int32
        lib.ldl_solve.argtypes = [ctypes.c_int32, i64p, i32p, f64p, f64p, f64p]
        lib.ldl_solve.restype = None
        _lib = lib
    return _lib


def static_degree_order(K: sp.csr_matrix) -> np.ndarray:
    """Permutation sorting nodes by ascending number of off-diagonal entries
    (ties by index)."""
    K = sp.csr_matrix(K)
    deg = np.diff(K.indptr).astype(np.int64)
    diag_present = np.zeros(K.shape[0], np.int64)
    rows = np.repeat(np.arange(K.shape[0]), np.diff(K.indptr))
    diag_present[rows[K.indices == rows]] = 1
    return np.argsort(deg - diag_present, kind="stable")


class LDL:
    """L D L' of a symmetric sparse matrix in a given symmetric order."""

    def __init__(self, K: sp.spmatrix, perm: np.ndarray | None = None):
        lib = _load()
        K = sp.csr_matrix(K, dtype=np.float64)
        n = K.shape[0]
        self.n = n
        self.perm = static_degree_order(K) if perm is None else np.asarray(perm, np.int64)
        Kp = K[self.perm][:, self.perm]
        U = sp.triu(Kp, format="csc")
        U.sort_indices()
        cp = U.indptr.astype(np.int64)
        ci = U.indices.astype(np.int32)
        cx = U.data.astype(np.float64)
        parent = np.empty(n, np.int32)
        cnt = np.empty(n, np.int64)
        lib.ldl_symbolic(n, cp, ci, parent, cnt)
        self.Lp = np.zeros(n + 1, np.int64)
        np.cumsum(cnt, out=self.Lp[1:])
        nnzL = int(self.Lp[-1])
        self.Li = np.empty(max(nnzL, 1), np.int32)
        self.Lx = np.empty(max(nnzL, 1), np.float64)
        self.D = np.empty(max(n, 1), np.float64)
        ok = lib.ldl_numeric(n, cp, ci, cx, self.Lp, parent, self.Li, self.Lx, self.D)
        if ok != n:
            raise np.linalg.LinAlgError(f"LDL': zero or non-finite pivot at permuted index {ok}")
        self.nnzL = nnzL

    def solve_permuted(self, b: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(b[self.perm], dtype=np.float64)
        _load().ldl_solve(self.n, self.Lp, self.Li, self.Lx, self.D, x)
        out = np.empty_like(x)
        out[self.perm] = x
        return out


class KKTFactor:
    """Factor of [[P + sigma I, A'], [A, -diag(1/rho)]] with refinement."""

    def __init__(self, P: sp.csr_matrix, A: sp.csr_matrix, sigma: float, rho):
        n = P.shape[0]
        m = A.shape[0]
        rho_vec = np.broadcast_to(np.asarray(rho, np.float64), (m,)).copy()
        self.n, self.m = n, m
        self.K = sp.bmat([[P + sigma * sp.identity(n), A.T],
                          [A, sp.diags(-1.0 / rho_vec) if m else None]], format="csr")
        self.ldl = LDL(self.K)
        self.max_rel_residual = 0.0

    def solve(self, rhs: np.ndarray, refine: int = 2) -> np.ndarray:
        sol = self.ldl.solve_permuted(rhs)
        for _ in range(refine):
            res = rhs - self.K @ sol
            sol = sol + self.ldl.solve_permuted(res)
        scale = max(np.max(np.abs(rhs)) if rhs.size else 0.0, 1e-300)
        rel = float(np.max(np.abs(rhs - self.K @ sol)) / scale) if rhs.size else 0.0
        self.max_rel_residual = max(self.max_rel_residual, rel)
        return sol
