"""Sparse formats of paper Section 4.3 (COO, CSR, CSC).  TEST INFRASTRUCTURE.

Plain loops over small matrices; zero-based indices throughout, as in the
paper.
"""
from __future__ import annotations

import numpy as np


def coo_from_dense(M):
    """COO of Section 4.3.1: entries sorted by row, then by column."""
    M = np.asarray(M, dtype=np.float64)
    value, row_index, column_index = [], [], []
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            if M[i, j] != 0.0:
                value.append(M[i, j])
                row_index.append(i)
                column_index.append(j)
    return np.array(value), np.array(row_index, np.int64), np.array(column_index, np.int64)


def row_pointer_from_row_index(nrows: int, row_index) -> np.ndarray:
    """CSR compression of Section 4.3.2: count the entries of each row, then
    take the cumulative sum with a leading zero."""
    counts = np.zeros(nrows, np.int64)
    for r in row_index:
        counts[r] += 1
    ptr = np.zeros(nrows + 1, np.int64)
    for r in range(nrows):
        ptr[r + 1] = ptr[r] + counts[r]
    return ptr


def csr_from_dense(M):
    value, row_index, column_index = coo_from_dense(M)
    return value, row_pointer_from_row_index(np.asarray(M).shape[0], row_index), column_index


def csc_from_dense(M):
    """CSC of Section 4.3.3: values column-major, column indices compressed."""
    M = np.asarray(M, dtype=np.float64)
    value, row_index = [], []
    ptr = [0]
    for j in range(M.shape[1]):
        for i in range(M.shape[0]):
            if M[i, j] != 0.0:
                value.append(M[i, j])
                row_index.append(i)
        ptr.append(len(value))
    return np.array(value), np.array(row_index, np.int64), np.array(ptr, np.int64)


def csr_of_transpose(nrows: int, ncols: int, value, row_pointer, column_index):
    """CSR of M' built from the CSR of M (the CSC of M read as the CSR of M',
    Section 4.3.3): count entries per column, prefix-sum, then place each
    entry in row-major order of M so that every row of M' is sorted."""
    nnz = len(value)
    counts = np.zeros(ncols, np.int64)
    for k in range(nnz):
        counts[column_index[k]] += 1
    tptr = np.zeros(ncols + 1, np.int64)
    for j in range(ncols):
        tptr[j + 1] = tptr[j] + counts[j]
    cursor = tptr[:-1].copy()
    tval = np.zeros(nnz)
    tcol = np.zeros(nnz, np.int64)
    for i in range(nrows):
        for k in range(row_pointer[i], row_pointer[i + 1]):
            j = column_index[k]
            tval[cursor[j]] = value[k]
            tcol[cursor[j]] = i
            cursor[j] += 1
    return tval, tptr, tcol


def row_index_from_row_pointer(row_pointer) -> np.ndarray:
    """RowIndex expanded from RowPointer (Section 5.4.3, used for the
    pre-multiplication D M)."""
    out = []
    for i in range(len(row_pointer) - 1):
        out.extend([i] * int(row_pointer[i + 1] - row_pointer[i]))
    return np.array(out, np.int64)
