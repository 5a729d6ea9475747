"""Seeded synthetic QP inputs shaped like the paper's benchmark classes.

This package is the one piece shared by the CPU oracle and the GPU solver: it
produces problem data (matrices in CSR, vectors) and nothing else.  It holds
none of the solver's arithmetic.
"""
from .problems import (  # noqa: F401
    QP,
    INF,
    random_qp,
    lasso_qp,
    portfolio_qp,
    equality_qp,
    box_qp,
    tiny_qp,
    rowlen_qp,
    infeasible_primal_qp,
    infeasible_dual_qp,
    random_primal_infeasible_qp,
    random_dual_infeasible_qp,
    control_qp,
    huber_qp,
    svm_qp,
    by_name,
)
