"""gbosqp: ADMM with warm-started Jacobi-PCG for sparse QPs on one GB300.

The solver is the C-ABI library ``libgbosqp.so`` (hand-written sm_103a
CUDA); ``paper_1912_04263_gb300.binding`` is its ctypes front end, which
loads the library on import and fails loudly if it has not been built.
"""
