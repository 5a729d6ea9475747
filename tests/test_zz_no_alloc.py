"""The allocation-free SpMV entry point (gbosqp_spmv_noalloc) gives the same
result as gbosqp_spmv, on two calls in a row.

It exists for callers that cannot let the library allocate device memory
during a call (real-time loops, code recording a stream capture, hosts whose
device memory belongs to another allocator); its scratch is a fixed device
array inside the library.  This file is collected last so that a run that
stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

import qpgen

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_04263_gb300 import binding
    return binding


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_spmv_matches_spmv(gb, prec):
    torch = pytest.importorskip("torch")
    # long rows (factor rows of 4000 nonzeros, a budget row of 8000, columns
    # of A' with hundreds): the scratch combines pieces of long rows
    qp = qpgen.portfolio_qp(8000, 50, 0)
    dtype = torch.float32 if prec == gb.FP32 else torch.float64
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    with gb.Solver(qp, precision=prec) as s:
        n, m = s.n, s.m
        for which, nin, nout in [(gb.MAT_A, n, m), (gb.MAT_PAT, n + m, n)]:
            x = rng.standard_normal(nin)
            xr = x.astype(np.float32).astype(np.float64) if prec == gb.FP32 else x
            ref = gb.gbosqp_spmv(s.h, which, xr)
            M = gb.gbosqp_get_scaled_csr(s.h, which)
            scale = abs(M) @ np.abs(xr)
            L = np.diff(M.indptr)
            tol = (L + 4) * U32 * scale + U32 * np.abs(ref) if prec == gb.FP32 else 1e-12 * scale
            xd = torch.as_tensor(xr, dtype=dtype, device=dev)
            for _ in range(2):
                yd = torch.full((nout,), float("nan"), dtype=dtype, device=dev)
                torch.cuda.synchronize()
                gb.gbosqp_spmv_noalloc(s.h, which, xd, yd)
                torch.cuda.synchronize()
                got = yd.double().cpu().numpy()
                assert np.all(np.isfinite(got))
                assert np.all(np.abs(got - ref) <= tol + 1e-300)
