"""The allocation-free SpMV entry point (gbosqp_spmv_noalloc), on two calls in
a row: its result matches the FP64 product of the scaled matrix the library
holds (read back through gbosqp_get_scaled_csr) within the FP32 rounding
bound of each row sum (FP32 handle) or 1e-12 relative (FP64 handle), and the
call leaves the device's free memory unchanged.

The entry point exists for callers that cannot let the library allocate
device memory during a call: real-time loops that cannot take the
allocator's latency, code recording a stream capture, and hosts whose device
memory belongs to another allocator.  Its scratch is a fixed device array
inside the library.  This file is collected last so that a run that stops at
the first failure has run every other test first.
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
def test_noalloc_spmv_matches_host_product(gb, prec):
    torch = pytest.importorskip("torch")
    # long rows (factor rows of 4000 nonzeros, a budget row of 8000, columns
    # of A' with hundreds): rows cut between warps combine through the scratch
    qp = qpgen.portfolio_qp(8000, 50, 0)
    dtype = torch.float32 if prec == gb.FP32 else torch.float64
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    with gb.Solver(qp, precision=prec) as s:
        n, m = s.n, s.m
        for which, nin, nout in [(gb.MAT_A, n, m), (gb.MAT_PAT, n + m, n)]:
            x = rng.standard_normal(nin)
            xr = x.astype(np.float32).astype(np.float64) if prec == gb.FP32 else x
            M = gb.gbosqp_get_scaled_csr(s.h, which)  # the working-precision values, exactly, in FP64
            ref = M @ xr
            scale = abs(M) @ np.abs(xr)
            L = np.diff(M.indptr)
            # FP32: the products and the recursive row sum each round, (L + 4) 2^-24 of sum |a x|
            tol = (L + 4) * U32 * scale if prec == gb.FP32 else 1e-12 * scale
            xd = torch.as_tensor(xr, dtype=dtype, device=dev)
            for _ in range(2):
                yd = torch.full((nout,), float("nan"), dtype=dtype, device=dev)
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info(dev)[0]
                gb.gbosqp_spmv_noalloc(s.h, which, xd, yd)
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info(dev)[0] == free0
                got = yd.double().cpu().numpy()
                assert np.all(np.isfinite(got))
                assert np.all(np.abs(got - ref) <= tol + 1e-300), float(np.max(np.abs(got - ref) / (tol + 1e-300)))
