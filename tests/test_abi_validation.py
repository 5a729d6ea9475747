"""osqp_setup's host-side argument checks (no GPU): every malformed shape,
size or pointer is refused with its error code and a message before any
CUDA call, and a well-formed problem on a machine without a usable GPU is
refused with the CUDA error rather than solved some other way."""
import ctypes

import numpy as np
import pytest

import qpgen

gb = pytest.importorskip("paper_1912_04263_gb300.binding")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return gb.lib()


def _setup(lib, P, A, q, l, u, s=None):
    s = s if s is not None else gb.default_settings()
    h = ctypes.c_void_p()
    rc = lib.osqp_setup(ctypes.byref(h), ctypes.byref(P), ctypes.byref(A), gb._ptr(q), gb._ptr(l), gb._ptr(u),
                        ctypes.byref(s))
    return rc, h.value, lib.gbosqp_setup_error().decode()


@pytest.fixture(scope="module")
def parts():
    qp = qpgen.random_qp(6, 9, 0)
    hp, ha = gb._HostCsr(qp.P), gb._HostCsr(qp.A)
    return qp, hp, ha


def _csr(base, **kw):
    c = gb.Csr(base.nrows, base.ncols, base.nnz, base.rowptr, base.colind, base.val)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("which,change,code,words", [
    ("P", dict(nrows=0, ncols=0), "ERR_DIMENSION", "n > 0"),
    ("P", dict(ncols=7), "ERR_DIMENSION", "n x n"),
    ("A", dict(ncols=5), "ERR_DIMENSION", "m x n"),
    ("A", dict(nrows=-1), "ERR_DIMENSION", "m x n"),
    ("P", dict(nnz=-3), "ERR_CSR", "negative nnz"),
    ("A", dict(nnz=1 << 31), "ERR_UNSUPPORTED", "2^31"),
    ("A", dict(nnz=(1 << 31) - 256), "ERR_UNSUPPORTED", "2^31 - 256"),
    ("P", dict(rowptr=None), "ERR_INVALID_ARG", "NULL CSR"),
    ("A", dict(colind=None), "ERR_INVALID_ARG", "NULL CSR"),
    ("A", dict(val=None), "ERR_INVALID_ARG", "NULL CSR"),
])
def test_malformed_problems_are_refused_on_the_host(lib, parts, which, change, code, words):
    qp, hp, ha = parts
    P = _csr(hp.c, **change) if which == "P" else hp.c
    A = _csr(ha.c, **change) if which == "A" else ha.c
    q, l, u = (np.ascontiguousarray(v, dtype=np.float64) for v in (qp.q, qp.l, qp.u))
    rc, h, msg = _setup(lib, P, A, q, l, u)
    assert rc == getattr(gb, code), (rc, msg)
    assert words in msg and not h


def test_too_many_variables_and_constraints_are_refused(lib):
    """[P A'] has n + m columns and the joint vectors n + m entries, all
    indexed with 32-bit integers: n + m must stay below 2^31 - 256.  The
    arrays are not read before the sizes are checked."""
    n, m = 1_200_000_000, 1_000_000_000
    rp = np.zeros(2, np.int64)
    v = np.zeros(1)
    P = gb.Csr(n, n, 0, rp.ctypes.data, None, None)
    A = gb.Csr(m, n, 0, rp.ctypes.data, None, None)
    rc, h, msg = _setup(lib, P, A, v, v, v)
    assert rc == gb.ERR_UNSUPPORTED and "n + m" in msg and not h


def test_an_upper_triangle_whose_full_form_could_overflow_is_refused(lib):
    """The full P built from an upper triangle has up to twice its
    nonzeros, with 32-bit offsets: an upper triangle of 2^30 - 128 or more
    nonzeros is refused before any array is read."""
    rp = np.zeros(2, np.int64)
    v = np.zeros(1)
    ci = np.zeros(1, np.int32)
    P = gb.Csr(1000, 1000, 1 << 30, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    A = gb.Csr(0, 1000, 0, rp.ctypes.data, None, None)
    s = gb.default_settings()
    s.P_is_upper = 1
    rc, h, msg = _setup(lib, P, A, v, v, v, s)
    assert rc == gb.ERR_UNSUPPORTED and "upper-triangular" in msg and not h


def test_null_vectors_are_refused(lib, parts):
    qp, hp, ha = parts
    q, l, u = (np.ascontiguousarray(v, dtype=np.float64) for v in (qp.q, qp.l, qp.u))
    for args in [(None, l, u), (q, None, u), (q, l, None)]:
        rc, h, msg = _setup(lib, hp.c, ha.c, *args)
        assert rc == gb.ERR_INVALID_ARG and msg == "NULL argument" and not h


def test_empty_matrices_need_no_arrays_beyond_the_row_pointer(lib):
    """nnz = 0 allows NULL column and value arrays: the host checks accept
    them, and on a machine without a GPU the call then stops at the device."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rp_p = np.zeros(4, np.int64)
    rp_a = np.zeros(1, np.int64)
    P = gb.Csr(3, 3, 0, rp_p.ctypes.data, None, None)
    A = gb.Csr(0, 3, 0, rp_a.ctypes.data, None, None)
    q = np.ones(3)
    e = np.zeros(1)
    rc, h, msg = _setup(lib, P, A, q, e, e)
    assert rc == gb.ERR_CUDA and "cuda" in msg.lower() and not h


@pytest.mark.parametrize("bad", ["nan", "std", "clamp"])
def test_learned_policy_parameters_are_checked_on_the_host(lib, parts, bad):
    qp, hp, ha = parts
    p = np.zeros(gb.POLICY_PARAMS, np.float32)
    p[4:8] = 1.0
    p[-4] = np.log(10.0)
    if bad == "nan":
        p[100] = np.nan
    elif bad == "std":
        p[6] = 0.0
    else:
        p[-4] = 0.0
    s = gb.default_settings(rho_policy=gb.RHO_LEARNED)
    s.policy_params = p.ctypes.data
    q, l, u = (np.ascontiguousarray(v, dtype=np.float64) for v in (qp.q, qp.l, qp.u))
    rc, h, msg = _setup(lib, hp.c, ha.c, q, l, u, s)
    assert rc == gb.ERR_POLICY and "policy" in msg and not h


def test_no_gpu_means_an_error_not_a_fallback():
    """A well-formed problem on a machine without a usable GPU: the set-up
    fails with the CUDA error and names the failing call."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import __graft_entry__
    __graft_entry__.build()
    qp = qpgen.random_qp(5, 7, 0)
    with pytest.raises(gb.GbosqpError) as e:
        gb.Solver(qp)
    assert e.value.code == gb.ERR_CUDA
    assert "cudaSetDevice" in str(e.value) or "cuda" in str(e.value).lower()
