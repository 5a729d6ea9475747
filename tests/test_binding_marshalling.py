"""The binding's marshalling of device tensors, on the CPU: the pointers and
sizes it hands to the library, and the tensors it refuses (wrong element
type or length, strided, on the host or on another device), checked against
a stand-in for the library that records its calls.  Real CPU torch tensors
check the torch attributes the binding reads."""
import ctypes

import pytest

from paper_1912_04263_gb300 import binding as gb


class _Dtype:
    def __init__(self, name):
        self.name = name

    def __str__(self):
        return "torch." + self.name


class _Dev:
    def __init__(self, kind, index):
        self.type, self.index = kind, index

    def __str__(self):
        return f"{self.type}:{self.index}"


class FakeTensor:
    """What the binding reads of a torch tensor, with a chosen address."""
    _next = 0x7000_0000

    def __init__(self, dtype, numel, cuda=True, index=0, contiguous=True):
        self.dtype = _Dtype(dtype)
        self._numel, self.is_cuda, self._contig = numel, cuda, contiguous
        self.device = _Dev("cuda" if cuda else "cpu", index if cuda else None)
        FakeTensor._next += 0x1000
        self.ptr = FakeTensor._next

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return self.ptr


class FakeLib:
    """Records the calls; holds one problem of sizes n, m."""

    def __init__(self, n, m, handle=0x5000):
        self.n, self.m, self.handle = n, m, handle
        self.calls = []

    def gbosqp_default_settings(self, sref):
        s = sref._obj
        s.precision, s.device = gb.FP32, 0
        return gb.OK

    def osqp_setup(self, href, pref, aref, q, l, u, sref):
        P, A = pref._obj, aref._obj
        self.calls.append(("setup", dict(P=(P.nrows, P.ncols, P.nnz, P.rowptr, P.colind, P.val),
                                         A=(A.nrows, A.ncols, A.nnz, A.rowptr, A.colind, A.val),
                                         q=q, l=l, u=u, loc=sref._obj.input_location)))
        href._obj.value = self.handle
        return gb.OK

    def gbosqp_dims(self, h, n, m, na, npat):
        n._obj.value, m._obj.value = self.n, self.m
        return gb.OK

    def gbosqp_get_solution_device(self, h, x, y, z):
        self.calls.append(("solution", (x, y, z)))
        return gb.OK

    def gbosqp_spmv_noalloc(self, h, which, x, y):
        self.calls.append(("spmv", (which, x, y)))
        return gb.OK

    def osqp_cleanup(self, h):
        self.calls.append(("cleanup", h))


N, M, NNZ_P, NNZ_A = 7, 11, 19, 30


def _args(**bad):
    t = dict(P_rowptr=FakeTensor("int64", N + 1), P_col=FakeTensor("int32", NNZ_P),
             P_val=FakeTensor("float64", NNZ_P), A_rowptr=FakeTensor("int64", M + 1),
             A_col=FakeTensor("int32", NNZ_A), A_val=FakeTensor("float64", NNZ_A),
             q=FakeTensor("float64", N), l=FakeTensor("float64", M), u=FakeTensor("float64", M))
    t.update(bad)
    return t


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib(N, M)
    monkeypatch.setattr(gb, "_lib", f)
    monkeypatch.setattr(gb, "_PRECISION", {})
    return f


def test_setup_device_passes_the_tensors_pointers_and_sizes(fake):
    t = _args()
    h = gb.osqp_setup_device(*t.values(), N, M, gb.default_settings(precision=gb.FP64))
    assert h == fake.handle and gb._PRECISION == {h: gb.FP64}
    (kind, c), = fake.calls
    assert kind == "setup" and c["loc"] == gb.DEVICE
    assert c["P"] == (N, N, NNZ_P, t["P_rowptr"].ptr, t["P_col"].ptr, t["P_val"].ptr)
    assert c["A"] == (M, N, NNZ_A, t["A_rowptr"].ptr, t["A_col"].ptr, t["A_val"].ptr)
    assert (c["q"], c["l"], c["u"]) == (t["q"].ptr, t["l"].ptr, t["u"].ptr)
    gb.osqp_cleanup(h)
    assert gb._PRECISION == {} and fake.calls[-1] == ("cleanup", h)


@pytest.mark.parametrize("bad,err,words", [
    (dict(P_rowptr=FakeTensor("int32", N + 1)), TypeError, "P_rowptr: expected a int64"),
    (dict(A_col=FakeTensor("int64", NNZ_A)), TypeError, "A_col: expected a int32"),
    (dict(q=FakeTensor("float32", N)), TypeError, "q: expected a float64"),
    (dict(A_rowptr=FakeTensor("int64", M)), ValueError, "A_rowptr: expected 12 elements"),
    (dict(P_col=FakeTensor("int32", NNZ_P - 1)), ValueError, "P_col: expected 19 elements"),
    (dict(u=FakeTensor("float64", M + 1)), ValueError, "u: expected 11 elements"),
    (dict(l=FakeTensor("float64", M, contiguous=False)), ValueError, "contiguous"),
    (dict(A_val=FakeTensor("float64", NNZ_A, cuda=False)), ValueError, "CUDA tensor"),
    (dict(P_val=FakeTensor("float64", NNZ_P, index=1)), ValueError, "on cuda:1"),
])
def test_setup_device_refuses_tensors_the_kernels_would_misread(fake, bad, err, words):
    with pytest.raises(err, match=words):
        gb.osqp_setup_device(*_args(**bad).values(), N, M)
    assert fake.calls == []


def test_setup_device_checks_the_settings_device(fake):
    s = gb.default_settings()
    s.device = 2
    with pytest.raises(ValueError, match="the solver runs on cuda:2"):
        gb.osqp_setup_device(*_args().values(), N, M, s)
    t = {k: FakeTensor(v.dtype.name, v.numel(), index=2) for k, v in _args().items()}
    gb.osqp_setup_device(*t.values(), N, M, s)
    assert fake.calls[0][0] == "setup"


def test_solution_device_sizes_follow_the_handle(fake):
    x, y, z = FakeTensor("float64", N), FakeTensor("float64", M), FakeTensor("float64", M)
    gb.gbosqp_get_solution_device(fake.handle, x, y, z)
    assert fake.calls == [("solution", (x.ptr, y.ptr, z.ptr))]
    with pytest.raises(ValueError, match="z: expected 11"):
        gb.gbosqp_get_solution_device(fake.handle, x, y, FakeTensor("float64", N))
    with pytest.raises(TypeError, match="x: expected a float64"):
        gb.gbosqp_get_solution_device(fake.handle, FakeTensor("float32", N), y, z)


@pytest.mark.parametrize("prec,dt,other", [(gb.FP32, "float32", "float64"), (gb.FP64, "float64", "float32")])
def test_noalloc_spmv_takes_the_handles_precision_and_shapes(fake, prec, dt, other):
    h = gb.osqp_setup_device(*_args().values(), N, M, gb.default_settings(precision=prec))
    fake.calls.clear()
    for which, nin, nout in [(gb.MAT_A, N, M), (gb.MAT_PAT, N + M, N)]:
        x, y = FakeTensor(dt, nin), FakeTensor(dt, nout)
        gb.gbosqp_spmv_noalloc(h, which, x, y)
        assert fake.calls[-1] == ("spmv", (which, x.ptr, y.ptr))
        with pytest.raises(TypeError):
            gb.gbosqp_spmv_noalloc(h, which, FakeTensor(other, nin), FakeTensor(other, nout))
        with pytest.raises(ValueError, match="y: expected"):
            gb.gbosqp_spmv_noalloc(h, which, x, FakeTensor(dt, nout + 1))
    assert len(fake.calls) == 2


def test_noalloc_spmv_on_an_unregistered_handle_takes_either_float_type(fake):
    for dt in ("float32", "float64"):
        gb.gbosqp_spmv_noalloc(0x6000, gb.MAT_A, FakeTensor(dt, N), FakeTensor(dt, M))
    with pytest.raises(TypeError, match="float32 or float64"):
        gb.gbosqp_spmv_noalloc(0x6000, gb.MAT_A, FakeTensor("int32", N), FakeTensor("int32", M))
    with pytest.raises(TypeError, match="y: expected a float32"):
        gb.gbosqp_spmv_noalloc(0x6000, gb.MAT_A, FakeTensor("float32", N), FakeTensor("float64", M))


def test_real_torch_tensors_pass_the_type_and_length_checks(fake):
    """The attribute names and the dtype spelling match torch: a CPU tensor of
    the right type and length gets as far as the device check."""
    torch = pytest.importorskip("torch")
    ok = dict(P_rowptr=torch.zeros(N + 1, dtype=torch.int64), P_col=torch.zeros(NNZ_P, dtype=torch.int32),
              P_val=torch.zeros(NNZ_P, dtype=torch.float64), A_rowptr=torch.zeros(M + 1, dtype=torch.int64),
              A_col=torch.zeros(NNZ_A, dtype=torch.int32), A_val=torch.zeros(NNZ_A, dtype=torch.float64),
              q=torch.zeros(N, dtype=torch.float64), l=torch.zeros(M, dtype=torch.float64),
              u=torch.zeros(M, dtype=torch.float64))
    with pytest.raises(ValueError, match="P_rowptr: expected a CUDA tensor, got one on cpu"):
        gb.osqp_setup_device(*ok.values(), N, M)
    with pytest.raises(TypeError, match="P_rowptr: expected a int64 tensor, got int32"):
        gb.osqp_setup_device(*dict(ok, P_rowptr=ok["P_rowptr"].int()).values(), N, M)
    strided = torch.zeros(2 * (N + 1), dtype=torch.int64)[::2]
    with pytest.raises(ValueError, match="contiguous"):
        gb.osqp_setup_device(*dict(ok, P_rowptr=strided).values(), N, M)
    assert fake.calls == []
    assert isinstance(gb.Csr().nnz, int) and ctypes.sizeof(gb.Csr) == 40
