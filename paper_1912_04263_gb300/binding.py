"""ctypes binding of libgbosqp.so (declared in include/gbosqp.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  The functions keep the C names (``osqp_setup``,
``osqp_solve``, ...); ``Solver`` is a small owner of one handle.  Importing
this module loads the library and raises if it is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbosqp.so")

OK = 0
ERR_INVALID_ARG, ERR_DIMENSION, ERR_CSR, ERR_BOUNDS, ERR_NONFINITE = -1, -2, -3, -4, -5
ERR_CUDA, ERR_OOM, ERR_DEVICE_TIMEOUT, ERR_UNSUPPORTED, ERR_POLICY = -6, -7, -8, -9, -10
SOLVED, MAX_ITER, NONFINITE, PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 1, 2, 3, 4, 5
FP32, FP64 = 0, 1
RHO_RATIO, RHO_LEARNED, RHO_FIXED = 0, 1, 2
HOST, DEVICE = 0, 1
LOOP_GRAPH, LOOP_HOST = 0, 1
PCG_CLASSIC, PCG_SINGLE_REDUCTION = 0, 1
MAT_A, MAT_PAT = 0, 1
CHECK_FIELDS = 16
POLICY_PARAMS = 4622
INFINITY = 1e20


class Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Settings(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("sigma", ctypes.c_double), ("rho0", ctypes.c_double),
                ("eps_abs", ctypes.c_double), ("eps_rel", ctypes.c_double), ("pcg_lambda", ctypes.c_double),
                ("pcg_eps_min", ctypes.c_double), ("rho_min", ctypes.c_double), ("rho_max", ctypes.c_double),
                ("eps_prim_inf", ctypes.c_double), ("eps_dual_inf", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("max_cg_iter", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("rho_every", ctypes.c_int32), ("scaling_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rho_policy", ctypes.c_int32), ("P_is_upper", ctypes.c_int32), ("input_location", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("device", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("rho_vector", ctypes.c_int32), ("pcg_variant", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("policy_params", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("pcg_iters", ctypes.c_int64),
                ("obj", ctypes.c_double), ("r_prim", ctypes.c_double), ("r_dual", ctypes.c_double),
                ("eps_prim", ctypes.c_double), ("eps_dual", ctypes.c_double), ("rho", ctypes.c_double),
                ("pcg_eps", ctypes.c_double), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("rho_updates", ctypes.c_int32), ("policy_fallbacks", ctypes.c_int32),
                ("nnz_P", ctypes.c_int64), ("nnz_A", ctypes.c_int64),
                ("setup_launches", ctypes.c_int64), ("solve_launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_PRECISION: dict = {}  # working precision of each live handle made through this module


def lib():
    """Load libgbosqp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "gbosqp_default_settings": (i32, [ctypes.POINTER(Settings)]),
        "osqp_setup": (i32, [ctypes.POINTER(_P), ctypes.POINTER(Csr), ctypes.POINTER(Csr), _P, _P, _P,
                             ctypes.POINTER(Settings)]),
        "osqp_solve": (i32, [_P]),
        "osqp_update_rho": (i32, [_P, dbl]),
        "osqp_warm_start": (i32, [_P, _P, _P]),
        "osqp_get_solution": (i32, [_P, _P, _P, _P]),
        "gbosqp_get_solution_device": (i32, [_P, _P, _P, _P]),
        "osqp_get_info": (i32, [_P, ctypes.POINTER(Info)]),
        "osqp_cleanup": (None, [_P]),
        "gbosqp_last_error": (ctypes.c_char_p, [_P]),
        "gbosqp_setup_error": (ctypes.c_char_p, []),
        "gbosqp_error_string": (ctypes.c_char_p, [i32]),
        "gbosqp_dims": (i32, [_P, _P, _P, _P, _P]),
        "gbosqp_get_scaling": (i32, [_P, _P, _P, _P]),
        "gbosqp_get_scaled_csr": (i32, [_P, i32, _P, _P, _P]),
        "gbosqp_spmv": (i32, [_P, i32, _P, _P, i32]),
        "gbosqp_pcg": (i32, [_P, dbl, _P, _P, dbl, i32, _P, _P, _P]),
        "gbosqp_set_iterates": (i32, [_P, _P, _P, _P, _P, dbl]),
        "gbosqp_get_iterates": (i32, [_P, _P, _P, _P, _P, _P]),
        "gbosqp_admm_iterations": (i32, [_P, i32, _P]),
        "gbosqp_check": (i32, [_P, _P]),
        "gbosqp_bench_kernel": (i32, [_P, i32, i32, _P]),
        "gbosqp_spmv_noalloc": (i32, [_P, i32, _P, _P]),
        "gbosqp_policy_forward": (i32, [_P, _P, i32, _P]),
        "gbosqp_mlp_grad": (i32, [_P, _P, _P, _P, i32, _P, _P]),
        "gbosqp_mlp_train": (i32, [_P, _P, _P, _P, i32, _P, i32, i32, ctypes.c_float, _P]),
        "gbosqp_set_pcg_lambda": (i32, [_P, dbl, dbl]),
        "osqp_update_lin_cost": (i32, [_P, _P]),
        "gbosqp_resume": (i32, [_P]),
        "osqp_update_bounds": (i32, [_P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a) -> int:
    return a.ctypes.data if a is not None else 0


def _vec(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.shape != (n,):
        raise ValueError(f"expected a vector of length {n}, got shape {a.shape}")
    return a


class GbosqpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{code} ({error_string(code)}): {msg}")
        self.code = code


def error_string(code: int) -> str:
    return lib().gbosqp_error_string(code).decode()


def default_settings(**overrides) -> Settings:
    s = Settings()
    lib().gbosqp_default_settings(ctypes.byref(s))
    for k, v in overrides.items():
        if not hasattr(s, k):
            raise AttributeError(k)
        setattr(s, k, v)
    return s


class _HostCsr:
    """Host CSR arrays kept alive while the C struct points at them."""

    def __init__(self, M):
        import scipy.sparse as sp
        M = sp.csr_matrix(M)
        M.sort_indices()
        self.rowptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
        self.col = np.ascontiguousarray(M.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(M.data, dtype=np.float64)
        self.c = Csr(M.shape[0], M.shape[1], int(M.nnz), _ptr(self.rowptr), _ptr(self.col), _ptr(self.val))


def osqp_setup(P, A, q, l, u, settings: Settings | None = None, P_is_upper: bool | None = None):
    """Set up a problem from host data (scipy sparse P, A; numpy q, l, u).
    P may be full or its upper triangle; by default the full matrix is
    passed with P_is_upper = 0.  Returns an opaque handle (int)."""
    import scipy.sparse as sp
    s = settings if settings is not None else default_settings()
    if P_is_upper is None:
        P_is_upper = False
    s.P_is_upper = 1 if P_is_upper else 0
    Pm = sp.triu(P, format="csr") if P_is_upper else P
    hp, ha = _HostCsr(Pm), _HostCsr(A)
    n, m = hp.c.nrows, ha.c.nrows
    qv, lv, uv = _vec(q, n), _vec(l, m), _vec(u, m)
    lv = np.where(np.isneginf(lv), -INFINITY, lv)
    uv = np.where(np.isposinf(uv), INFINITY, uv)
    s.input_location = HOST
    h = ctypes.c_void_p()
    rc = lib().osqp_setup(ctypes.byref(h), ctypes.byref(hp.c), ctypes.byref(ha.c), _ptr(qv), _ptr(lv), _ptr(uv),
                          ctypes.byref(s))
    if rc != OK:
        raise GbosqpError(rc, lib().gbosqp_setup_error().decode())
    _PRECISION[h.value] = int(s.precision)
    return h.value


def _device_ptr(t, name: str, dtype: str, numel: int, device: int | None = None) -> int:
    """Data pointer of a torch tensor that the library reads or writes as
    numel contiguous elements of dtype in CUDA device memory.  The library
    cannot see the extent of a device buffer, so a tensor of another element
    type, on the host, strided, of another length or on another device than
    the handle's is refused here rather than misread by the kernels."""
    got = str(t.dtype).replace("torch.", "")
    if got != dtype:
        raise TypeError(f"{name}: expected a {dtype} tensor, got {got}")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: the tensor must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor, got one on {t.device}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name}: on cuda:{t.device.index}, the solver runs on cuda:{device}")
    return t.data_ptr()


def osqp_setup_device(P_rowptr, P_col, P_val, A_rowptr, A_col, A_val, q, l, u, n: int, m: int,
                      settings: Settings | None = None, P_is_upper: bool = False):
    """Set up from device-resident arrays (contiguous torch tensors on the
    settings' CUDA device: int64 row pointers of n + 1 and m + 1 entries,
    int32 column indices and float64 values of nnz entries each, float64 q
    of n and l, u of m entries; infinite bounds as +-1e20)."""
    s = settings if settings is not None else default_settings()
    s.P_is_upper = 1 if P_is_upper else 0
    s.input_location = DEVICE
    d = s.device
    nnz_p, nnz_a = int(P_val.numel()), int(A_val.numel())
    cp = Csr(n, n, nnz_p, _device_ptr(P_rowptr, "P_rowptr", "int64", n + 1, d),
             _device_ptr(P_col, "P_col", "int32", nnz_p, d), _device_ptr(P_val, "P_val", "float64", nnz_p, d))
    ca = Csr(m, n, nnz_a, _device_ptr(A_rowptr, "A_rowptr", "int64", m + 1, d),
             _device_ptr(A_col, "A_col", "int32", nnz_a, d), _device_ptr(A_val, "A_val", "float64", nnz_a, d))
    qp_, lp, up = (_device_ptr(q, "q", "float64", n, d), _device_ptr(l, "l", "float64", m, d),
                   _device_ptr(u, "u", "float64", m, d))
    h = ctypes.c_void_p()
    rc = lib().osqp_setup(ctypes.byref(h), ctypes.byref(cp), ctypes.byref(ca), qp_, lp, up, ctypes.byref(s))
    if rc != OK:
        raise GbosqpError(rc, lib().gbosqp_setup_error().decode())
    _PRECISION[h.value] = int(s.precision)
    return h.value


def _check(h, rc):
    if rc < 0:
        raise GbosqpError(rc, lib().gbosqp_last_error(h).decode())
    return rc


def osqp_solve(h) -> int:
    return _check(h, lib().osqp_solve(h))


def osqp_update_rho(h, rho: float) -> None:
    _check(h, lib().osqp_update_rho(h, float(rho)))


def osqp_warm_start(h, x=None, y=None) -> None:
    n, m = dims(h)[:2]
    xv = None if x is None else _vec(x, n)
    yv = None if y is None else _vec(y, m)
    _check(h, lib().osqp_warm_start(h, _ptr(xv), _ptr(yv)))


def gbosqp_resume(h) -> None:
    """The next solve continues from the current iterates, rho, PCG
    tolerance and lambda."""
    _check(h, lib().gbosqp_resume(h))


def osqp_update_lin_cost(h, q) -> None:
    """Replace q (host array) keeping the set-up's equilibration."""
    n = dims(h)[0]
    qv = _vec(q, n)
    _check(h, lib().osqp_update_lin_cost(h, _ptr(qv)))


def osqp_update_bounds(h, l=None, u=None) -> None:
    """Replace l and/or u (host arrays; None keeps that side)."""
    m = dims(h)[1]
    lv = None if l is None else _vec(l, m)
    uv = None if u is None else _vec(u, m)
    _check(h, lib().osqp_update_bounds(h, _ptr(lv), _ptr(uv)))


def dims(h):
    n, m = ctypes.c_int32(), ctypes.c_int32()
    na, npat = ctypes.c_int64(), ctypes.c_int64()
    _check(h, lib().gbosqp_dims(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(na), ctypes.byref(npat)))
    return n.value, m.value, na.value, npat.value


def osqp_get_solution(h):
    n, m = dims(h)[:2]
    x, y, z = np.empty(n), np.empty(m), np.empty(m)
    _check(h, lib().osqp_get_solution(h, _ptr(x), _ptr(y), _ptr(z)))
    return x, y, z


def gbosqp_get_solution_device(h, x, y, z) -> None:
    """Copy the solution into device tensors (contiguous float64 CUDA
    tensors of n, m and m entries)."""
    n, m = dims(h)[:2]
    _check(h, lib().gbosqp_get_solution_device(h, _device_ptr(x, "x", "float64", n), _device_ptr(y, "y", "float64", m),
                                               _device_ptr(z, "z", "float64", m)))


def osqp_get_info(h) -> dict:
    info = Info()
    _check(h, lib().osqp_get_info(h, ctypes.byref(info)))
    return info.as_dict()


def osqp_cleanup(h) -> None:
    if h:
        _PRECISION.pop(h, None)
        lib().osqp_cleanup(h)


def gbosqp_get_scaling(h):
    n, m = dims(h)[:2]
    D, E, c = np.empty(n), np.empty(m), ctypes.c_double()
    _check(h, lib().gbosqp_get_scaling(h, _ptr(D), _ptr(E), ctypes.byref(c)))
    return D, E, c.value


def gbosqp_get_scaled_csr(h, which: int):
    import scipy.sparse as sp
    n, m, na, npat = dims(h)
    nr, nc, nnz = (m, n, na) if which == MAT_A else (n, n + m, npat)
    rp = np.empty(nr + 1, np.int64)
    col = np.empty(max(nnz, 1), np.int32)
    val = np.empty(max(nnz, 1), np.float64)
    _check(h, lib().gbosqp_get_scaled_csr(h, which, _ptr(rp), _ptr(col), _ptr(val)))
    return sp.csr_matrix((val[:nnz], col[:nnz], rp), shape=(nr, nc))


def gbosqp_spmv(h, which: int, x, fp64_accumulate: bool = False) -> np.ndarray:
    n, m = dims(h)[:2]
    nin, nout = (n, m) if which == MAT_A else (n + m, n)
    xv = _vec(x, nin)
    y = np.empty(nout)
    _check(h, lib().gbosqp_spmv(h, which, _ptr(xv), _ptr(y), 1 if fp64_accumulate else 0))
    return y


def gbosqp_pcg(h, rho: float, b, x0, eps: float, max_iter: int):
    n = dims(h)[0]
    bv, xv = _vec(b, n), _vec(x0, n)
    x = np.empty(n)
    it, rn = ctypes.c_int32(), ctypes.c_double()
    _check(h, lib().gbosqp_pcg(h, float(rho), _ptr(bv), _ptr(xv), float(eps), int(max_iter), _ptr(x),
                               ctypes.byref(it), ctypes.byref(rn)))
    return x, it.value, rn.value


def gbosqp_set_iterates(h, x, z, y, xt, rho: float) -> None:
    n, m = dims(h)[:2]
    _check(h, lib().gbosqp_set_iterates(h, _ptr(_vec(x, n)), _ptr(_vec(z, m)), _ptr(_vec(y, m)),
                                        _ptr(_vec(xt, n)), float(rho)))


def gbosqp_get_iterates(h):
    n, m = dims(h)[:2]
    x, z, y, xt, rho = np.empty(n), np.empty(m), np.empty(m), np.empty(n), ctypes.c_double()
    _check(h, lib().gbosqp_get_iterates(h, _ptr(x), _ptr(z), _ptr(y), _ptr(xt), ctypes.byref(rho)))
    return x, z, y, xt, rho.value


def gbosqp_admm_iterations(h, k: int):
    per = np.zeros(max(k, 1), np.int32)
    st = _check(h, lib().gbosqp_admm_iterations(h, int(k), per.ctypes.data))
    return st, per[:k]


(K_PCG_DIRECTION, K_PCG_KAPPLY, K_PCG_UPDATE, K_PCG_INIT, K_ADMM_UPDATE, K_CHECK_A, K_CHECK_B, K_INF_A,
 K_INF_B, K_PCG_SR_DIRECTION, K_PCG_SR_KAPPLY) = range(11)


def gbosqp_bench_kernel(h, kernel: int, reps: int) -> float:
    """Mean duration (ms) of one solve kernel, timed with CUDA events."""
    ms = ctypes.c_double()
    _check(h, lib().gbosqp_bench_kernel(h, int(kernel), int(reps), ctypes.byref(ms)))
    return ms.value


def gbosqp_spmv_noalloc(h, which: int, x, y) -> None:
    """y = M x on device tensors of the handle's working precision (float32
    for FP32, float64 for FP64; x of n entries and y of m for MAT_A, x of
    n + m and y of n for MAT_PAT), without any device allocation in the call
    (asynchronous on the handle's stream)."""
    n, m = dims(h)[:2]
    nin, nout = (n, m) if which == MAT_A else (n + m, n)
    prec = _PRECISION.get(h)
    if prec is None:  # a handle made by a direct library call: take the tensor's type
        dt = str(x.dtype).replace("torch.", "")
        if dt not in ("float32", "float64"):
            raise TypeError(f"x: expected a float32 or float64 tensor, got {dt}")
    else:
        dt = "float32" if prec == FP32 else "float64"
    _check(h, lib().gbosqp_spmv_noalloc(h, int(which), _device_ptr(x, "x", dt, nin), _device_ptr(y, "y", dt, nout)))


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _rc(rc):
    if rc != OK:
        raise GbosqpError(rc, error_string(rc))


def gbosqp_policy_forward(params, features) -> np.ndarray:
    p = _f32(params, (POLICY_PARAMS,))
    f = _f32(features)
    f = f.reshape(-1, 4)
    out = np.empty((f.shape[0], 2), np.float32)
    _rc(lib().gbosqp_policy_forward(p.ctypes.data, f.ctypes.data, f.shape[0], out.ctypes.data))
    return out


def gbosqp_mlp_grad(params, features, targets, weights):
    p = _f32(params, (POLICY_PARAMS,))
    f = _f32(features).reshape(-1, 4)
    n = f.shape[0]
    t = _f32(targets, (n, 2))
    w = _f32(weights, (n, 2))
    g = np.zeros(POLICY_PARAMS, np.float32)
    loss = np.zeros(1, np.float32)
    _rc(lib().gbosqp_mlp_grad(p.ctypes.data, f.ctypes.data, t.ctypes.data, w.ctypes.data, n, g.ctypes.data,
                              loss.ctypes.data))
    return g, float(loss[0])


def gbosqp_mlp_train(params, features, targets, weights, batches, lr: float):
    """Adam on the device; batches: (steps, batch) int array of sample indices.
    Returns (new params, loss per step)."""
    p = _f32(params, (POLICY_PARAMS,)).copy()
    f = _f32(features).reshape(-1, 4)
    n = f.shape[0]
    t = _f32(targets, (n, 2))
    w = _f32(weights, (n, 2))
    b = np.ascontiguousarray(np.asarray(batches, dtype=np.int32))
    steps, bs = b.shape
    hist = np.zeros(max(steps, 1), np.float32)
    _rc(lib().gbosqp_mlp_train(p.ctypes.data, f.ctypes.data, t.ctypes.data, w.ctypes.data, n, b.ctypes.data, steps,
                               bs, ctypes.c_float(lr), hist.ctypes.data))
    return p, hist[:steps]


def gbosqp_set_pcg_lambda(h, lam: float, eps: float) -> None:
    _check(h, lib().gbosqp_set_pcg_lambda(h, float(lam), float(eps)))


POLICY_MAGIC = b"GBRHOPOL"


def save_policy(path: str, params) -> None:
    """Write policy parameters: 8-byte magic, count (uint32), CRC32 of the
    float32 payload (uint32), payload (little-endian float32)."""
    import zlib
    p = _f32(params, (POLICY_PARAMS,)).astype("<f4")
    payload = p.tobytes()
    with open(path, "wb") as fh:
        fh.write(POLICY_MAGIC + np.uint32(POLICY_PARAMS).tobytes() + np.uint32(zlib.crc32(payload)).tobytes() + payload)


def load_policy(path: str) -> np.ndarray:
    import zlib
    with open(path, "rb") as fh:
        raw = fh.read()
    if raw[:8] != POLICY_MAGIC:
        raise ValueError(f"{path}: not a policy file")
    count = int(np.frombuffer(raw[8:12], "<u4")[0])
    crc = int(np.frombuffer(raw[12:16], "<u4")[0])
    payload = raw[16:]
    if count != POLICY_PARAMS or len(payload) != 4 * count or zlib.crc32(payload) != crc:
        raise ValueError(f"{path}: corrupt policy file")
    return np.frombuffer(payload, "<f4").astype(np.float32).copy()


CHECK_NAMES = ["r_prim", "r_dual", "eps_prim", "eps_dual", "r_prim_s", "r_dual_s", "norm_Ax_s", "norm_z_s",
               "norm_Px_s", "norm_Aty_s", "norm_q_s", "obj", "rho_ratio", "lambda", "stall_count", "fallbacks"]


def gbosqp_check(h) -> dict:
    out = np.zeros(CHECK_FIELDS)
    _check(h, lib().gbosqp_check(h, _ptr(out)))
    return dict(zip(CHECK_NAMES, out[:len(CHECK_NAMES)].tolist()))


class Solver:
    """Owner of one solver handle."""

    def __init__(self, qp=None, *, P=None, q=None, A=None, l=None, u=None, P_is_upper=False, **settings):
        if qp is not None:
            P, q, A, l, u = qp.P, qp.q, qp.A, qp.l, qp.u
        policy = settings.pop("policy_params", None)
        s = default_settings(**settings)
        self._policy = None
        if policy is not None:
            self._policy = np.ascontiguousarray(np.asarray(policy, np.float32))
            if self._policy.size != POLICY_PARAMS:
                raise ValueError(f"policy_params must have {POLICY_PARAMS} floats")
            s.policy_params = self._policy.ctypes.data
        self.h = osqp_setup(P, A, q, l, u, s, P_is_upper=P_is_upper)
        self.n, self.m = dims(self.h)[:2]

    def solve(self) -> int:
        return osqp_solve(self.h)

    def solution(self):
        return osqp_get_solution(self.h)

    def info(self) -> dict:
        return osqp_get_info(self.h)

    def update_rho(self, rho: float):
        osqp_update_rho(self.h, rho)

    def warm_start(self, x=None, y=None):
        osqp_warm_start(self.h, x, y)

    def update_lin_cost(self, q):
        osqp_update_lin_cost(self.h, q)

    def update_bounds(self, l=None, u=None):
        osqp_update_bounds(self.h, l, u)

    def close(self):
        if getattr(self, "h", None):
            osqp_cleanup(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
