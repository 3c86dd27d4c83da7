"""Python binding of libsylv, the GB300 factorized Krylov solver for A X + X B = C1 C2^T.

Argument marshalling only: every step of the solve runs in the CUDA kernels of
``lib/libsylv.so`` behind the C ABI declared in ``include/sylv.h``.  The
functions keep the C names (``sylv_create``, ``sylv_cg``, ``sylv_bicgstab``, ``sylv_cgs``, ``sylv_cr``, ``sylv_gpbicg``,
``sylv_get_factors``, ``sylv_get_history``, ``sylv_get_hessenberg``,
``sylv_apply``, ``sylv_destroy``); ``Solver`` wraps a handle.

There is no fallback: if the library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsylv.so")

SYLV_OK, SYLV_EINVAL, SYLV_ENOMEM, SYLV_ENOTCONV, SYLV_EBREAKDOWN = 0, 1, 2, 3, 4
SYLV_ENONFINITE, SYLV_ETIMEOUT, SYLV_ECUDA, SYLV_ESTATE = 5, 6, 7, 8
SYLV_FP64, SYLV_MIXED = 0, 1
STATUS_NAMES = {0: "converged", 1: "einval", 2: "enomem", 3: "maxit", 4: "breakdown", 5: "nonfinite",
                6: "timeout", 7: "ecuda", 8: "estate"}

# every symbol include/sylv.h declares
EXPORTS = ["sylv_default_options", "sylv_create", "sylv_cg", "sylv_bicgstab", "sylv_cgs", "sylv_cr",
           "sylv_gpbicg", "sylv_compress", "sylv_get_factors",
           "sylv_get_history", "sylv_get_hessenberg", "sylv_small_operator", "sylv_set_timeout", "sylv_apply", "sylv_get_profile", "sylv_spmm_noalloc",
           "sylv_create_batch", "sylv_batch_instance", "sylv_strerror", "sylv_last_error", "sylv_destroy"]


class sylv_csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)), ("col_idx", ctypes.POINTER(ctypes.c_int32)),
                ("val", ctypes.POINTER(ctypes.c_double))]


class sylv_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("lyapunov", ctypes.c_int32), ("poll_every", ctypes.c_int32),
                ("refine_max", ctypes.c_int32), ("deflate_tol", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("no_true_residual", ctypes.c_int32), ("stream_mode", ctypes.c_int32), ("small_gemm", ctypes.c_int32),
                ("basis_gemm", ctypes.c_int32), ("stop_margin", ctypes.c_double), ("cert_gemm", ctypes.c_int32)]


class sylv_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class sylv_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("matvecs", ctypes.c_int64),
                ("width", ctypes.c_int64), ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("refinements", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("true_rel_bound", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["status_name"] = STATUS_NAMES.get(self.status, "unknown")
        return d


_lib = None


class SylvError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({last_error()})")


def load(path: Optional[str] = None):
    """Load libsylv.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"{p} not found: build it with `python -m paper_2605_28274_gb300.build`")
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    lib.sylv_default_options.argtypes = [P(sylv_options)]
    lib.sylv_default_options.restype = None
    lib.sylv_create.argtypes = [P(sylv_csr), P(sylv_csr), dp, dp, ctypes.c_int64, P(sylv_options),
                                P(ctypes.c_void_p)]
    lib.sylv_create.restype = ctypes.c_int
    for f in ("sylv_cg", "sylv_bicgstab", "sylv_cgs", "sylv_cr", "sylv_gpbicg"):
        getattr(lib, f).argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, P(sylv_info)]
        getattr(lib, f).restype = ctypes.c_int
    lib.sylv_compress.argtypes = [ctypes.c_void_p, ctypes.c_double, P(ctypes.c_int64)]
    lib.sylv_compress.restype = ctypes.c_int
    lib.sylv_get_factors.argtypes = [ctypes.c_void_p, dp, dp, dp, P(ctypes.c_int64)]
    lib.sylv_get_factors.restype = ctypes.c_int
    lib.sylv_get_history.argtypes = [ctypes.c_void_p, dp, ctypes.c_int64, P(ctypes.c_int64)]
    lib.sylv_get_history.restype = ctypes.c_int
    lib.sylv_get_hessenberg.argtypes = [ctypes.c_void_p, ctypes.c_int32, dp, ctypes.c_int64, P(ctypes.c_int32)]
    lib.sylv_get_hessenberg.restype = ctypes.c_int
    lib.sylv_small_operator.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp, dp]
    lib.sylv_small_operator.restype = ctypes.c_int
    lib.sylv_set_timeout.argtypes = [ctypes.c_void_p, ctypes.c_double]
    lib.sylv_set_timeout.restype = ctypes.c_int
    lib.sylv_apply.argtypes = [ctypes.c_void_p, ctypes.c_int32, dp, dp, ctypes.c_int64]
    lib.sylv_apply.restype = ctypes.c_int
    lib.sylv_get_profile.argtypes = [ctypes.c_void_p, P(sylv_kernel_stat), ctypes.c_int32, P(ctypes.c_int32)]
    lib.sylv_get_profile.restype = ctypes.c_int
    lib.sylv_spmm_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p]
    lib.sylv_spmm_noalloc.restype = ctypes.c_int
    lib.sylv_create_batch.argtypes = [ctypes.c_int32, P(sylv_csr), P(sylv_csr), P(dp), P(dp), P(ctypes.c_int64),
                                      P(sylv_options), P(ctypes.c_void_p)]
    lib.sylv_create_batch.restype = ctypes.c_int
    lib.sylv_batch_instance.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_void_p)]
    lib.sylv_batch_instance.restype = ctypes.c_int
    lib.sylv_strerror.argtypes = [ctypes.c_int]
    lib.sylv_strerror.restype = ctypes.c_char_p
    lib.sylv_last_error.argtypes = []
    lib.sylv_last_error.restype = ctypes.c_char_p
    lib.sylv_destroy.argtypes = [ctypes.c_void_p]
    lib.sylv_destroy.restype = None
    if path is None:
        _lib = lib
    return lib


def last_error() -> str:
    if _lib is None:
        return ""
    return (_lib.sylv_last_error() or b"").decode()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _csr_arrays(M):
    """(nrows, row_ptr, col_idx, val) from an object with row_ptr/col_idx/val or a scipy CSR."""
    if hasattr(M, "row_ptr"):
        rp, ci, v, n = M.row_ptr, M.col_idx, M.val, M.nrows
    else:
        rp, ci, v, n = M.indptr, M.indices, M.data, M.shape[0]
    return (int(n), np.ascontiguousarray(rp, dtype=np.int32), np.ascontiguousarray(ci, dtype=np.int32),
            np.ascontiguousarray(v, dtype=np.float64))


def _make_csr(M):
    n, rp, ci, v = _csr_arrays(M)
    c = sylv_csr(n, n, int(ci.shape[0]), rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                 ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(v))
    return c, (rp, ci, v)


def sylv_default_options() -> sylv_options:
    o = sylv_options()
    load().sylv_default_options(ctypes.byref(o))
    return o


def sylv_create(A, B, C1: np.ndarray, C2: Optional[np.ndarray], opt: Optional[sylv_options] = None):
    """Returns a handle (c_void_p).  C1, C2 are (n, s), (m, s) arrays; B = C2 = None with opt.lyapunov."""
    lib = load()
    ca, keep_a = _make_csr(A)
    cb, keep_b = (None, None) if B is None else _make_csr(B)
    C1f = np.asfortranarray(C1, dtype=np.float64)
    C2f = None if C2 is None else np.asfortranarray(C2, dtype=np.float64)
    s = C1f.shape[1]
    h = ctypes.c_void_p()
    rc = lib.sylv_create(ctypes.byref(ca), None if cb is None else ctypes.byref(cb), _dptr(C1f),
                         None if C2f is None else _dptr(C2f), s, None if opt is None else ctypes.byref(opt),
                         ctypes.byref(h))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_create")
    return h


def sylv_cg(h, tol: float, maxit: int) -> sylv_info:
    info = sylv_info()
    load().sylv_cg(h, tol, maxit, ctypes.byref(info))
    return info


def sylv_bicgstab(h, tol: float, maxit: int) -> sylv_info:
    info = sylv_info()
    load().sylv_bicgstab(h, tol, maxit, ctypes.byref(info))
    return info


def sylv_cgs(h, tol: float, maxit: int) -> sylv_info:
    info = sylv_info()
    load().sylv_cgs(h, tol, maxit, ctypes.byref(info))
    return info


def sylv_cr(h, tol: float, maxit: int) -> sylv_info:
    info = sylv_info()
    load().sylv_cr(h, tol, maxit, ctypes.byref(info))
    return info


def sylv_gpbicg(h, tol: float, maxit: int) -> sylv_info:
    info = sylv_info()
    load().sylv_gpbicg(h, tol, maxit, ctypes.byref(info))
    return info


def sylv_compress(h, tol: float) -> int:
    q = ctypes.c_int64(0)
    rc = load().sylv_compress(h, tol, ctypes.byref(q))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_compress")
    return int(q.value)


def sylv_get_factors(h, n: int, m: int, want=("V", "X", "W"), out=None):
    """V (n x r), X^ (r x r), W (m x r) as Fortran-ordered float64 arrays.

    ``out`` may map "V"/"X"/"W" to preallocated arrays (e.g. views of pinned
    host memory) with room for at least that many elements; they are filled
    in column-major order and returned reshaped."""
    lib = load()
    r = ctypes.c_int64()
    rc = lib.sylv_get_factors(h, None, None, None, ctypes.byref(r))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_factors")
    r = r.value
    out = out or {}

    def buf(key, rows, cols):
        if key not in want:
            return None
        if key in out:
            flat = out[key].reshape(-1)
            assert flat.dtype == np.float64 and flat.size >= rows * cols
            return flat[: rows * cols].reshape((rows, cols), order="F")
        return np.empty((rows, cols), order="F")

    V, X, W = buf("V", n, r), buf("X", r, r), buf("W", m, r)
    rc = lib.sylv_get_factors(h, None if V is None else _dptr(V), None if X is None else _dptr(X),
                              None if W is None else _dptr(W), None)
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_factors")
    return V, X, W


def sylv_get_history(h) -> np.ndarray:
    lib = load()
    L = ctypes.c_int64()
    rc = lib.sylv_get_history(h, None, 0, ctypes.byref(L))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_history")
    out = np.empty(L.value)
    rc = lib.sylv_get_history(h, _dptr(out), L.value, None)
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_history")
    return out


def sylv_get_hessenberg(h, side: int, s: int) -> np.ndarray:
    lib = load()
    nb = ctypes.c_int32()
    rc = lib.sylv_get_hessenberg(h, side, None, 0, ctypes.byref(nb))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_hessenberg")
    rows, cols = nb.value * s, (nb.value - 1) * s
    H = np.zeros((rows, cols), order="F")
    rc = lib.sylv_get_hessenberg(h, side, _dptr(H), rows * cols, None)
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_hessenberg")
    return H


def sylv_small_operator(h, Z: np.ndarray, s: int) -> np.ndarray:
    """[H Z, 0] + [Z G^T; 0] (eq. 3.7) with the last solve's H, G; Z is r x r."""
    r = Z.shape[0]
    Zf = np.asfortranarray(Z, dtype=np.float64)
    out = np.zeros((r + s, r + s), order="F")
    rc = load().sylv_small_operator(h, r, _dptr(Zf), _dptr(out))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_small_operator")
    return np.ascontiguousarray(out)


def sylv_set_timeout(h, timeout_s: float) -> None:
    rc = load().sylv_set_timeout(h, float(timeout_s))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_set_timeout")


def sylv_apply(h, side: int, X: np.ndarray) -> np.ndarray:
    Xf = np.asfortranarray(X, dtype=np.float64)
    Y = np.empty_like(Xf, order="F")
    rc = load().sylv_apply(h, side, _dptr(Xf), _dptr(Y), Xf.shape[1])
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_apply")
    return Y


def sylv_get_profile(h) -> list:
    """Per-kernel-class totals of the last solve (needs options.profile = 1)."""
    lib = load()
    cnt = ctypes.c_int32()
    rc = lib.sylv_get_profile(h, None, 0, ctypes.byref(cnt))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_profile")
    arr = (sylv_kernel_stat * max(1, cnt.value))()
    rc = lib.sylv_get_profile(h, arr, cnt.value, ctypes.byref(cnt))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_get_profile")
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes,
             "flops": arr[i].flops} for i in range(cnt.value)]


def sylv_spmm_noalloc(n: int, nnz: int, row_ptr: int, col_idx: int, val: int, X: int, Y: int, k: int,
                      stream: int = 0) -> int:
    """Y = A X with device pointers only (integers); allocates nothing.  Returns the status code."""
    return load().sylv_spmm_noalloc(n, nnz, row_ptr, col_idx, val, X, Y, k, stream or None)


def sylv_create_batch(As, C1s, opt: Optional[sylv_options] = None):
    """Batched Lyapunov handle for instances (A_i, C1_i); opt.lyapunov must be 1."""
    lib = load()
    count = len(As)
    arr = (sylv_csr * count)()
    keep = []
    for i, A in enumerate(As):
        c, k = _make_csr(A)
        arr[i] = c
        keep.append(k)
    cs = [np.asfortranarray(C, dtype=np.float64) for C in C1s]
    ptrs = (ctypes.POINTER(ctypes.c_double) * count)(*[_dptr(C) for C in cs])
    svec = (ctypes.c_int64 * count)(*[C.shape[1] for C in cs])
    h = ctypes.c_void_p()
    rc = lib.sylv_create_batch(count, arr, None, ptrs, None, svec, None if opt is None else ctypes.byref(opt),
                               ctypes.byref(h))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_create_batch")
    return h


def sylv_batch_instance(h, inst: int):
    out = ctypes.c_void_p()
    rc = load().sylv_batch_instance(h, inst, ctypes.byref(out))
    if rc != SYLV_OK:
        raise SylvError(rc, "sylv_batch_instance")
    return out


def sylv_destroy(h) -> None:
    if h is not None and h.value:
        load().sylv_destroy(h)


class BatchSolver:
    """Many Lyapunov equations A_i X_i + X_i A_i^T = C_i C_i^T solved together by
    batched factorized CG: ``BatchSolver([A_0, ...], [C_0, ...]).cg(tol, maxit)``."""

    def __init__(self, As, C1s, poll_every: int = 0, cuda_stream: int = 0, timeout_s: float = 0.0,
                 no_true_residual: bool = False, stop_margin: float = 0.0):
        o = sylv_default_options()
        o.lyapunov = 1
        o.stop_margin = stop_margin
        if poll_every:
            o.poll_every = poll_every
        o.cuda_stream = cuda_stream or None
        o.timeout_s = timeout_s or 3600.0
        o.no_true_residual = 1 if no_true_residual else 0
        self.ns = [_csr_arrays(A)[0] for A in As]
        self.h = sylv_create_batch(As, C1s, o)

    def cg(self, tol: float, maxit: int) -> dict:
        return sylv_cg(self.h, tol, maxit).as_dict()

    def instance(self, i: int):
        return sylv_batch_instance(self.h, i)

    def factors(self, i: int):
        n = self.ns[i]
        return sylv_get_factors(self.instance(i), n, n)

    def history(self, i: int) -> np.ndarray:
        return sylv_get_history(self.instance(i))

    def close(self) -> None:
        sylv_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass


class Solver:
    """Owns one handle: ``Solver(A, B, C1, C2, precision="fp64"|"mixed", lyapunov=False)``."""

    def __init__(self, A, B, C1, C2, precision: str = "fp64", lyapunov: bool = False, poll_every: int = 0,
                 deflate_tol: float = 0.0, cuda_stream: int = 0, timeout_s: float = 0.0, refine_max: int = 0,
                 profile: bool = False, stream_mode: int = 0, small_gemm: int = 0, basis_gemm: int = 0,
                 no_true_residual: bool = False, stop_margin: float = 0.0, cert_gemm: int = 0):
        o = sylv_default_options()
        o.cert_gemm = cert_gemm
        o.no_true_residual = 1 if no_true_residual else 0
        o.stop_margin = stop_margin
        o.precision = SYLV_MIXED if precision == "mixed" else SYLV_FP64
        o.lyapunov = 1 if lyapunov else 0
        if poll_every:
            o.poll_every = poll_every
        if refine_max:
            o.refine_max = refine_max
        o.deflate_tol = deflate_tol
        o.timeout_s = timeout_s or 3600.0
        o.cuda_stream = cuda_stream or None
        o.profile = 1 if profile else 0
        o.stream_mode = stream_mode
        o.small_gemm = small_gemm
        o.basis_gemm = basis_gemm
        self.n = _csr_arrays(A)[0]
        self.m = self.n if lyapunov else _csr_arrays(B)[0]
        self.s = C1.shape[1]
        self.h = sylv_create(A, None if lyapunov else B, C1, None if lyapunov else C2, o)

    def cg(self, tol: float, maxit: int) -> dict:
        return sylv_cg(self.h, tol, maxit).as_dict()

    def bicgstab(self, tol: float, maxit: int) -> dict:
        return sylv_bicgstab(self.h, tol, maxit).as_dict()

    def cgs(self, tol: float, maxit: int) -> dict:
        return sylv_cgs(self.h, tol, maxit).as_dict()

    def cr(self, tol: float, maxit: int) -> dict:
        return sylv_cr(self.h, tol, maxit).as_dict()

    def gpbicg(self, tol: float, maxit: int) -> dict:
        return sylv_gpbicg(self.h, tol, maxit).as_dict()

    def compress(self, tol: float) -> int:
        """Replaces the factors of the last solve by rank-q ones (see sylv_compress); returns q."""
        return sylv_compress(self.h, tol)

    def factors(self, out=None):
        return sylv_get_factors(self.h, self.n, self.m, out=out)

    def history(self) -> np.ndarray:
        return sylv_get_history(self.h)

    def hessenberg(self, side: int) -> np.ndarray:
        return sylv_get_hessenberg(self.h, side, self.s)

    def small_operator(self, Z: np.ndarray) -> np.ndarray:
        return sylv_small_operator(self.h, Z, self.s)

    def set_timeout(self, timeout_s: float) -> None:
        sylv_set_timeout(self.h, timeout_s)

    def apply(self, side: int, X: np.ndarray) -> np.ndarray:
        return sylv_apply(self.h, side, X)

    def profile(self) -> list:
        return sylv_get_profile(self.h)

    def close(self) -> None:
        sylv_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass
