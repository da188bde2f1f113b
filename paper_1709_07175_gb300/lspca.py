"""Thin ctypes binding of liblspca (include/lspca.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Functions carry the C names; tensors are torch CUDA tensors (device memory),
their data pointers and sizes are passed through unchanged.  The library is
loaded on first use; a missing library raises ``LspcaLibraryError`` (there is
no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblspca.so")

LSPCA_F64, LSPCA_F32, LSPCA_BF16, LSPCA_E4M3 = 0, 1, 2, 3
OMEGA_GAUSSIAN, OMEGA_VERY_SPARSE = 0, 1
WANT_GRAM, FORCE_SIMT = 2, 16
OK, ERR_INVALID, ERR_NOMEM, WARN_RANK_DEFICIENT, ERR_NUMERIC, ERR_TIMEOUT, ERR_CUDA, ERR_BUSY = range(8)

DTYPE_CODES = {torch.float64: LSPCA_F64, torch.float32: LSPCA_F32, torch.bfloat16: LSPCA_BF16,
               torch.float8_e4m3fn: LSPCA_E4M3}
RESULT_DTYPE = {LSPCA_F64: torch.float64, LSPCA_F32: torch.float32, LSPCA_BF16: torch.float32,
                LSPCA_E4M3: torch.float32}


class LspcaLibraryError(RuntimeError):
    pass


class LspcaError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {lspca_strerror(code)} ({code})")
        self.code = code


class lspca_omega(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("p", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class lspca_report(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_sketch", ctypes.c_double), ("ms_chain", ctypes.c_double),
                ("ms_small", ctypes.c_double), ("ms_qr", ctypes.c_double), ("bytes_x", ctypes.c_double),
                ("rank", ctypes.c_int32), ("device_status", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("qr_path", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_I32, _I64, _U32, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t

_SIGS = {
    "lspca_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _SZ]),
    "lspca_destroy": (ctypes.c_int, [_P]),
    "lspca_fit": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _U32, _P, _P, _P, _P, _P,
                                 ctypes.POINTER(lspca_report)]),
    "spca_fit": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _U32, _P, _P, _P, _P, _P,
                                ctypes.POINTER(lspca_report)]),
    "lspca_fit_host": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _U32, _I64, _P, _P, _P,
                                      _P, ctypes.POINTER(lspca_report)]),
    "lspca_fit_project_host": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _U32, _I64, _P,
                                              _P, _P, _P, _P, _P, ctypes.POINTER(lspca_report)]),
    "lspca_fit_oversampled": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, _I32, lspca_omega, _U32, _P,
                                             _P, _P, _P, ctypes.POINTER(lspca_report)]),
    "lspca_fit_csr": (ctypes.c_int, [_P, _P, _P, _P, _I64, _I64, _I64, _I32, lspca_omega, _U32, _P, _P, _P, _P,
                                     ctypes.POINTER(lspca_report)]),
    "lspca_project_csr": (ctypes.c_int, [_P, _P, _P, _P, _I64, _I64, _I64, _P, _I32, _P, _P]),
    "lspca_project": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _P, _I32, _P, _P]),
    "lspca_omega_materialize": (ctypes.c_int, [_P, lspca_omega, _I64, _I32, _I32, _P, _P]),
    "lspca_sketch": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _U32, _P, _P]),
    "lspca_chain": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _P, _I32, _U32, _P, _P, _P]),
    "lspca_decompose": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I32, _P, _P, _P, _P]),
    "lspca_sync_status": (ctypes.c_int, [_P, _P]),
    "lspca_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lspca_launch_count": (ctypes.c_int64, [_P]),
    "lspca_chain_noalloc": (ctypes.c_int, [_P, _I32, _I64, _I64, _I64, _P, _I32, _P, _P, _P]),
    "lspca_sum_partials": (ctypes.c_int, [_P, _P, _I32, _I64, _P, _P]),
    "lspca_wait_probe": (ctypes.c_int, [_P, _I64, _P, _P]),
    "lspca_srv_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _SZ, _I32]),
    "lspca_srv_destroy": (ctypes.c_int, [_P]),
    "lspca_srv_register_v": (ctypes.c_int, [_P, _P, _I64, _I32, ctypes.POINTER(_I32)]),
    "lspca_srv_submit_project": (ctypes.c_int, [_P, _I32, _P, _I32, _I64, _I64, _P, ctypes.POINTER(_I64)]),
    "lspca_srv_submit_fit": (ctypes.c_int, [_P, _P, _I32, _I64, _I64, _I64, _I32, lspca_omega, _P, _P,
                                            ctypes.POINTER(_I64)]),
    "lspca_srv_step": (ctypes.c_int, [_P, ctypes.POINTER(_I32)]),
    "lspca_srv_poll": (ctypes.c_int, [_P, _I64, ctypes.POINTER(_I32)]),
    "lspca_srv_wait": (ctypes.c_int, [_P, _I64, _I32]),
    "lspca_srv_release": (ctypes.c_int, [_P, _I64]),
    "lspca_srv_launch_count": (ctypes.c_int64, [_P]),
    "lspca_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "lspca_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblspca.so and declare the signatures of include/lspca.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LspcaLibraryError(f"liblspca.so not built ({path}); run paper_1709_07175_gb300.build.build()")
    try:
        lib = ctypes.CDLL(path)
    except OSError as e:
        raise LspcaLibraryError(f"cannot load {path}: {e}") from e
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensors passed to liblspca must be row-major contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def omega(kind: str | int, seed: int = 0, p: int = 0) -> lspca_omega:
    k = {"gaussian": OMEGA_GAUSSIAN, "sparse": OMEGA_VERY_SPARSE}.get(kind, kind)
    return lspca_omega(int(k), int(p), int(seed))


def _xargs(X: torch.Tensor):
    """X may be a row-strided view (unit column stride, ldx = stride(0) >= n)."""
    if X.dim() != 2 or X.stride(1) != 1 or X.stride(0) < X.shape[1]:
        raise ValueError("X must be a row-major 2-D tensor (unit column stride)")
    return X.data_ptr(), DTYPE_CODES[X.dtype], X.shape[0], X.shape[1], X.stride(0)


# ---- the C entry points, same names -----------------------------------------

def lspca_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _P()
    rc = load().lspca_create(ctypes.byref(h), device, hbm_budget_bytes)
    if rc:
        raise LspcaError(rc, "lspca_create")
    return h.value


def lspca_destroy(ctx: int) -> int:
    return load().lspca_destroy(ctx)


def lspca_fit_host(ctx, Xh, k, om, flags, slice_rows, V, sigma, rank=None, stream=None, report=None) -> int:
    """Xh: a CPU tensor (pinned for overlapped copies); V, sigma, rank: CUDA tensors."""
    x, xt, m, n, ldx = _xargs(Xh)
    rep = ctypes.byref(report) if report is not None else None
    return load().lspca_fit_host(ctx, x, xt, m, n, ldx, k, om, flags, int(slice_rows), _ptr(V), _ptr(sigma),
                                 _ptr(rank), _stream(stream), rep)


def lspca_fit(ctx, X, k, om, flags, V, sigma, gram=None, rank=None, stream=None, report=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    rp = ctypes.byref(report) if report is not None else None
    return load().lspca_fit(ctx, x, xt, m, n, ldx, k, om, flags, _ptr(V), _ptr(sigma), _ptr(gram), _ptr(rank),
                            _stream(stream), rp)


def lspca_fit_oversampled(ctx, X, k, l, om, flags, V, sigma, rank=None, stream=None, report=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    rp = ctypes.byref(report) if report is not None else None
    return load().lspca_fit_oversampled(ctx, x, xt, m, n, ldx, k, l, om, flags, _ptr(V), _ptr(sigma), _ptr(rank),
                                        _stream(stream), rp)


def _csr_args(row_ptr, col, val):
    """Device CSR arrays (int64 row offsets, int32 columns, FP32 values) -> pointers, m, nnz."""
    if row_ptr.dtype != torch.int64 or col.dtype != torch.int32 or val.dtype != torch.float32:
        raise TypeError("CSR arrays must be int64 row offsets, int32 column indices and float32 values")
    nnz = val.numel()
    return _ptr(row_ptr), (_ptr(col) if nnz else None), (_ptr(val) if nnz else None), row_ptr.numel() - 1, nnz


def lspca_fit_csr(ctx, row_ptr, col, val, n, k, om, flags, V, sigma, rank=None, stream=None, report=None) -> int:
    rp_, cp, vp, m, nnz = _csr_args(row_ptr, col, val)
    rp = ctypes.byref(report) if report is not None else None
    return load().lspca_fit_csr(ctx, rp_, cp, vp, m, n, nnz, k, om, flags, _ptr(V), _ptr(sigma), _ptr(rank),
                                _stream(stream), rp)


def lspca_project_csr(ctx, row_ptr, col, val, n, V, k, Y, stream=None) -> int:
    rp_, cp, vp, m, nnz = _csr_args(row_ptr, col, val)
    return load().lspca_project_csr(ctx, rp_, cp, vp, m, n, nnz, _ptr(V), k, _ptr(Y), _stream(stream))


def spca_fit(ctx, X, k, om, flags, V, sigma, gram=None, rank=None, stream=None, report=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    rp = ctypes.byref(report) if report is not None else None
    return load().spca_fit(ctx, x, xt, m, n, ldx, k, om, flags, _ptr(V), _ptr(sigma), _ptr(gram), _ptr(rank),
                           _stream(stream), rp)


def lspca_fit_project_host(ctx, Xh, k, om, flags, slice_rows, Xd, V, sigma, Yh, rank=None, stream=None,
                           report=None) -> int:
    """Xh, Yh: CPU tensors (pinned for overlapped copies); Xd, V, sigma, rank: CUDA tensors."""
    x, xt, m, n, ldx = _xargs(Xh)
    rep = ctypes.byref(report) if report is not None else None
    return load().lspca_fit_project_host(ctx, x, xt, m, n, ldx, k, om, flags, int(slice_rows), _ptr(Xd), _ptr(V),
                                         _ptr(sigma), _ptr(rank), _ptr(Yh), _stream(stream), rep)


def lspca_project(ctx, X, V, k, Y, stream=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    return load().lspca_project(ctx, x, xt, m, n, ldx, _ptr(V), k, _ptr(Y), _stream(stream))


def lspca_omega_materialize(ctx, om, n, k, t, out, stream=None) -> int:
    return load().lspca_omega_materialize(ctx, om, n, k, t, _ptr(out), _stream(stream))


def lspca_sketch(ctx, X, k, om, flags, U, stream=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    return load().lspca_sketch(ctx, x, xt, m, n, ldx, k, om, flags, _ptr(U), _stream(stream))


def lspca_chain(ctx, X, U, k, flags, F, G=None, stream=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    return load().lspca_chain(ctx, x, xt, m, n, ldx, _ptr(U), k, flags, _ptr(F), _ptr(G), _stream(stream))


def lspca_chain_noalloc(X, U, k, F, status=None, stream=None) -> int:
    x, xt, m, n, ldx = _xargs(X)
    return load().lspca_chain_noalloc(x, xt, m, n, ldx, _ptr(U), k, _ptr(F), _ptr(status), _stream(stream))


def lspca_sum_partials(ctx, parts, out, stream=None) -> int:
    """parts: (nparts, ...) FP64 CUDA tensor; out: FP64 CUDA tensor of one part's shape."""
    return load().lspca_sum_partials(ctx, _ptr(parts), parts.shape[0], out.numel(), _ptr(out), _stream(stream))


def lspca_wait_probe(ctx, limit_ns, waited_ns=None, stream=None) -> int:
    """waited_ns: optional int64 CUDA tensor of one element."""
    return load().lspca_wait_probe(ctx, int(limit_ns), _ptr(waited_ns), _stream(stream))


def lspca_decompose(ctx, F, k, n, m, vt, V, sigma, rank=None, stream=None) -> int:
    return load().lspca_decompose(ctx, _ptr(F), k, n, m, vt, _ptr(V), _ptr(sigma), _ptr(rank), _stream(stream))


def lspca_sync_status(ctx, stream=None) -> int:
    return load().lspca_sync_status(ctx, _stream(stream))


def lspca_strerror(code: int) -> str:
    return load().lspca_strerror(code).decode()


def lspca_launch_count(ctx) -> int:
    return load().lspca_launch_count(ctx)


def lspca_profile(ctx, enable: bool) -> int:
    return load().lspca_profile(ctx, 1 if enable else 0)


def lspca_profile_read(ctx):
    ms = (ctypes.c_double * 7)()
    calls = _I64()
    rc = load().lspca_profile_read(ctx, ms, ctypes.byref(calls))
    if rc:
        raise LspcaError(rc, "lspca_profile_read")
    return list(ms), calls.value


# ---- serving ------------------------------------------------------------------

def lspca_srv_create(device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 64) -> int:
    h = _P()
    rc = load().lspca_srv_create(ctypes.byref(h), device, hbm_budget_bytes, max_inflight)
    if rc:
        raise LspcaError(rc, "lspca_srv_create")
    return h.value


def lspca_srv_destroy(srv) -> int:
    return load().lspca_srv_destroy(srv)


def lspca_srv_register_v(srv, V) -> int:
    vid = _I32()
    rc = load().lspca_srv_register_v(srv, _ptr(V), V.shape[0], V.shape[1], ctypes.byref(vid))
    if rc:
        raise LspcaError(rc, "lspca_srv_register_v")
    return vid.value


def lspca_srv_submit_project(srv, v_id, X, Y) -> tuple:
    x, xt, m, n, ldx = _xargs(X)
    req = _I64()
    rc = load().lspca_srv_submit_project(srv, v_id, x, xt, m, ldx, _ptr(Y), ctypes.byref(req))
    return rc, req.value


def lspca_srv_submit_fit(srv, X, k, om, V, sigma) -> tuple:
    x, xt, m, n, ldx = _xargs(X)
    req = _I64()
    rc = load().lspca_srv_submit_fit(srv, x, xt, m, n, ldx, k, om, _ptr(V), _ptr(sigma), ctypes.byref(req))
    return rc, req.value


def lspca_srv_step(srv) -> tuple:
    u = _I32()
    rc = load().lspca_srv_step(srv, ctypes.byref(u))
    return rc, u.value


def lspca_srv_poll(srv, req) -> tuple:
    d = _I32()
    rc = load().lspca_srv_poll(srv, req, ctypes.byref(d))
    return rc, bool(d.value)


def lspca_srv_wait(srv, req, timeout_ms: int = 60000) -> int:
    return load().lspca_srv_wait(srv, req, timeout_ms)


def lspca_srv_release(srv, req) -> int:
    return load().lspca_srv_release(srv, req)


def lspca_srv_launch_count(srv) -> int:
    return load().lspca_srv_launch_count(srv)


class Server:
    """Continuous-batching server (lspca_srv_*): projections and fits."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 64):
        self.handle = lspca_srv_create(device, hbm_budget_bytes, max_inflight)
        self.device = device
        self._keep = {}

    def close(self):
        if self.handle:
            lspca_srv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register_v(self, V) -> int:
        vid = lspca_srv_register_v(self.handle, V)
        self._keep[("v", vid)] = V
        return vid

    def submit_project(self, v_id, X):
        k = self._keep[("v", v_id)].shape[1]
        Y = torch.empty(X.shape[0], k, dtype=torch.float32, device=X.device)
        rc, req = lspca_srv_submit_project(self.handle, v_id, X, Y)
        _check(rc, "lspca_srv_submit_project")
        self._keep[req] = (X, Y)
        return req, Y

    def submit_fit(self, X, k, om):
        V = torch.empty(X.shape[1], k, dtype=torch.float32, device=X.device)
        sigma = torch.empty(k, dtype=torch.float64, device=X.device)
        rc, req = lspca_srv_submit_fit(self.handle, X, k, om, V, sigma)
        _check(rc, "lspca_srv_submit_fit")
        self._keep[req] = (X, V, sigma)
        return req, V, sigma

    def step(self) -> int:
        rc, u = lspca_srv_step(self.handle)
        _check(rc, "lspca_srv_step")
        return u

    def done(self, req) -> bool:
        rc, d = lspca_srv_poll(self.handle, req)
        _check(rc, "lspca_srv_poll")
        return d

    def wait(self, req, timeout_ms: int = 60000):
        _check(lspca_srv_wait(self.handle, req, timeout_ms), "lspca_srv_wait")

    def release(self, req):
        rc = lspca_srv_release(self.handle, req)
        if rc == OK:
            self._keep.pop(req, None)
        return rc


# ---- a small convenience wrapper (allocates outputs with torch) --------------

def _check(rc: int, what: str, allow=(OK,)):
    if rc not in allow:
        raise LspcaError(rc, what)
    return rc


@dataclass
class FitResult:
    V: torch.Tensor
    sigma: torch.Tensor
    rank: torch.Tensor
    gram: torch.Tensor | None
    status: int
    report: dict | None


class Context:
    """Owns one lspca_ctx on a device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = lspca_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            lspca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _fit(self, fn, X, k, om, flags=0, report=True, stream=None) -> FitResult:
        dev = X.device
        rt = RESULT_DTYPE[DTYPE_CODES[X.dtype]]
        V = torch.empty(X.shape[1], k, dtype=rt, device=dev)
        sigma = torch.empty(k, dtype=torch.float64, device=dev)
        rank = torch.empty(1, dtype=torch.int32, device=dev)
        gram = torch.empty(k, k, dtype=torch.float64, device=dev) if flags & WANT_GRAM else None
        rep = lspca_report() if report else None
        rc = fn(self.handle, X, k, om, flags, V, sigma, gram, rank, stream, rep)
        _check(rc, fn.__name__, allow=(OK, WARN_RANK_DEFICIENT))
        return FitResult(V, sigma, rank, gram, rc, rep.as_dict() if rep is not None else None)

    def fit(self, X, k, om, flags=0, report=True, stream=None) -> FitResult:
        return self._fit(lspca_fit, X, k, om, flags, report, stream)

    def fit_oversampled(self, X, k, l, om, flags=0, report=True, stream=None) -> FitResult:
        """Fit with an l-column Omega (l >= k), truncated to the top k."""
        dev = X.device
        rt = RESULT_DTYPE[DTYPE_CODES[X.dtype]]
        V = torch.empty(X.shape[1], k, dtype=rt, device=dev)
        sigma = torch.empty(k, dtype=torch.float64, device=dev)
        rank = torch.empty(1, dtype=torch.int32, device=dev)
        rep = lspca_report() if report else None
        rc = lspca_fit_oversampled(self.handle, X, k, l, om, flags, V, sigma, rank, stream, rep)
        _check(rc, "lspca_fit_oversampled", allow=(OK, WARN_RANK_DEFICIENT))
        return FitResult(V, sigma, rank, None, rc, rep.as_dict() if rep is not None else None)

    def fit_csr(self, row_ptr, col, val, n, k, om, report=True, stream=None) -> FitResult:
        """Fit a sparse X given by device CSR arrays (rows = samples)."""
        dev = val.device
        V = torch.empty(n, k, dtype=torch.float32, device=dev)
        sigma = torch.empty(k, dtype=torch.float64, device=dev)
        rank = torch.empty(1, dtype=torch.int32, device=dev)
        rep = lspca_report() if report else None
        rc = lspca_fit_csr(self.handle, row_ptr, col, val, n, k, om, 0, V, sigma, rank, stream, rep)
        _check(rc, "lspca_fit_csr", allow=(OK, WARN_RANK_DEFICIENT))
        return FitResult(V, sigma, rank, None, rc, rep.as_dict() if rep is not None else None)

    def project_csr(self, row_ptr, col, val, n, V, stream=None):
        k = V.shape[1]
        Y = torch.empty(row_ptr.numel() - 1, k, dtype=torch.float32, device=V.device)
        _check(lspca_project_csr(self.handle, row_ptr, col, val, n, V, k, Y, stream), "lspca_project_csr")
        return Y

    def fit_host(self, Xh, k, om, slice_rows=0, report=True, stream=None) -> FitResult:
        """Fit a host-resident X (CPU tensor, pinned for overlapped copies) slice by slice."""
        dev = torch.device(f"cuda:{self.device}")
        V = torch.empty(Xh.shape[1], k, dtype=torch.float32, device=dev)
        sigma = torch.empty(k, dtype=torch.float64, device=dev)
        rank = torch.empty(1, dtype=torch.int32, device=dev)
        rep = lspca_report() if report else None
        rc = lspca_fit_host(self.handle, Xh, k, om, 0, slice_rows, V, sigma, rank, stream, rep)
        _check(rc, "lspca_fit_host", allow=(OK, WARN_RANK_DEFICIENT))
        return FitResult(V, sigma, rank, None, rc, rep.as_dict() if rep is not None else None)

    def spca(self, X, k, om, flags=0, report=True, stream=None) -> FitResult:
        return self._fit(spca_fit, X, k, om, flags, report, stream)

    def project(self, X, V, stream=None) -> torch.Tensor:
        k = V.shape[1]
        Y = torch.empty(X.shape[0], k, dtype=V.dtype, device=X.device)
        _check(lspca_project(self.handle, X, V, k, Y, stream), "lspca_project")
        return Y

    def omega(self, om, n, k, dtype=torch.float64) -> torch.Tensor:
        out = torch.empty(n, k, dtype=dtype, device=f"cuda:{self.device}")
        _check(lspca_omega_materialize(self.handle, om, n, k, DTYPE_CODES[dtype], out), "lspca_omega_materialize")
        return out

    def sketch(self, X, k, om, flags=0) -> torch.Tensor:
        rt = RESULT_DTYPE[DTYPE_CODES[X.dtype]]
        U = torch.empty(X.shape[0], k, dtype=rt, device=X.device)
        _check(lspca_sketch(self.handle, X, k, om, flags, U), "lspca_sketch")
        return U

    def chain(self, X, U, flags=0, want_gram=False):
        k = U.shape[1]
        F = torch.empty(k, X.shape[1], dtype=torch.float64, device=X.device)
        G = torch.empty(k, k, dtype=torch.float64, device=X.device) if want_gram else None
        _check(lspca_chain(self.handle, X, U, k, flags, F, G), "lspca_chain")
        return F, G

    def decompose(self, F, m, vt=torch.float64):
        k, n = F.shape
        V = torch.empty(n, k, dtype=vt, device=F.device)
        sigma = torch.empty(k, dtype=torch.float64, device=F.device)
        rank = torch.empty(1, dtype=torch.int32, device=F.device)
        _check(lspca_decompose(self.handle, F, k, n, m, DTYPE_CODES[vt], V, sigma, rank), "lspca_decompose")
        return V, sigma, rank

    def sync_status(self, stream=None) -> int:
        return lspca_sync_status(self.handle, stream)

    def launch_count(self) -> int:
        return lspca_launch_count(self.handle)
