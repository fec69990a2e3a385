"""Thin Python binding of the C ABI in ``include/glu.h`` (ctypes).

The functions carry the C names and only marshal arguments: numpy arrays are
passed as host pointers, torch tensors as host or device pointers; every step
of the factorization and the solves runs in the CUDA library.  PyTorch serves
only for device memory and streams.  There is no CPU fallback: if the
library is not built (``paper_1908_00204_gb300.build.build()``) every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

GLU_OK = 0
GLU_ERR_INVALID = -1
GLU_ERR_STRUCT_SINGULAR = -2
GLU_ERR_ZERO_PIVOT = -3
GLU_ERR_NONFINITE = -4
GLU_ERR_OOM = -5
GLU_ERR_CUDA = -6
GLU_ERR_TIMEOUT = -7
GLU_ERR_NOT_FACTORED = -8
GLU_ERR_INTERNAL = -9
GLU_ERR_TOO_LARGE = -10
GLU_NOALLOC_SCRATCH_DOUBLES = 4194304


class glu_options(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("mode_force", C.c_int32), ("tail_threshold", C.c_int32),
                ("piece_updates", C.c_int32), ("wide_threshold", C.c_int32), ("use_graph", C.c_int32),
                ("verbose", C.c_int32), ("host_only", C.c_int32), ("solve_mode", C.c_int32),
                ("spin_limit_us", C.c_int32), ("fault_row", C.c_int32), ("solve_tail", C.c_int32),
                ("factor_tail", C.c_int32), ("solve_blocks", C.c_int32),
                ("factor_blocks", C.c_int32), ("row_lookup", C.c_int32),
                ("src_min", C.c_int32), ("lane_max", C.c_int32), ("lane_segs", C.c_int32),
                ("gpu_analysis", C.c_int32)]


class glu_stats(C.Structure):
    _fields_ = [("n", C.c_int32), ("nlevels", C.c_int32), ("nnz_a", C.c_int64), ("nnz_lu", C.c_int64),
                ("nnz_l", C.c_int64), ("nnz_u", C.c_int64), ("n_deps", C.c_int64), ("n_pairs", C.c_int64),
                ("n_updates", C.c_int64), ("flops", C.c_double), ("levels_by_mode", C.c_int32 * 3),
                ("solve_levels_fwd", C.c_int32), ("solve_levels_bwd", C.c_int32),
                ("max_level_width", C.c_int32), ("device_bytes", C.c_int64), ("analyze_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("tail_rows", C.c_int32),
                ("factor_tail_cols", C.c_int32), ("row_lookup", C.c_int32), ("spare", C.c_int32),
                ("lookup_bytes", C.c_int64), ("n_runs", C.c_int64)]


class glu_refine_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("berr", C.c_double),
                ("berr_first", C.c_double)]


_lock = threading.Lock()
_lib = None


def load_library(path: Optional[str] = None):
    """Load libglu.so (built in-tree); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or os.environ.get("GLU_LIBRARY") or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"GLU CUDA library not built ({path}); run paper_1908_00204_gb300.build.build()")
        lib = C.CDLL(path)
        P, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "glu_default_options": (None, [C.POINTER(glu_options)]),
            "glu_analyze": (C.c_int, [i32, P, P, P, C.POINTER(P)]),
            "glu_analyze_opts": (C.c_int, [i32, P, P, P, C.POINTER(glu_options), C.POINTER(P)]),
            "glu_set_stream": (C.c_int, [P, P]),
            "glu_factor": (C.c_int, [P, P]),
            "glu_sync": (C.c_int, [P]),
            "glu_solve": (C.c_int, [P, P, P, i32]),
            "glu_solve_noalloc": (C.c_int, [P, P, P, i32]),
            "glu_factor_f32": (C.c_int, [P, P]),
            "glu_factor_batched": (C.c_int, [P, P, i32, i64]),
            "glu_get_factors_batched": (C.c_int, [P, i32, P]),
            "glu_get_factors_batched_f32": (C.c_int, [P, i32, P]),
            "glu_get_factors_f32": (C.c_int, [P, P]),
            "glu_factor_batched_f32": (C.c_int, [P, P, i32, i64]),
            "glu_solve_batched": (C.c_int, [P, P, P, i32, i32]),
            "glu_solve_batched_refine": (C.c_int, [P, P, P, i32, i32, C.c_double, i32,
                                                   C.POINTER(glu_refine_info)]),
            "glu_solve_refine": (C.c_int, [P, P, P, i32, C.c_double, i32, C.POINTER(glu_refine_info)]),
            "glu_get_fill": (C.c_int, [P, C.POINTER(P), C.POINTER(P), C.POINTER(i64)]),
            "glu_get_deps": (C.c_int, [P, C.POINTER(P), C.POINTER(P)]),
            "glu_get_levels": (C.c_int, [P, C.POINTER(i32), C.POINTER(P), C.POINTER(P)]),
            "glu_get_factors": (C.c_int, [P, P]),
            "glu_get_stats": (C.c_int, [P, C.POINTER(glu_stats)]),
            "glu_last_error_info": (C.c_int, [P, C.POINTER(i32)]),
            "glu_destroy": (None, [P]),
            "glu_order_nd": (C.c_int, [i32, P, P, P]),
            "glu_static_pivot": (C.c_int, [i32, P, P, P, P, P, P]),
            "glu_apply_static_pivot": (C.c_int, [i32, P, P, P, P, P, P, P, P]),
            "glu_strerror": (C.c_char_p, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GluError(RuntimeError):
    def __init__(self, code: int, where: str, column: int = -1):
        lib = load_library()
        msg = lib.glu_strerror(code).decode()
        super().__init__(f"{where}: {msg} (code {code}" + (f", column {column})" if column >= 0 else ")"))
        self.code = code
        self.column = column


def _check(code: int, where: str, h=None):
    if code != GLU_OK:
        col = -1
        if h is not None and code in (GLU_ERR_ZERO_PIVOT, GLU_ERR_NONFINITE):
            c = C.c_int32(-1)
            load_library().glu_last_error_info(h._ptr, C.byref(c))
            col = c.value
        raise GluError(code, where, col)


def _ptr(a, dtype):
    """Raw pointer of a numpy array or torch tensor, after checking dtype/contiguity."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[np.dtype(dtype).type]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def default_options(**kw) -> glu_options:
    o = glu_options()
    load_library().glu_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Handle:
    """Owns a glu_handle*; freed by glu_destroy or garbage collection."""

    def __init__(self, ptr, n, nnz_a):
        self._ptr = ptr
        self.n = n
        self.nnz_a = nnz_a

    def __del__(self):
        try:
            glu_destroy(self)
        except Exception:
            pass

    # convenience wrappers
    def factor(self, values):
        return glu_factor(self, values)

    def solve(self, b, x=None):
        return glu_solve(self, b, x)

    def stats(self):
        return glu_get_stats(self)


def glu_analyze(n, colptr, rowidx, perm=None, options: Optional[glu_options] = None) -> Handle:
    lib = load_library()
    colptr = np.ascontiguousarray(colptr, np.int32)
    rowidx = np.ascontiguousarray(rowidx, np.int32)
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, np.int32)
        pp = perm.ctypes.data
    out = C.c_void_p()
    if options is None:
        rc = lib.glu_analyze(int(n), colptr.ctypes.data, rowidx.ctypes.data, pp, C.byref(out))
    else:
        rc = lib.glu_analyze_opts(int(n), colptr.ctypes.data, rowidx.ctypes.data, pp, C.byref(options),
                                  C.byref(out))
    _check(rc, "glu_analyze")
    return Handle(out, int(n), int(colptr[n]) if n > 0 else 0)


def glu_set_stream(h: Handle, stream) -> None:
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(load_library().glu_set_stream(h._ptr, stream), "glu_set_stream")


def glu_factor(h: Handle, values) -> None:
    if values is not None and len(values) != h.nnz_a:
        raise ValueError(f"values must have nnz(A) = {h.nnz_a} entries")
    _check(load_library().glu_factor(h._ptr, _ptr(values, np.float64)), "glu_factor", h)


def glu_factor_f32(h: Handle, values) -> None:
    if values is not None and len(values) != h.nnz_a:
        raise ValueError(f"values must have nnz(A) = {h.nnz_a} entries")
    _check(load_library().glu_factor_f32(h._ptr, _ptr(values, np.float64)), "glu_factor_f32", h)


def glu_solve_refine(h: Handle, b, x=None, tol: float = 1e-12, maxit: int = 10, nrhs: Optional[int] = None):
    """FP32-factor solve with FP64 refinement; returns (x, info dict)."""
    k = _nrhs(b, h.n) if nrhs is None else nrhs
    if x is None:
        x = np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
    info = glu_refine_info()
    _check(load_library().glu_solve_refine(h._ptr, _ptr(b, np.float64), _ptr(x, np.float64), int(k),
                                           float(tol), int(maxit), C.byref(info)), "glu_solve_refine", h)
    return x, {name: getattr(info, name) for name, _ in glu_refine_info._fields_}


def _batch_values(h, values):
    """(batch, nnz_a) values -> (pointer, batch, ld)."""
    shape = tuple(values.shape)
    if len(shape) != 2 or shape[1] < h.nnz_a:
        raise ValueError("batched values must be (batch, >= nnz(A))")
    return _ptr(values, np.float64), shape[0], shape[1]


def glu_factor_batched(h: Handle, values) -> None:
    """FP64 refactorization of every row of ``values`` (batch, nnz(A))."""
    p, B, ld = _batch_values(h, values)
    _check(load_library().glu_factor_batched(h._ptr, p, B, ld), "glu_factor_batched", h)


def glu_factor_batched_f32(h: Handle, values) -> None:
    p, B, ld = _batch_values(h, values)
    _check(load_library().glu_factor_batched_f32(h._ptr, p, B, ld), "glu_factor_batched_f32", h)


def _batch_rhs(h, b):
    shape = tuple(b.shape)
    if len(shape) != 3 or shape[2] != h.n:
        raise ValueError("batched right-hand sides must be (batch, nrhs, n)")
    return shape[0], shape[1]


def glu_solve_batched(h: Handle, b, x=None):
    B, k = _batch_rhs(h, b)
    if x is None:
        x = np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
    _check(load_library().glu_solve_batched(h._ptr, _ptr(b, np.float64), _ptr(x, np.float64), k, B),
           "glu_solve_batched", h)
    return x


def glu_solve_batched_refine(h: Handle, b, x=None, tol: float = 1e-12, maxit: int = 10):
    B, k = _batch_rhs(h, b)
    if x is None:
        x = np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
    info = glu_refine_info()
    _check(load_library().glu_solve_batched_refine(h._ptr, _ptr(b, np.float64), _ptr(x, np.float64), k, B,
                                                   float(tol), int(maxit), C.byref(info)),
           "glu_solve_batched_refine", h)
    return x, {name: getattr(info, name) for name, _ in glu_refine_info._fields_}


def glu_sync(h: Handle) -> None:
    _check(load_library().glu_sync(h._ptr), "glu_sync", h)


def glu_sync_status(h: Handle):
    """glu_sync without raising: (code, column), column -1 unless the code is
    GLU_ERR_ZERO_PIVOT or GLU_ERR_NONFINITE."""
    code = load_library().glu_sync(h._ptr)
    col = glu_last_error_info(h) if code in (GLU_ERR_ZERO_PIVOT, GLU_ERR_NONFINITE) else -1
    return code, col


def _nrhs(b, n):
    shape = tuple(b.shape)
    if len(shape) == 1:
        if shape[0] != n:
            raise ValueError("right-hand side length != n")
        return 1
    if len(shape) == 2 and shape[1] == n:
        return shape[0]
    raise ValueError("right-hand sides must be (n,) or (nrhs, n)")


def glu_solve(h: Handle, b, x=None, nrhs: Optional[int] = None):
    """x with A x = b; b is (n,) or (nrhs, n), numpy (host) or torch (host/device)."""
    k = _nrhs(b, h.n) if nrhs is None else nrhs
    if x is None:
        if isinstance(b, np.ndarray):
            x = np.empty_like(b)
        else:
            x = b.new_empty(b.shape)
    _check(load_library().glu_solve(h._ptr, _ptr(b, np.float64), _ptr(x, np.float64), int(k)), "glu_solve", h)
    return x


def glu_solve_noalloc(h: Handle, b, x, nrhs: Optional[int] = None):
    """glu_solve with the library's fixed scratch array: b and x must be CUDA tensors."""
    k = _nrhs(b, h.n) if nrhs is None else nrhs
    _check(load_library().glu_solve_noalloc(h._ptr, _ptr(b, np.float64), _ptr(x, np.float64), int(k)),
           "glu_solve_noalloc", h)
    return x


def glu_get_fill(h: Handle):
    cp, ri, nnz = C.c_void_p(), C.c_void_p(), C.c_int64()
    _check(load_library().glu_get_fill(h._ptr, C.byref(cp), C.byref(ri), C.byref(nnz)), "glu_get_fill")
    return (np.ctypeslib.as_array(C.cast(cp, C.POINTER(C.c_int64)), (h.n + 1,)).copy(),
            np.ctypeslib.as_array(C.cast(ri, C.POINTER(C.c_int32)), (max(nnz.value, 1),))[:nnz.value].copy())


def glu_get_deps(h: Handle):
    dp, di = C.c_void_p(), C.c_void_p()
    _check(load_library().glu_get_deps(h._ptr, C.byref(dp), C.byref(di)), "glu_get_deps")
    ptr = np.ctypeslib.as_array(C.cast(dp, C.POINTER(C.c_int64)), (h.n + 1,)).copy()
    m = int(ptr[-1])
    idx = np.ctypeslib.as_array(C.cast(di, C.POINTER(C.c_int32)), (max(m, 1),))[:m].copy() if m else \
        np.zeros(0, np.int32)
    return ptr, idx


def glu_get_levels(h: Handle):
    nl = C.c_int32()
    lp, lc = C.c_void_p(), C.c_void_p()
    _check(load_library().glu_get_levels(h._ptr, C.byref(nl), C.byref(lp), C.byref(lc)), "glu_get_levels")
    ptr = np.ctypeslib.as_array(C.cast(lp, C.POINTER(C.c_int32)), (nl.value + 1,)).copy()
    cols = np.ctypeslib.as_array(C.cast(lc, C.POINTER(C.c_int32)), (max(h.n, 1),))[:h.n].copy()
    return ptr, cols


def glu_get_factors(h: Handle) -> np.ndarray:
    st = glu_get_stats(h)
    out = np.empty(max(st["nnz_lu"], 1), np.float64)
    _check(load_library().glu_get_factors(h._ptr, out.ctypes.data), "glu_get_factors", h)
    return out[:st["nnz_lu"]]


def glu_get_factors_f32(h: Handle) -> np.ndarray:
    st = glu_get_stats(h)
    out = np.empty(max(st["nnz_lu"], 1), np.float32)
    _check(load_library().glu_get_factors_f32(h._ptr, out.ctypes.data), "glu_get_factors_f32", h)
    return out[:st["nnz_lu"]]


def glu_get_factors_batched_f32(h: Handle, set_index: int) -> np.ndarray:
    st = glu_get_stats(h)
    out = np.empty(max(st["nnz_lu"], 1), np.float32)
    _check(load_library().glu_get_factors_batched_f32(h._ptr, int(set_index), out.ctypes.data),
           "glu_get_factors_batched_f32", h)
    return out[:st["nnz_lu"]]


def glu_get_factors_batched(h: Handle, set_index: int) -> np.ndarray:
    st = glu_get_stats(h)
    out = np.empty(max(st["nnz_lu"], 1), np.float64)
    _check(load_library().glu_get_factors_batched(h._ptr, int(set_index), out.ctypes.data),
           "glu_get_factors_batched", h)
    return out[:st["nnz_lu"]]


def glu_get_stats(h: Handle) -> dict:
    s = glu_stats()
    _check(load_library().glu_get_stats(h._ptr, C.byref(s)), "glu_get_stats")
    d = {name: getattr(s, name) for name, _ in glu_stats._fields_}
    d["levels_by_mode"] = list(s.levels_by_mode)
    return d


def glu_last_error_info(h: Handle) -> int:
    c = C.c_int32(-1)
    _check(load_library().glu_last_error_info(h._ptr, C.byref(c)), "glu_last_error_info")
    return c.value


def glu_destroy(h: Handle) -> None:
    if h._ptr:
        load_library().glu_destroy(h._ptr)
        h._ptr = None


def glu_order_nd(n: int, colptr, rowidx) -> np.ndarray:
    """Nested-dissection ordering of the pattern of A + A^T: perm[new] = old."""
    cp = np.ascontiguousarray(colptr, np.int32)
    ri = np.ascontiguousarray(rowidx, np.int32)
    perm = np.empty(max(n, 1), np.int32)
    _check(load_library().glu_order_nd(int(n), cp.ctypes.data, ri.ctypes.data, perm.ctypes.data), "glu_order_nd")
    return perm[:n]


def glu_static_pivot(n: int, colptr, rowidx, values):
    """Row matching with scaling: (row_perm, row_scale, col_scale), see
    apply_static_pivot."""
    cp = np.ascontiguousarray(colptr, np.int32)
    ri = np.ascontiguousarray(rowidx, np.int32)
    va = np.ascontiguousarray(values, np.float64)
    rp = np.empty(max(n, 1), np.int32)
    rs = np.empty(max(n, 1), np.float64)
    cs = np.empty(max(n, 1), np.float64)
    _check(load_library().glu_static_pivot(int(n), cp.ctypes.data, ri.ctypes.data, va.ctypes.data, rp.ctypes.data,
                                           rs.ctypes.data, cs.ctypes.data), "glu_static_pivot")
    return rp[:n], rs[:n], cs[:n]


def glu_apply_static_pivot(n: int, colptr, rowidx, values, row_perm, row_scale=None, col_scale=None):
    """CSC of B = P_r D_r A D_c (glu_apply_static_pivot): (colptr, rowidx, values)."""
    cp = np.ascontiguousarray(colptr, np.int32)
    ri = np.ascontiguousarray(rowidx, np.int32)
    va = np.ascontiguousarray(values, np.float64)
    rp = np.ascontiguousarray(row_perm, np.int32)
    rs = None if row_scale is None else np.ascontiguousarray(row_scale, np.float64)
    cs = None if col_scale is None else np.ascontiguousarray(col_scale, np.float64)
    nnz = int(cp[n]) if n > 0 else 0
    out_ri = np.empty(max(nnz, 1), np.int32)
    out_va = np.empty(max(nnz, 1), np.float64)
    _check(load_library().glu_apply_static_pivot(int(n), cp.ctypes.data, ri.ctypes.data, va.ctypes.data,
                                                 rp.ctypes.data, None if rs is None else rs.ctypes.data,
                                                 None if cs is None else cs.ctypes.data, out_ri.ctypes.data,
                                                 out_va.ctypes.data), "glu_apply_static_pivot")
    return cp.copy(), out_ri[:nnz], out_va[:nnz]


apply_static_pivot = glu_apply_static_pivot


def glu_strerror(code: int) -> str:
    return load_library().glu_strerror(int(code)).decode()
