"""CPU oracle for the GLU3.0 refactorization path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never loads it, and it never
loads the CUDA library: the two share no code.

Each function follows one step of the method (Peng & Tan, GLU3.0):

* ``permute``   -- B = P A P^T and the input checks (Section II-C, preprocessing)
* ``symbolic``  -- fill-in of L+U by Gilbert-Peierls reachability (Section II-A)
* ``deps``      -- relaxed dependency detection, Algorithm 4 (Section III-A)
* ``levels``    -- longest-path levelization of the dependency graph (Section II-C)
* ``numeric``   -- Gilbert-Peierls left-looking LU, Algorithm 1 (Section II-A)
* ``solve``     -- forward/backward substitution (Section I)
* ``flops``     -- l_j + 2 l_j u_j summed over columns (Algorithm 2)

The C source is built with gcc (``-O2 -ffp-contract=off``) on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glu_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
# a test may point the wrapper at a deliberately broken build of the source
_SO_OVERRIDE = os.environ.get("GLU_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "invalid", -2: "structurally singular", -3: "zero pivot",
          -4: "non-finite", -5: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code, column=-1):
        super().__init__(f"oracle: {ERRORS.get(code, code)} (column {column})")
        self.code = code
        self.column = column


def build(force: bool = False) -> str:
    """Compile the oracle's C source into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_SO_OVERRIDE if _SO_OVERRIDE else build())
        P = C.c_void_p
        i32, i64 = C.c_int32, C.c_int64
        lib.oracle_permute.argtypes = [i32, P, P, P, P, P, P]
        lib.oracle_symbolic.argtypes = [i32, P, P, C.POINTER(P), C.POINTER(P), C.POINTER(i64)]
        lib.oracle_deps.argtypes = [i32, P, P, C.POINTER(P), C.POINTER(P)]
        lib.oracle_levels.argtypes = [i32, P, P, P, C.POINTER(i32), C.POINTER(P), C.POINTER(P)]
        lib.oracle_numeric.argtypes = [i32, P, P, P, P, P, P, C.POINTER(i32)]
        lib.oracle_solve.argtypes = [i32, P, P, P, P, P, P, i32]
        lib.oracle_solve_levels.argtypes = [i32, P, P, P, P]
        lib.oracle_flops.argtypes = [i32, P, P]
        lib.oracle_flops.restype = C.c_double
        lib.oracle_residual.argtypes = [i32, P, P, P, P, P, P, i32]
        lib.oracle_residual.restype = None
        lib.oracle_free.argtypes = [P]
        lib.oracle_free.restype = None
        _lib = lib
        return lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _take(ptr, count, dtype):
    """Copy a malloc'ed C array into numpy and free it."""
    lib = _load()
    if count == 0:
        lib.oracle_free(ptr)
        return np.zeros(0, dtype)
    ct = {np.int32: C.c_int32, np.int64: C.c_int64, np.float64: C.c_double}[dtype]
    arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(count,)).copy()
    lib.oracle_free(ptr)
    return arr


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def permute(n, colptr, rowidx, perm=None):
    """B = P A P^T. Returns (bcolptr, browidx, bsrc) with bsrc the A index of each B entry."""
    lib = _load()
    colptr, rowidx = _i32(colptr), _i32(rowidx)
    perm = _i32(np.arange(n) if perm is None else perm)
    nnz = int(colptr[n]) if n > 0 else 0
    bcp = np.zeros(n + 1, np.int32)
    bri = np.zeros(max(nnz, 1), np.int32)
    bsrc = np.zeros(max(nnz, 1), np.int64)
    rc = lib.oracle_permute(n, _p(colptr), _p(rowidx), _p(perm), _p(bcp), _p(bri), _p(bsrc))
    if rc != 0:
        raise OracleError(rc)
    return bcp, bri[:nnz], bsrc[:nnz]


def symbolic(n, bcolptr, browidx):
    """Filled pattern of L+U-I: (lu_colptr int64[n+1], lu_rowidx int32[nnz])."""
    lib = _load()
    bcolptr, browidx = _i32(bcolptr), _i32(browidx)
    cp, ri, nnz = C.c_void_p(), C.c_void_p(), C.c_int64()
    rc = lib.oracle_symbolic(n, _p(bcolptr), _p(browidx), C.byref(cp), C.byref(ri), C.byref(nnz))
    if rc != 0:
        raise OracleError(rc)
    return _take(cp, n + 1, np.int64), _take(ri, nnz.value, np.int32)


def deps(n, lu_colptr, lu_rowidx):
    """Algorithm 4 dependency lists: (dep_ptr int64[n+1], dep_idx int32)."""
    lib = _load()
    cp = np.ascontiguousarray(lu_colptr, np.int64)
    ri = _i32(lu_rowidx)
    dp, di = C.c_void_p(), C.c_void_p()
    rc = lib.oracle_deps(n, _p(cp), _p(ri), C.byref(dp), C.byref(di))
    if rc != 0:
        raise OracleError(rc)
    dptr = _take(dp, n + 1, np.int64)
    return dptr, _take(di, int(dptr[-1]), np.int32)


def levels(n, dep_ptr, dep_idx):
    """Levels: (level_of int32[n], level_ptr int32[L+1], level_cols int32[n])."""
    lib = _load()
    dp = np.ascontiguousarray(dep_ptr, np.int64)
    di = _i32(dep_idx)
    lvl = np.zeros(max(n, 1), np.int32)
    nl = C.c_int32()
    lp, lc = C.c_void_p(), C.c_void_p()
    rc = lib.oracle_levels(n, _p(dp), _p(di), _p(lvl), C.byref(nl), C.byref(lp), C.byref(lc))
    if rc != 0:
        raise OracleError(rc)
    return lvl[:n], _take(lp, nl.value + 1, np.int32), _take(lc, n, np.int32)


def numeric(n, bcolptr, browidx, bval, lu_colptr, lu_rowidx):
    """Algorithm 1 on B's values (B's CSC order). Returns lu_val (pattern order)."""
    lib = _load()
    bcolptr, browidx = _i32(bcolptr), _i32(browidx)
    bval = np.ascontiguousarray(bval, np.float64)
    cp = np.ascontiguousarray(lu_colptr, np.int64)
    ri = _i32(lu_rowidx)
    out = np.zeros(max(int(cp[-1]), 1), np.float64)
    bad = C.c_int32(-1)
    rc = lib.oracle_numeric(n, _p(bcolptr), _p(browidx), _p(bval), _p(cp), _p(ri), _p(out),
                            C.byref(bad))
    if rc != 0:
        raise OracleError(rc, bad.value)
    return out[: int(cp[-1])]


def solve(n, lu_colptr, lu_rowidx, lu_val, perm, b):
    """x with A x = b for every row of b (shape (nrhs, n))."""
    lib = _load()
    b = np.ascontiguousarray(np.atleast_2d(b), np.float64)
    x = np.zeros_like(b)
    cp = np.ascontiguousarray(lu_colptr, np.int64)
    ri = _i32(lu_rowidx)
    lv = np.ascontiguousarray(lu_val, np.float64)
    perm = _i32(np.arange(n) if perm is None else perm)
    rc = lib.oracle_solve(n, _p(cp), _p(ri), _p(lv), _p(perm), _p(b), _p(x), b.shape[0])
    if rc != 0:
        raise OracleError(rc)
    return x


def solve_levels(n, lu_colptr, lu_rowidx):
    lib = _load()
    cp = np.ascontiguousarray(lu_colptr, np.int64)
    ri = _i32(lu_rowidx)
    lf = np.zeros(max(n, 1), np.int32)
    lb = np.zeros(max(n, 1), np.int32)
    lib.oracle_solve_levels(n, _p(cp), _p(ri), _p(lf), _p(lb))
    return lf[:n], lb[:n]


def flops(n, lu_colptr, lu_rowidx) -> float:
    lib = _load()
    cp = np.ascontiguousarray(lu_colptr, np.int64)
    ri = _i32(lu_rowidx)
    return float(lib.oracle_flops(n, _p(cp), _p(ri)))


def residual(n, colptr, rowidx, aval, b, x):
    """r = b - A x on A's own CSC, rows of b/x are right-hand sides."""
    lib = _load()
    colptr, rowidx = _i32(colptr), _i32(rowidx)
    aval = np.ascontiguousarray(aval, np.float64)
    b = np.ascontiguousarray(np.atleast_2d(b), np.float64)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    r = np.zeros_like(b)
    lib.oracle_residual(n, _p(colptr), _p(rowidx), _p(aval), _p(b), _p(x), _p(r), b.shape[0])
    return r


class Factorization:
    """Everything the oracle computes for one matrix (test convenience)."""

    def __init__(self, n, colptr, rowidx, perm=None, values=None):
        self.n = n
        self.colptr = _i32(colptr)
        self.rowidx = _i32(rowidx)
        self.perm = _i32(np.arange(n) if perm is None else perm)
        self.bcolptr, self.browidx, self.bsrc = permute(n, self.colptr, self.rowidx, self.perm)
        self.lu_colptr, self.lu_rowidx = symbolic(n, self.bcolptr, self.browidx)
        self.dep_ptr, self.dep_idx = deps(n, self.lu_colptr, self.lu_rowidx)
        self.level_of, self.level_ptr, self.level_cols = levels(n, self.dep_ptr, self.dep_idx)
        self.lu_val = None
        if values is not None:
            self.factor(values)

    @property
    def nnz(self):
        return int(self.lu_colptr[-1])

    @property
    def nlevels(self):
        return int(self.level_ptr.size - 1)

    def factor(self, values):
        values = np.ascontiguousarray(values, np.float64)
        self.lu_val = numeric(self.n, self.bcolptr, self.browidx, values[self.bsrc],
                              self.lu_colptr, self.lu_rowidx)
        return self.lu_val

    def solve(self, b):
        return solve(self.n, self.lu_colptr, self.lu_rowidx, self.lu_val, self.perm, b)

    def flops(self):
        return flops(self.n, self.lu_colptr, self.lu_rowidx)
