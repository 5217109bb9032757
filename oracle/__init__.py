"""CPU FP64 oracle for GS(p), GMRES(m) with CGS2 and Bi-CGSTAB.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  It shares no code
with the CUDA library and is never on the product path.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, FP64); this
module marshals numpy arrays to it.  ``dense_solve`` and ``eigvals`` are
LAPACK routines via numpy, used only as independent checks.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from .build import build as _build

CONVERGED, MAXIT, BREAKDOWN, STAGNATED = 0, 1, 2, 3
CONV_NAMES = {0: "converged", 1: "maxit", 2: "breakdown", 3: "stagnated"}
_ERRORS = {1: "invalid argument", 2: "zero row", 3: "non-finite value", 4: "out of memory"}


class OracleError(RuntimeError):
    pass


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("refreshes", C.c_int),
                ("conv", C.c_int), ("relres_true", C.c_double), ("relres_rec", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build())
        vp = C.c_void_p
        L.or_gs_scale.argtypes = [C.c_int, _ip, _ip, _dp, vp, C.c_double, vp]
        L.or_gs_scale_sym.argtypes = [C.c_int, _ip, _ip, _dp, vp, C.c_double, _dp, vp]
        L.or_spmv.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
        L.or_metric_weights.argtypes = [C.c_int, _ip, _dp, _dp]
        L.or_arnoldi.argtypes = [C.c_int, _ip, _ip, _dp, _dp, C.c_int, _dp, _dp]
        L.or_gmres.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_int, C.c_double,
                               C.c_int, vp, vp, C.POINTER(_Info), vp, vp, C.c_int]
        L.or_bicgstab.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_int,
                                  C.c_int, vp, vp, C.POINTER(_Info), vp, vp, C.c_int]
        L.or_ilu0.argtypes = [C.c_int, _ip, _ip, _dp, _dp]
        L.or_ilu0_apply.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
        L.or_ilu0_apply.restype = None
        _lib = L
    return _lib


def _csr(rowptr, colidx, val):
    return (np.ascontiguousarray(rowptr, dtype=np.int32),
            np.ascontiguousarray(colidx, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st):
    if st != 0:
        raise OracleError(_ERRORS.get(st, f"status {st}"))


def gs_scale(rowptr, colidx, val, b=None, p=2.0):
    """GS(p), Eq. (2): returns (D A values, D b or None, d) with d_i = 1/||a_i||_p."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    val = val.copy()
    n = len(rowptr) - 1
    bb = None if b is None else np.array(b, dtype=np.float64)
    d = np.empty(n)
    _check(lib().or_gs_scale(n, rowptr, colidx, val, _ptr(bb), float(p), _ptr(d)))
    return val, bb, d


def gs_scale_sym(rowptr, colidx, val, b=None, p=2.0):
    """Two-sided GS (Sec. 2): returns (D^1/2 A D^1/2 values, D^1/2 b or None,
    s, w) with s_i = (1/||a_i||_p)^(1/2) and w the stopping-metric weights
    of the scaled system (w_i = (1/||a_i||_2) / s_i)."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    val = val.copy()
    n = len(rowptr) - 1
    bb = None if b is None else np.array(b, dtype=np.float64)
    s = np.empty(n)
    w = np.empty(n)
    _check(lib().or_gs_scale_sym(n, rowptr, colidx, val, _ptr(bb), float(p), s, _ptr(w)))
    return val, bb, s, w


def spmv(rowptr, colidx, val, x):
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(len(rowptr) - 1)
    lib().or_spmv(len(y), rowptr, colidx, val, x, y)
    return y


def metric_weights(rowptr, val):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    w = np.empty(len(rowptr) - 1)
    _check(lib().or_metric_weights(len(w), rowptr, val, w))
    return w


def arnoldi(rowptr, colidx, val, v0, k):
    """k CGS2 Arnoldi steps: returns (V [n, k+1] column-major as columns, H [(k+1), k], steps)."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    n = len(rowptr) - 1
    V = np.zeros((k + 1) * n)
    H = np.zeros((k + 1) * k)
    steps = lib().or_arnoldi(n, rowptr, colidx, val, np.ascontiguousarray(v0, dtype=np.float64), k, V, H)
    return V.reshape(k + 1, n).T, H.reshape(k, k + 1).T, steps


def ilu0(rowptr, colidx, val):
    """ILU(0) factors (Saad Alg. 10.4) on A's pattern: L unit lower and U
    stored together in A's layout."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    lu = np.empty_like(val)
    _check(lib().or_ilu0(len(rowptr) - 1, rowptr, colidx, val, lu))
    return lu


def ilu0_apply(rowptr, colidx, lu, r):
    """z = (LU)^-1 r."""
    rowptr, colidx, lu = _csr(rowptr, colidx, lu)
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.empty_like(r)
    lib().or_ilu0_apply(len(r), rowptr, colidx, lu, r, z)
    return z


def gmres(rowptr, colidx, val, b, m=30, tol=1e-8, maxit=10000, x0=None, w=None, history=False, lu=None,
          trace=False):
    """Restarted GMRES(m) with CGS2, right-preconditioned by ILU(0) factors
    lu when given; returns (x, info dict[, history][, cycles]).  With
    trace=True, cycles is a list of dicts, one per cycle: steps, tau (the
    least-squares target it ran with), est (its last estimate) and mu (the
    weighted metric after it)."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    n = len(rowptr) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    hist = np.full(maxit, np.nan) if history else None
    cap = maxit + 1
    tr = np.full(4 * cap, np.nan) if trace else None
    info = _Info()
    lu = None if lu is None else np.ascontiguousarray(lu, dtype=np.float64)
    _check(lib().or_gmres(n, rowptr, colidx, val, b, x, int(m), float(tol), int(maxit),
                          _ptr(ww), _ptr(lu), C.byref(info), _ptr(hist), _ptr(tr), cap if trace else 0))
    d = info.as_dict()
    out = [x, d]
    if history:
        out.append(hist[: d["iters"]])
    if trace:
        t = tr.reshape(cap, 4)
        out.append([dict(steps=int(r[0]), tau=float(r[1]), est=float(r[2]), mu=float(r[3]))
                    for r in t if not np.isnan(r[0])])
    return tuple(out)


def bicgstab(rowptr, colidx, val, b, tol=1e-8, maxit=10000, refresh=3, x0=None, w=None, history=False, lu=None,
             trace=False):
    """Bi-CGSTAB with true-residual confirmation, right-preconditioned by
    ILU(0) factors lu when given; returns (x, info dict[, history][, checks]).
    With trace=True, checks lists each true-residual confirmation as a dict:
    iters (the count at that point) and mu (the true metric found)."""
    rowptr, colidx, val = _csr(rowptr, colidx, val)
    n = len(rowptr) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    hist = np.full(maxit, np.nan) if history else None
    cap = int(refresh) + 2
    tr = np.full(2 * cap, np.nan) if trace else None
    info = _Info()
    lu = None if lu is None else np.ascontiguousarray(lu, dtype=np.float64)
    _check(lib().or_bicgstab(n, rowptr, colidx, val, b, x, float(tol), int(maxit), int(refresh),
                             _ptr(ww), _ptr(lu), C.byref(info), _ptr(hist), _ptr(tr), cap if trace else 0))
    d = info.as_dict()
    out = [x, d]
    if history:
        out.append(hist[: d["iters"]])
    if trace:
        t = tr.reshape(cap, 2)
        out.append([dict(iters=int(r[0]), mu=float(r[1])) for r in t if not np.isnan(r[0])])
    return tuple(out)


def relres(rowptr, colidx, val, b, x, x0=None, w=None):
    """The stopping metric of Sec. 2.2 for a given x: ||W(b - Ax)|| / ||W(b - Ax0)||."""
    if w is None:
        w = metric_weights(rowptr, val)
    r = np.asarray(b) - spmv(rowptr, colidx, val, x)
    r0 = np.asarray(b) - (0.0 if x0 is None else spmv(rowptr, colidx, val, x0))
    return float(np.linalg.norm(w * r) / np.linalg.norm(w * r0))


def dense_solve(A, b):
    """LAPACK LU with partial pivoting (numpy), an independent check."""
    return np.linalg.solve(A, b)


def lp_norm_def(row, p):
    """||x||_p straight from its definition, for tiny hand-built rows in tests."""
    row = np.abs(np.asarray(row, dtype=np.float64))
    if math.isinf(p):
        return float(row.max())
    return float((row**p).sum() ** (1.0 / p))
