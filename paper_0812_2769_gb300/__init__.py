"""Python binding of libgsk: geometric scaling GS(p) with restarted GMRES(m)
and Bi-CGSTAB on GB300 (sm_103a).

This module only marshals arguments to the C ABI declared in
``include/gsk.h``: torch tensors supply device memory and streams, and every
step of the computation runs in the library's CUDA kernels.  There is no CPU
path: if ``libgsk.so`` has not been built, loading raises.

Typical use::

    import torch, paper_0812_2769_gb300 as gsk
    A = gsk.Csr.from_host(rowptr, colidx, val, device="cuda")
    b = torch.as_tensor(rhs, device="cuda")
    gsk.gs_scale(A, b, p=2.0)                 # Sec. 2, Eq. (2)
    x = torch.zeros_like(b)
    info = gsk.bicgstab_solve(A, b, x, tol=1e-8)
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsk.so")

OK, ERR_ARG, ERR_ZERO_ROW, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = range(7)
F64, F32 = 0, 1
CONVERGED, MAXIT, BREAKDOWN, STAGNATED = 0, 1, 2, 3
CONV_NAMES = {0: "converged", 1: "maxit", 2: "breakdown", 3: "stagnated"}
METRIC_GS2, METRIC_PLAIN = 0, 1
PREC_F64, PREC_MIXED = 0, 1
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_ZERO_ROW", 3: "ERR_NONFINITE", 4: "ERR_OOM", 5: "ERR_CUDA",
                6: "ERR_TIMEOUT"}


class GskError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CsrC(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("val", C.c_void_p), ("dtype", C.c_int32)]


class OptsC(C.Structure):
    _fields_ = [("maxit", C.c_int32), ("refresh", C.c_int32), ("precision", C.c_int32), ("metric", C.c_int32),
                ("weights", C.c_void_p), ("inner_tol", C.c_double), ("inner_maxit", C.c_int32),
                ("max_refinements", C.c_int32), ("precond", C.c_void_p), ("batch_block", C.c_int32),
                ("batch_large_n", C.c_int32)]


class InfoC(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("refreshes", C.c_int32),
                ("refinements", C.c_int32), ("conv", C.c_int32), ("relres_true", C.c_double),
                ("relres_rec", C.c_double), ("ms", C.c_float)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["conv_name"] = CONV_NAMES.get(self.conv, str(self.conv))
        return d


class LaunchRecordC(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("step", C.c_int32), ("ms", C.c_float)]


_lib = None

# every entry point of include/gsk.h, with its ctypes signature
SIGNATURES = {
    "gsk_version": ([], C.c_char_p),
    "gsk_ctx_create": ([C.POINTER(C.c_void_p), C.c_int], C.c_int),
    "gsk_ctx_destroy": ([C.c_void_p], C.c_int),
    "gsk_last_error": ([C.c_void_p], C.c_char_p),
    "gsk_opts_default": ([C.POINTER(OptsC)], None),
    "gs_scale": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "gsk_profile_gs_scale": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                              C.POINTER(C.c_float)], C.c_int),
    "gs_scale_static": ([C.POINTER(CsrC), C.c_void_p, C.c_double, C.c_void_p, C.c_void_p], C.c_int),
    "gs_scale_sym": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p],
                     C.c_int),
    "gsk_diag_mul": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "gsk_ilu0_create": ([C.c_void_p, C.POINTER(CsrC), C.POINTER(C.c_void_p), C.c_void_p], C.c_int),
    "gsk_ilu0_destroy": ([C.c_void_p], C.c_int),
    "gsk_ilu0_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gsk_ilu0_info": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "gsk_spmv": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "gmres_solve": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                     C.POINTER(OptsC), C.POINTER(InfoC), C.c_void_p], C.c_int),
    "gsk_arnoldi": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                     C.c_void_p], C.c_int),
    "bicgstab_solve": ([C.c_void_p, C.POINTER(CsrC), C.c_void_p, C.c_void_p, C.c_double,
                        C.POINTER(OptsC), C.POINTER(InfoC), C.c_void_p], C.c_int),
    "gsk_workspace_bytes": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
    "gsk_small_system_rows": ([C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "gsk_gmres_small_system_rows": ([C.c_void_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "gsk_kernel_name": ([C.c_int], C.c_char_p),
    "bicgstab_solve_batched": ([C.c_void_p, C.c_int, C.POINTER(CsrC), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_double), C.c_double, C.POINTER(OptsC), C.POINTER(InfoC),
                                C.POINTER(C.c_int32), C.c_void_p], C.c_int),
    "gmres_solve_batched": ([C.c_void_p, C.c_int, C.POINTER(CsrC), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                             C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_double, C.POINTER(OptsC),
                             C.POINTER(InfoC), C.POINTER(C.c_int32), C.c_void_p], C.c_int),
    "gsk_profile_solve": ([C.c_void_p, C.c_int, C.POINTER(CsrC), C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                           C.POINTER(OptsC), C.c_int, C.POINTER(LaunchRecordC), C.c_int, C.POINTER(C.c_int),
                           C.POINTER(InfoC), C.c_void_p], C.c_int),
}


def lib():
    """Load libgsk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_0812_2769_gb300.build` "
                              "(or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def version() -> str:
    return lib().gsk_version().decode()


class Context:
    """A library context on one CUDA device (workspace, cached graphs)."""

    def __init__(self, device: int = 0):
        self.device = device
        self._h = C.c_void_p()
        st = lib().gsk_ctx_create(C.byref(self._h), device)
        if st != OK:
            raise GskError(st, "gsk_ctx_create failed")

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return lib().gsk_last_error(self._h).decode()

    def check(self, st: int):
        if st != OK:
            raise GskError(st, self.last_error())

    def close(self):
        if self._h:
            lib().gsk_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


_default_ctx: dict[int, Context] = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


def _torch():
    import torch

    return torch


@dataclass
class Csr:
    """A device CSR matrix held in torch tensors (int32 indices)."""

    rowptr: object
    colidx: object
    val: object

    @property
    def n(self) -> int:
        return int(self.rowptr.numel()) - 1

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    @property
    def dtype(self) -> int:
        return F64 if self.val.dtype == _torch().float64 else F32

    @classmethod
    def from_host(cls, rowptr, colidx, val, device="cuda", dtype=None):
        torch = _torch()
        val_t = torch.as_tensor(val)
        if dtype is not None:
            val_t = val_t.to(dtype)
        return cls(torch.as_tensor(rowptr, dtype=torch.int32).to(device).contiguous(),
                   torch.as_tensor(colidx, dtype=torch.int32).to(device).contiguous(),
                   val_t.to(device).contiguous())

    def c(self) -> CsrC:
        return CsrC(self.n, self.nnz, self.rowptr.data_ptr(), self.colidx.data_ptr(), self.val.data_ptr(),
                    self.dtype)


def _stream_ptr(stream):
    if stream is None:
        return C.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def opts(maxit=10000, refresh=3, precision=PREC_F64, metric=METRIC_GS2, weights=None, inner_tol=1e-5,
         inner_maxit=0, max_refinements=0, precond=None, batch_block=0, batch_large_n=0) -> OptsC:
    """Solver options; precond: an Ilu0 of the matrix being solved (applied on
    the right), or None; batch_block / batch_large_n: the batched solvers'
    block size and grid-wide threshold (0 = defaults; see autotune)."""
    o = OptsC()
    lib().gsk_opts_default(C.byref(o))
    o.maxit, o.refresh, o.precision, o.metric = maxit, refresh, precision, metric
    o.weights = None if weights is None else weights.data_ptr()
    o.inner_tol, o.inner_maxit, o.max_refinements = inner_tol, inner_maxit, max_refinements
    o.precond = None if precond is None else precond.handle
    o.batch_block, o.batch_large_n = batch_block, batch_large_n
    return o


class Ilu0:
    """ILU(0) factors of a device CSR matrix (FP64, diagonal present, sorted
    columns), computed on the device by gsk_ilu0_create; use as
    opts(precond=...) or apply z = (LU)^-1 r with apply().  Keeps a reference
    to the matrix, whose structure the factors share."""

    def __init__(self, A: Csr, ctx: Context | None = None, stream=None):
        self.ctx = ctx or default_context(A.val.device.index or 0)
        self.A = A
        self._h = C.c_void_p()
        Ac = A.c()
        self.ctx.check(lib().gsk_ilu0_create(self.ctx.handle, C.byref(Ac), C.byref(self._h), _stream_ptr(stream)))

    @property
    def handle(self):
        return self._h

    def apply(self, r, z=None, stream=None):
        if z is None:
            z = _torch().empty_like(r)
        self.ctx.check(lib().gsk_ilu0_apply(self.ctx.handle, self._h, _ptr(r), _ptr(z), _stream_ptr(stream)))
        return z

    def info(self) -> dict:
        """Levels of the forward and backward sweeps and whether they run in
        one thread block (z in shared memory) or across the grid."""
        lo, up, one = C.c_int(0), C.c_int(0), C.c_int(0)
        self.ctx.check(lib().gsk_ilu0_info(self._h, C.byref(lo), C.byref(up), C.byref(one)))
        return {"levels_lower": lo.value, "levels_upper": up.value, "one_block": bool(one.value)}

    def close(self):
        if self._h:
            lib().gsk_ilu0_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown
            pass


def gs_scale(A: Csr, b=None, p: float = 2.0, d_out=None, ctx: Context | None = None, stream=None):
    """GS(p) in place on A (and b): row i divided by ||a_i||_p (Sec. 2, Eq. (2)),
    in one pass.  On error (GskError) only the rows that caused it are left
    unscaled; gs_scale_static leaves A and b untouched on error."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    ctx.check(lib().gs_scale(ctx.handle, C.byref(Ac), _ptr(b), float(p), _ptr(d_out), _stream_ptr(stream)))
    return d_out


def gs_scale_static(A: Csr, b=None, p: float = 2.0, d_out=None, stream=None):
    """GS(p) in place without any device allocation (no context): for callers
    that may not allocate device memory.  Scratch is a fixed array inside the
    library (at most 1,048,576 rows when d_out is None); calls that overlap on
    the GPU race on it.  Raises GskError with the status on failure."""
    Ac = A.c()
    with _torch().cuda.device(A.val.device):  # the library's array on A's device
        st = lib().gs_scale_static(C.byref(Ac), _ptr(b), float(p), _ptr(d_out), _stream_ptr(stream))
    if st != OK:
        raise GskError(st, "gs_scale_static failed")
    return d_out


def gs_scale_sym(A: Csr, b=None, p: float = 2.0, weights: bool = False, s_out=None, w_out=None,
                 ctx: Context | None = None, stream=None):
    """Two-sided scaling in place (Sec. 2): A <- D^1/2 A D^1/2, b <- D^1/2 b
    with D = diag(1/||a_i||_p).  Returns (s, w): s = diag(D^1/2), so that
    diag_mul(s, y) turns the scaled system's solution y into x; with
    weights=True (or a w_out buffer) also w, the stopping-metric weights that
    make a solve of the scaled system stop on the GS(2)-scaled residual of
    the original system (pass opts(weights=w)); else w is None."""
    import torch

    ctx = ctx or default_context(A.val.device.index or 0)
    if s_out is None:
        s_out = torch.empty(A.n, dtype=torch.float64, device=A.val.device)
    if w_out is None and weights:
        w_out = torch.empty(A.n, dtype=torch.float64, device=A.val.device)
    Ac = A.c()
    ctx.check(lib().gs_scale_sym(ctx.handle, C.byref(Ac), _ptr(b), float(p), _ptr(s_out), _ptr(w_out),
                                 _stream_ptr(stream)))
    return s_out, w_out


def diag_mul(s, x, ctx: Context | None = None, stream=None):
    """x <- s * x on the device (x FP64 or FP32, s FP64)."""
    import torch

    ctx = ctx or default_context(x.device.index or 0)
    dt = F64 if x.dtype == torch.float64 else F32
    ctx.check(lib().gsk_diag_mul(ctx.handle, int(x.numel()), _ptr(s), _ptr(x), dt, _stream_ptr(stream)))
    return x


def gsk_spmv(A: Csr, x, y, ctx: Context | None = None, stream=None):
    """y = A x on the device."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    ctx.check(lib().gsk_spmv(ctx.handle, C.byref(Ac), _ptr(x), _ptr(y), _stream_ptr(stream)))
    return y


def gmres_solve(A: Csr, b, x, m: int = 30, tol: float = 1e-8, options: OptsC | None = None,
                ctx: Context | None = None, stream=None, sync: bool = True):
    """Restarted GMRES(m) with CGS2 (Sec. 2); x holds x0 on entry, the solution on exit."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    info = InfoC()
    o = options if options is not None else opts()
    ctx.check(lib().gmres_solve(ctx.handle, C.byref(Ac), _ptr(b), _ptr(x), int(m), float(tol), C.byref(o),
                                C.byref(info) if sync else None, _stream_ptr(stream)))
    return info.as_dict() if sync else None


def arnoldi(A: Csr, v0, m: int, ctx: Context | None = None, stream=None):
    """m steps of GMRES's Arnoldi process (CGS2, Sec. 2) on the device from
    v0; returns (H, k): H the (k+1) x k Hessenberg matrix (numpy FP64) with
    A V_k = V_{k+1} H, k <= m the steps taken (fewer at an invariant
    subspace).  The eigenvalues of H[:k, :k] are the Ritz values."""
    import numpy as np

    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    H = np.zeros((m, m + 1), dtype=np.float64)  # column-major (m+1) x m, transposed view
    k = C.c_int(0)
    ctx.check(lib().gsk_arnoldi(ctx.handle, C.byref(Ac), _ptr(v0), int(m),
                                H.ctypes.data_as(C.POINTER(C.c_double)), C.byref(k), _stream_ptr(stream)))
    k = k.value
    return np.ascontiguousarray(H.T[: k + 1, :k]), k


def bicgstab_solve(A: Csr, b, x, tol: float = 1e-8, options: OptsC | None = None, ctx: Context | None = None,
                   stream=None, sync: bool = True):
    """Bi-CGSTAB (Sec. 2); x holds x0 on entry, the solution on exit."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    info = InfoC()
    o = options if options is not None else opts()
    ctx.check(lib().bicgstab_solve(ctx.handle, C.byref(Ac), _ptr(b), _ptr(x), float(tol), C.byref(o),
                                   C.byref(info) if sync else None, _stream_ptr(stream)))
    return info.as_dict() if sync else None


def bicgstab_solve_batched(As, bs, xs, p=2.0, tol: float = 1e-8, options: OptsC | None = None,
                           ctx: Context | None = None, stream=None, sync: bool = True, check: bool = True):
    """GS(p) + Bi-CGSTAB on many systems in one persistent launch.  As: list of
    Csr; bs, xs: lists of device tensors; p: one value or a list (NaN = no
    scaling).  Returns (list of info dicts, list of statuses) when sync."""
    n = len(As)
    ctx = ctx or default_context(As[0].val.device.index or 0 if n else 0)
    arr = (CsrC * n)(*[A.c() for A in As])
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    pv = [p] * n if not isinstance(p, (list, tuple)) else list(p)
    pa = (C.c_double * n)(*[float(v) for v in pv])
    infos = (InfoC * n)() if sync else None
    stat = (C.c_int32 * n)() if sync else None
    o = options if options is not None else opts()
    st = lib().bicgstab_solve_batched(ctx.handle, n, arr, bp, xp, pa, float(tol), C.byref(o), infos, stat,
                                      _stream_ptr(stream))
    if check and st != OK:
        ctx.check(st)
    if not sync:
        return None
    return [i.as_dict() for i in infos], list(stat)


def gmres_solve_batched(As, bs, xs, m=30, p=2.0, tol: float = 1e-8, options: OptsC | None = None,
                        ctx: Context | None = None, stream=None, sync: bool = True, check: bool = True):
    """GS(p) + GMRES(m) on many systems in one persistent launch (one block per
    system; FP64).  m, p: one value or a list.  Returns (list of info dicts,
    list of statuses) when sync."""
    n = len(As)
    ctx = ctx or default_context(As[0].val.device.index or 0 if n else 0)
    arr = (CsrC * n)(*[A.c() for A in As])
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    pv = [p] * n if not isinstance(p, (list, tuple)) else list(p)
    mv = [m] * n if not isinstance(m, (list, tuple)) else list(m)
    pa = (C.c_double * n)(*[float(v) for v in pv])
    ma = (C.c_int * n)(*[int(v) for v in mv])
    infos = (InfoC * n)() if sync else None
    stat = (C.c_int32 * n)() if sync else None
    o = options if options is not None else opts()
    st = lib().gmres_solve_batched(ctx.handle, n, arr, bp, xp, pa, ma, float(tol), C.byref(o), infos, stat,
                                   _stream_ptr(stream))
    if check and st != OK:
        ctx.check(st)
    if not sync:
        return None
    return [i.as_dict() for i in infos], list(stat)


def profile_solve(A: Csr, b, x, solver: str = "bicgstab", m: int = 30, tol: float = 1e-8,
                  options: OptsC | None = None, max_iters: int = 50, ctx: Context | None = None, stream=None):
    """Run a solver's kernels from a host loop with CUDA events around each
    launch (a profiling aid).  Returns (records, info): records is a list of
    (kernel name, step, ms) in launch order."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    cap = 64 + 8 * max_iters + 16 * (max_iters // max(m, 1) + 2)
    recs = (LaunchRecordC * cap)()
    nrec = C.c_int()
    info = InfoC()
    o = options if options is not None else opts()
    ctx.check(lib().gsk_profile_solve(ctx.handle, 0 if solver == "gmres" else 1, C.byref(Ac), _ptr(b), _ptr(x),
                                      int(m), float(tol), C.byref(o), int(max_iters), recs, cap, C.byref(nrec),
                                      C.byref(info), _stream_ptr(stream)))
    out = [(lib().gsk_kernel_name(r.kernel).decode(), r.step, r.ms) for r in recs[: nrec.value]]
    return out, info.as_dict()


def profile_gs_scale(A: Csr, b=None, p: float = 2.0, d_out=None, ctx: Context | None = None, stream=None) -> float:
    """gs_scale, returning the device time of its GS(p) kernel alone in ms
    (CUDA events around the launch; a profiling aid)."""
    ctx = ctx or default_context(A.val.device.index or 0)
    Ac = A.c()
    ms = C.c_float()
    ctx.check(lib().gsk_profile_gs_scale(ctx.handle, C.byref(Ac), _ptr(b), float(p), _ptr(d_out),
                                         _stream_ptr(stream), C.byref(ms)))
    return ms.value


def gmres_small_system_rows(m: int = 30, ctx: Context | None = None) -> int:
    """The largest system (about 7 nonzeros per row) gmres_solve with restart
    length m runs on one thread-block cluster (0: the path is off)."""
    ctx = ctx or default_context(0)
    out = C.c_int()
    ctx.check(lib().gsk_gmres_small_system_rows(ctx.handle, int(m), C.byref(out)))
    return out.value


def small_system_rows(ctx: Context | None = None) -> int:
    """The largest system bicgstab_solve runs on one thread-block cluster (0:
    the path is off or unavailable)."""
    ctx = ctx or default_context(0)
    out = C.c_int()
    ctx.check(lib().gsk_small_system_rows(ctx.handle, C.byref(out)))
    return int(out.value)


def workspace_bytes(n: int, nnz: int, solver: str = "bicgstab", m: int = 30, precision: int = PREC_F64) -> int:
    out = C.c_size_t()
    st = lib().gsk_workspace_bytes(n, nnz, 0 if solver == "gmres" else 1, m, precision, C.byref(out))
    if st != OK:
        raise GskError(st, "gsk_workspace_bytes")
    return int(out.value)


INF = math.inf
