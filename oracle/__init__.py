"""Python view of the FP64 CPU oracle (``hec_oracle.c``).

TEST INFRASTRUCTURE ONLY: the correctness reference for the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The library under test never
imports it and shares no code with it.

The C source is compiled on first use (``gcc -O2 -ffp-contract=off``) into
``oracle/_build/liboracle.so``; ``build()`` forces that step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hec_oracle.c")
_HDR = os.path.join(_HERE, "hec_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID = -1
ERR_ZERO_PIVOT = -3
MAXIT = 1
BREAKDOWN = 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-Wall", "-Wno-unused-variable", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int), ("rp", C.POINTER(C.c_int)), ("ci", C.POINTER(C.c_int)),
                ("va", C.POINTER(C.c_double)), ("lev", C.POINTER(C.c_int))]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_resid", C.c_double), ("est_resid", C.c_double)]


_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_spmv.argtypes = [C.c_int, _ip, _ip, _dp, C.c_double, _dp, C.c_double, _dp]
            lib.orc_spmv.restype = None
            lib.orc_spmv_range.argtypes = [C.c_int, _ip, _ip, _dp, C.c_double, _dp, C.c_double,
                                           _dp, C.c_int, C.c_int]
            lib.orc_spmv_range.restype = None
            lib.orc_dot.argtypes = [C.c_int, _dp, _dp]
            lib.orc_dot.restype = C.c_double
            lib.orc_nrm2.argtypes = [C.c_int, _dp]
            lib.orc_nrm2.restype = C.c_double
            lib.orc_axpby.argtypes = [C.c_int, C.c_double, _dp, C.c_double, _dp]
            lib.orc_axpby.restype = None
            lib.orc_waxpby.argtypes = [C.c_int, C.c_double, _dp, C.c_double, _dp, _dp]
            lib.orc_waxpby.restype = None
            lib.orc_iluk.argtypes = [C.c_int, _ip, _ip, _dp, C.c_int, C.POINTER(_CSR)]
            lib.orc_iluk.restype = C.c_int
            lib.orc_csr_free.argtypes = [C.POINTER(_CSR)]
            lib.orc_csr_free.restype = None
            lib.orc_levels.argtypes = [C.c_int, _ip, _ip, C.c_int, _ip]
            lib.orc_levels.restype = C.c_int
            lib.orc_lsolve_unit.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
            lib.orc_lsolve_unit.restype = None
            lib.orc_usolve.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp]
            lib.orc_usolve.restype = C.c_int
            lib.orc_ras_setup.argtypes = [C.c_int, _ip, _ip, _dp, C.c_int, C.c_int, C.c_int,
                                          C.POINTER(C.c_int)]
            lib.orc_ras_setup.restype = C.c_void_p
            lib.orc_ras_apply.argtypes = [C.c_void_p, _dp, _dp]
            lib.orc_ras_apply.restype = None
            lib.orc_ras_nblocks.argtypes = [C.c_void_p]
            lib.orc_ras_nblocks.restype = C.c_int
            lib.orc_ras_block_size.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                               C.POINTER(C.c_int)]
            lib.orc_ras_block_size.restype = C.c_int
            lib.orc_ras_block_rows.argtypes = [C.c_void_p, C.c_int, _ip]
            lib.orc_ras_block_rows.restype = None
            lib.orc_ras_block_factor.argtypes = [C.c_void_p, C.c_int]
            lib.orc_ras_block_factor.restype = C.POINTER(_CSR)
            lib.orc_ras_free.argtypes = [C.c_void_p]
            lib.orc_ras_free.restype = None
            lib.orc_jacobi_setup.argtypes = [C.c_int, _ip, _ip, _dp, C.c_double,
                                             C.POINTER(C.c_int)]
            lib.orc_jacobi_setup.restype = C.c_void_p
            for name in ("orc_bicgstab", "orc_cg"):
                f = getattr(lib, name)
                f.argtypes = [C.c_int, _ip, _ip, _dp, C.c_void_p, _dp, _dp, C.c_double, C.c_int,
                              C.POINTER(_Info)]
                f.restype = C.c_int
            lib.orc_gmres.argtypes = [C.c_int, _ip, _ip, _dp, C.c_void_p, _dp, _dp, C.c_double,
                                      C.c_int, C.c_int, C.POINTER(_Info)]
            lib.orc_gmres.restype = C.c_int
            _lib = lib
    return _lib


def _arrs(A):
    return (np.ascontiguousarray(A.row_ptr, np.int32), np.ascontiguousarray(A.col, np.int32),
            np.ascontiguousarray(A.val, np.float64))


class Factor:
    """A combined ILU factor (L strictly below the diagonal, U on and above)."""

    def __init__(self, n, row_ptr, col, val, lev):
        self.n = n
        self.row_ptr = row_ptr
        self.col = col
        self.val = val
        self.lev = lev

    def split(self):
        """Return (L, U) as (row_ptr, col, val) triples; L strictly lower, U upper incl. diag."""
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        out = []
        for mask in (self.col < rows, self.col >= rows):
            r = rows[mask]
            rp = np.zeros(self.n + 1, np.int32)
            np.cumsum(np.bincount(r, minlength=self.n), out=rp[1:])
            out.append((rp, self.col[mask].copy(), self.val[mask].copy()))
        return out[0], out[1]

    def to_dense(self):
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def _factor_from(cs: _CSR) -> Factor:
    n = cs.n
    rp = np.ctypeslib.as_array(cs.rp, shape=(n + 1,)).copy()
    nnz = int(rp[-1])
    ci = np.ctypeslib.as_array(cs.ci, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    va = np.ctypeslib.as_array(cs.va, shape=(nnz,)).copy() if nnz else np.zeros(0)
    lev = np.ctypeslib.as_array(cs.lev, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    return Factor(n, rp, ci, va, lev)


# ---------------------------------------------------------------- vector ops
def spmv(A, x, alpha=1.0, beta=0.0, y=None):
    """Eq. 2: alpha*A*x + beta*y (new array)."""
    rp, ci, va = _arrs(A)
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros(A.n) if y is None else np.array(y, dtype=np.float64, copy=True)
    _load().orc_spmv(A.n, rp, ci, va, float(alpha), x, float(beta), out)
    return out


def spmv_rows(A, x, lo: int, hi: int):
    """Rows [lo, hi) of A x (the oracle's row loop on that range)."""
    rp, ci, va = _arrs(A)
    y = np.zeros(A.n)
    _load().orc_spmv_range(A.n, rp, ci, va, 1.0, np.ascontiguousarray(x, np.float64), 0.0, y,
                           int(lo), int(hi))
    return y[lo:hi]


def spmv_threads(A, x, threads: int):
    """y = A x with the oracle's row loop split into `threads` row ranges run
    on host threads (the library call releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    rp, ci, va = _arrs(A)
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros(A.n)
    cuts = np.linspace(0, A.n, threads + 1).astype(int)
    lib = _load()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda t: lib.orc_spmv_range(A.n, rp, ci, va, 1.0, x, 0.0, y,
                                                 int(cuts[t]), int(cuts[t + 1])), range(threads)))
    return y


def dot(x, y):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    return _load().orc_dot(x.shape[0], x, y)


def nrm2(x):
    x = np.ascontiguousarray(x, np.float64)
    return _load().orc_nrm2(x.shape[0], x)


def axpby(a, x, b, y):
    """Eq. 3: returns a*x + b*y."""
    out = np.array(y, dtype=np.float64, copy=True)
    _load().orc_axpby(out.shape[0], float(a), np.ascontiguousarray(x, np.float64), float(b), out)
    return out


def waxpby(a, x, b, y):
    """Eq. 4: returns z = a*x + b*y."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.empty_like(x)
    _load().orc_waxpby(x.shape[0], float(a), x, float(b), y, z)
    return z


# ---------------------------------------------------------------- ILU(k), levels, solves
def iluk(A, k: int) -> Factor:
    """Eqs. 9-10 / Algorithm 2.  Raises on zero pivot or invalid input."""
    rp, ci, va = _arrs(A)
    cs = _CSR()
    st = _load().orc_iluk(A.n, rp, ci, va, int(k), C.byref(cs))
    if st != OK:
        raise OracleError(st)
    try:
        return _factor_from(cs)
    finally:
        _load().orc_csr_free(C.byref(cs))


def levels(n, row_ptr, col, upper: bool):
    """Eq. 11: per-row level (1-based) and level count."""
    lev = np.zeros(n, np.int32)
    nlev = _load().orc_levels(n, np.ascontiguousarray(row_ptr, np.int32),
                              np.ascontiguousarray(col, np.int32), int(bool(upper)), lev)
    return lev, nlev


def level_sets(lev, nlev):
    """Canonical (level_ptr, level_rows): rows ascending inside each level."""
    order = np.lexsort((np.arange(lev.shape[0]), lev)).astype(np.int32)
    ptr = np.zeros(nlev + 1, np.int32)
    np.cumsum(np.bincount(lev - 1, minlength=nlev), out=ptr[1:])
    return ptr, order


def lsolve_unit(F: Factor, b):
    y = np.zeros(F.n)
    _load().orc_lsolve_unit(F.n, F.row_ptr, F.col, F.val, np.ascontiguousarray(b, np.float64), y)
    return y


def usolve(F: Factor, y):
    z = np.zeros(F.n)
    st = _load().orc_usolve(F.n, F.row_ptr, F.col, F.val, np.ascontiguousarray(y, np.float64), z)
    if st != OK:
        raise OracleError(st)
    return z


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__("oracle status %d" % status)
        self.status = status


# ---------------------------------------------------------------- RAS
class RAS:
    """Section 2.5 restricted additive Schwarz with per-block ILU(k)."""

    def __init__(self, A, k: int, nblocks: int, overlap: int):
        rp, ci, va = _arrs(A)
        st = C.c_int(0)
        self._h = _load().orc_ras_setup(A.n, rp, ci, va, int(k), int(nblocks), int(overlap),
                                        C.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.n = A.n
        self.nblocks = nblocks

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_ras_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def apply(self, r):
        z = np.zeros(self.n)
        _load().orc_ras_apply(self._h, np.ascontiguousarray(r, np.float64), z)
        return z

    def block(self, b):
        """(rows of V_b, own_lo, own_hi, Factor)."""
        lo, hi = C.c_int(0), C.c_int(0)
        nv = _load().orc_ras_block_size(self._h, b, C.byref(lo), C.byref(hi))
        rows = np.zeros(nv, np.int32)
        _load().orc_ras_block_rows(self._h, b, rows)
        F = _factor_from(_load().orc_ras_block_factor(self._h, b).contents)
        return rows, lo.value, hi.value, F


class Jacobi(RAS):
    """Damped Jacobi z = omega D^{-1} r (a smoother the paper builds from
    SpMV and vector operations), usable wherever a RAS object is."""

    def __init__(self, A, omega: float = 1.0):
        rp, ci, va = _arrs(A)
        st = C.c_int(0)
        self._h = _load().orc_jacobi_setup(A.n, rp, ci, va, float(omega), C.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.n = A.n
        self.nblocks = 0
        self.omega = omega


# ---------------------------------------------------------------- Krylov
class Info:
    def __init__(self, ci: _Info):
        self.iters = ci.iters
        self.restarts = ci.restarts
        self.status = ci.status
        self.rel_resid = ci.rel_resid
        self.est_resid = ci.est_resid

    def __repr__(self):
        return ("Info(iters=%d, restarts=%d, status=%d, rel_resid=%.3e, est_resid=%.3e)"
                % (self.iters, self.restarts, self.status, self.rel_resid, self.est_resid))


def bicgstab(A, b, M=None, x0=None, tol=1e-8, maxit=1000):
    """Right-preconditioned BiCGSTAB (Section 2.7; the van der Vorst 1992 /
    Saad Section 7.4.2 recurrences on A M^{-1}).  M: a RAS object or None.
    Returns (x, Info)."""
    rp, ci, va = _arrs(A)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = _Info()
    _load().orc_bicgstab(A.n, rp, ci, va, M.handle if M is not None else None,
                         np.ascontiguousarray(b, np.float64), x, float(tol), int(maxit),
                         C.byref(info))
    return x, Info(info)


def cg(A, b, M=None, x0=None, tol=1e-8, maxit=1000):
    """Preconditioned conjugate gradients.  M: RAS, Jacobi or None."""
    rp, ci, va = _arrs(A)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = _Info()
    _load().orc_cg(A.n, rp, ci, va, M.handle if M is not None else None,
                   np.ascontiguousarray(b, np.float64), x, float(tol), int(maxit), C.byref(info))
    return x, Info(info)


def gmres(A, b, M=None, x0=None, tol=1e-8, maxit=1000, restart=30):
    """Restarted right-preconditioned GMRES(m).  Returns (x, Info)."""
    rp, ci, va = _arrs(A)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = _Info()
    st = _load().orc_gmres(A.n, rp, ci, va, M.handle if M is not None else None,
                           np.ascontiguousarray(b, np.float64), x, float(tol), int(maxit),
                           int(restart), C.byref(info))
    if st == ERR_INVALID:
        raise OracleError(st)
    return x, Info(info)
