"""ctypes binding of the C ABI in ``include/hecgpu.h`` (same names, argument
marshalling only -- every step of the computation runs in the CUDA library).

Device vectors are ``torch.Tensor`` objects on a CUDA device (float64,
contiguous); host vectors are numpy arrays.  ``stream`` defaults to torch's
current stream.  Every failing call raises :class:`HecError`.  Importing this
module loads ``_build/libhecgpu.so``; if the library has not been built the
import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhecgpu.so")
# the same library compiled with HEC_DEBUG (device-side checks, see hec_debug_record)
DEBUG_LIB_PATH = os.path.join(_HERE, "_build", "debug", "libhecgpu.so")

OK = 0
ERR_INVALID = -1
ERR_OOM = -2
ERR_ZERO_PIVOT = -3
ERR_UNSORTED_CSR = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_DEBUG = -7
MAXIT = 1
BREAKDOWN = 2
GMRES = 0
BICGSTAB = 1
CG = 2
HOST_ONLY = 1
X0_ZERO = 1
SOLVE_EAGER = 2
MIXED_FP32 = 4
FACTOR_L = 0
FACTOR_U = 1
TRSV_AUTO = 0
TRSV_STREAMED = 1
TRSV_RESIDENT = 2


class HecError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s failed: status %d (%s): %s" % (where, status, _status_name(status), msg))
        self.status = status


def _status_name(s):
    return {OK: "ok", ERR_INVALID: "invalid", ERR_OOM: "oom", ERR_ZERO_PIVOT: "zero pivot",
            ERR_UNSORTED_CSR: "unsorted csr", ERR_CUDA: "cuda", ERR_TIMEOUT: "timeout",
            ERR_DEBUG: "debug check", MAXIT: "maxit", BREAKDOWN: "breakdown"}.get(s, "?")


class CSR_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32)]


class Opts_t(C.Structure):
    _fields_ = [("ell_width", C.c_int32), ("ell_ld_align", C.c_int32), ("flags", C.c_int32),
                ("reserved", C.c_int32)]


class MatrixInfo_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("ell_width", C.c_int32),
                ("ell_ld", C.c_int32), ("tail_rows", C.c_int32), ("tail_nnz", C.c_int32),
                ("device_bytes", C.c_int64)]


class PrecondInfo_t(C.Structure):
    _fields_ = [("nblocks", C.c_int32), ("overlap", C.c_int32), ("k", C.c_int32),
                ("scheduled", C.c_int32), ("rows_total", C.c_int64), ("factor_nnz", C.c_int64),
                ("max_levels_L", C.c_int32), ("max_levels_U", C.c_int32),
                ("apply_bytes", C.c_int64), ("device_bytes", C.c_int64),
                ("ring_slots", C.c_int32), ("global_passes", C.c_int32),
                ("apply_bytes_f32", C.c_int64), ("trsv_parts", C.c_int32),
                ("import_slots", C.c_int32), ("split_blocks", C.c_int32),
                ("trsv_resident", C.c_int32)]


class SolveOpts_t(C.Structure):
    _fields_ = [("method", C.c_int32), ("flags", C.c_int32), ("spin_limit", C.c_int64)]


class SolveInfo_t(C.Structure):
    _fields_ = [("iters", C.c_int32), ("restarts", C.c_int32), ("status", C.c_int32),
                ("fp64_finish", C.c_int32), ("rel_resid", C.c_double), ("est_resid", C.c_double),
                ("kernel_launches", C.c_int64), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64)]


class BatchCSR_t(C.Structure):
    _fields_ = [("nsys", C.c_int32), ("reserved", C.c_int32), ("sys_ptr", C.c_void_p),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class BatchConfig_t(C.Structure):
    _fields_ = [("threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("ell_width", C.c_int32),
                ("nstages", C.c_int32)]


class BatchInfo_t(C.Structure):
    _fields_ = [("nsys", C.c_int32), ("ilu_k", C.c_int32), ("rows", C.c_int64),
                ("nnz", C.c_int64), ("factor_nnz", C.c_int64), ("max_n", C.c_int32),
                ("ring_slots", C.c_int32), ("device_bytes", C.c_int64),
                ("config", BatchConfig_t)]


class BatchSysInfo_t(C.Structure):
    _fields_ = [("iters", C.c_int32), ("cycles", C.c_int32), ("status", C.c_int32),
                ("reorth", C.c_int32), ("rel_resid", C.c_double)]


class ServerOpts_t(C.Structure):
    _fields_ = [("device_budget", C.c_int64), ("lanes", C.c_int32), ("restart", C.c_int32),
                ("maxit", C.c_int32), ("flags", C.c_int32), ("tol", C.c_double),
                ("small_rows", C.c_int32), ("block_rows", C.c_int32),
                ("keep_solutions", C.c_int32), ("reserved", C.c_int32)]


class Request_t(C.Structure):
    _fields_ = [("A", CSR_t), ("b", C.c_void_p), ("ilu_k", C.c_int32), ("reserved", C.c_int32),
                ("key", C.c_uint64), ("tag", C.c_uint64)]


class Result_t(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("tag", C.c_uint64), ("status", C.c_int32),
                ("iters", C.c_int32), ("rel_resid", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_setup", C.c_double), ("t_done", C.c_double),
                ("lane", C.c_int32), ("reused", C.c_int32), ("fp64_finish", C.c_int32),
                ("refactored", C.c_int32), ("device_bytes", C.c_int64)]


_vp = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_dbl = C.c_double

_SIGS = {
    "hec_status_string": ([C.c_int], C.c_char_p),
    "hec_last_error": ([], C.c_char_p),
    "hec_set_allocator": ([_vp, _vp, _vp], C.c_int),
    "hec_build": ([C.POINTER(CSR_t), C.POINTER(Opts_t), _vp, C.POINTER(_vp)], C.c_int),
    "hec_matrix_info": ([_vp, C.POINTER(MatrixInfo_t)], C.c_int),
    "hec_matrix_export": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "hec_matrix_destroy": ([_vp], None),
    "hec_spmv": ([_vp, _dbl, _vp, _dbl, _vp, _vp, _vp, _vp, _vp], C.c_int),
    "hec_spmv_f32": ([_vp, C.c_float, _vp, C.c_float, _vp, _vp, _vp], C.c_int),
    "hec_axpby": ([_i32, _dbl, _vp, _dbl, _vp, _vp], C.c_int),
    "hec_waxpby": ([_i32, _dbl, _vp, _dbl, _vp, _vp, _vp], C.c_int),
    "hec_dot": ([_i32, _vp, _vp, _vp, _vp], C.c_int),
    "hec_nrm2": ([_i32, _vp, _vp, _vp], C.c_int),
    "hec_multidot": ([_i32, _i32, _vp, _i64, _vp, _vp, _vp], C.c_int),
    "ilu_k_setup": ([_vp, _i32, _i32, _i32, _vp, C.POINTER(_vp)], C.c_int),
    "hec_jacobi_setup": ([_vp, C.c_double, _vp, C.POINTER(_vp)], C.c_int),
    "hec_refactor": ([_vp, _vp, _vp, _vp], C.c_int),
    "level_schedule": ([_vp, _vp], C.c_int),
    "hec_precond_info": ([_vp, C.POINTER(PrecondInfo_t)], C.c_int),
    "hec_precond_get_block": ([_vp, _i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32), _vp],
                              C.c_int),
    "hec_precond_get_factor": ([_vp, _i32, C.POINTER(_i32), _vp, _vp, _vp, _vp], C.c_int),
    "hec_precond_get_levels": ([_vp, _i32, _i32, C.POINTER(_i32), _vp, _vp], C.c_int),
    "hec_precond_get_layout": ([_vp, _i32, C.POINTER(_i64), C.POINTER(_i32), C.POINTER(_i32),
                                C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32), _vp, _vp, _vp,
                                _vp], C.c_int),
    "hec_precond_set_trsv_parts": ([_vp, _i32], C.c_int),
    "hec_precond_set_trsv_kernel": ([_vp, _i32], C.c_int),
    "hec_debug_record": ([_vp, _i32], C.c_int),
    "hec_precond_apply": ([_vp, _vp, _vp, _i64, _vp], C.c_int),
    "hec_precond_status": ([_vp, _vp], C.c_int),
    "hec_precond_apply_noalloc": ([_vp, _vp, _vp, _i64, _vp], C.c_int),
    "hec_precond_apply_f32": ([_vp, _vp, _vp, _i64, _vp], C.c_int),
    "hec_precond_destroy": ([_vp], None),
    "krylov_solve": ([_vp, _vp, _vp, _vp, _dbl, _i32, _i32, C.POINTER(SolveOpts_t), _vp,
                      C.POINTER(SolveInfo_t)], C.c_int),
    "hec_workspace_bytes": ([_vp, _vp, _i32, C.POINTER(SolveOpts_t), C.POINTER(_i64)], C.c_int),
    "hec_build_batched": ([C.POINTER(BatchCSR_t), C.POINTER(BatchConfig_t), _vp, C.POINTER(_vp)],
                          C.c_int),
    "ilu_k_setup_batched": ([_vp, _i32], C.c_int),
    "hec_batch_info": ([_vp, C.POINTER(BatchInfo_t)], C.c_int),
    "hec_batch_set_config": ([_vp, C.POINTER(BatchConfig_t)], C.c_int),
    "hec_batch_autotune": ([_vp, _i32, _i32, C.POINTER(SolveOpts_t), _vp, C.POINTER(BatchConfig_t)],
                           C.c_int),
    "krylov_solve_batched": ([_vp, _vp, _vp, _i32, _dbl, _i32, _i32, C.POINTER(SolveOpts_t), _vp,
                              C.POINTER(SolveInfo_t), _vp], C.c_int),
    "hec_batch_apply": ([_vp, _i32, _vp, _vp, _i32, _vp], C.c_int),
    "hec_batch_destroy": ([_vp], None),
    "hec_server_create": ([C.POINTER(ServerOpts_t), C.POINTER(_vp)], C.c_int),
    "hec_server_submit": ([_vp, C.POINTER(Request_t), C.POINTER(C.c_uint64)], C.c_int),
    "hec_server_poll": ([_vp, _vp, _i32, C.POINTER(_i32), _i32], C.c_int),
    "hec_server_solution": ([_vp, C.c_uint64, _vp, _i32], C.c_int),
    "hec_server_clock": ([_vp], C.c_double),
    "hec_server_stats": ([_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32),
                          C.POINTER(_i64)], C.c_int),
    "hec_server_destroy": ([_vp], None),
}

_lock = threading.Lock()
_lib = None
_alloc_keep = []


def load_library(path: str = LIB_PATH):
    """Load the CUDA library and declare every ABI signature."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError("CUDA library %s is missing: run __graft_entry__.build()" % path)
            lib = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc, where, ok=(OK,)):
    if rc not in ok:
        raise HecError(rc, where, _lib.hec_last_error().decode(errors="replace"))
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return C.c_void_p(t.ctypes.data)
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, int):
        return C.c_void_p(t)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(t))


def use_torch_allocator():
    """Route every device allocation of the library through torch's caching allocator."""
    import torch
    lib = load_library()
    AF = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    FF = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # the library reports HEC_ERR_OOM
            return None

    def _free(p, stream, ctx):
        torch.cuda.caching_allocator_delete(int(p))

    fa, ff = AF(_alloc), FF(_free)
    _alloc_keep[:] = [fa, ff]
    _check(lib.hec_set_allocator(C.cast(fa, C.c_void_p), C.cast(ff, C.c_void_p), None),
           "hec_set_allocator")


def use_cuda_allocator():
    _check(load_library().hec_set_allocator(None, None, None), "hec_set_allocator")


# ------------------------------------------------------------------ matrix
class Matrix:
    """An HEC matrix handle (Section 2.1)."""

    def __init__(self, handle, n, nnz):
        self._h = handle
        self.n = n
        self.nnz = nnz

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = MatrixInfo_t()
        _check(_lib.hec_matrix_info(self._h, C.byref(inf)), "hec_matrix_info")
        return {f: getattr(inf, f) for f, _ in MatrixInfo_t._fields_}

    def export(self):
        """Host copies of the ELL slab and CSR tail."""
        inf = self.info()
        K, ld, nt, tn = inf["ell_width"], inf["ell_ld"], inf["tail_rows"], inf["tail_nnz"]
        ec = np.zeros(K * ld, np.int32)
        ev = np.zeros(K * ld, np.float64)
        tr = np.zeros(nt, np.int32)
        tp = np.zeros(nt + 1, np.int32)
        tc = np.zeros(tn, np.int32)
        tv = np.zeros(tn, np.float64)
        _check(_lib.hec_matrix_export(self._h, _ptr(ec), _ptr(ev), _ptr(tr), _ptr(tp), _ptr(tc),
                                      _ptr(tv)), "hec_matrix_export")
        return dict(K=K, ld=ld, ell_col=ec.reshape(K, ld), ell_val=ev.reshape(K, ld),
                    tail_rows=tr, tail_ptr=tp, tail_col=tc, tail_val=tv)

    def destroy(self):
        if self._h and _lib is not None:
            _lib.hec_matrix_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hec_build(row_ptr, col, val, ell_width=0, ell_ld_align=0, host_only=False, stream=None):
    """Section 2.1: CSR (numpy host arrays or torch device tensors) -> HEC matrix."""
    lib = load_library()
    on_dev = hasattr(row_ptr, "data_ptr")
    if not on_dev:
        row_ptr = np.ascontiguousarray(row_ptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
    n = int(row_ptr.shape[0] - 1)
    nnz = int(col.shape[0])
    A = CSR_t(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(val), 1 if on_dev else 0)
    o = Opts_t(int(ell_width), int(ell_ld_align), HOST_ONLY if host_only else 0, 0)
    h = C.c_void_p()
    st = C.c_void_p(0) if host_only else _stream(stream)
    _check(lib.hec_build(C.byref(A), C.byref(o), st, C.byref(h)), "hec_build")
    return Matrix(h, n, nnz)


def hec_spmv(A: Matrix, alpha, x, beta, y_in, y_out, w=None, dots=None, stream=None):
    """Eq. 2: y_out = alpha A x + beta y_in, optional fused dots (see the header)."""
    _check(load_library().hec_spmv(A.handle, float(alpha), _ptr(x), float(beta), _ptr(y_in),
                                   _ptr(y_out), _ptr(w), _ptr(dots), _stream(stream)), "hec_spmv")


def hec_spmv_f32(A: Matrix, alpha, x, beta, y_in, y_out, stream=None):
    """FP32 SpMV of the mixed-precision inner solves (float32 tensors)."""
    _check(load_library().hec_spmv_f32(A.handle, float(alpha), _ptr(x), float(beta), _ptr(y_in),
                                       _ptr(y_out), _stream(stream)), "hec_spmv_f32")


def hec_axpby(a, x, b, y, stream=None):
    _check(load_library().hec_axpby(int(y.numel()), float(a), _ptr(x), float(b), _ptr(y),
                                    _stream(stream)), "hec_axpby")


def hec_waxpby(a, x, b, y, z, stream=None):
    _check(load_library().hec_waxpby(int(z.numel()), float(a), _ptr(x), float(b), _ptr(y),
                                     _ptr(z), _stream(stream)), "hec_waxpby")


def hec_dot(x, y, result, stream=None):
    _check(load_library().hec_dot(int(x.numel()), _ptr(x), _ptr(y), _ptr(result),
                                  _stream(stream)), "hec_dot")


def hec_nrm2(x, result, stream=None):
    _check(load_library().hec_nrm2(int(x.numel()), _ptr(x), _ptr(result), _stream(stream)),
           "hec_nrm2")


def hec_multidot(n, k, V, ldv, w, h, stream=None):
    _check(load_library().hec_multidot(int(n), int(k), _ptr(V), int(ldv), _ptr(w), _ptr(h),
                                       _stream(stream)), "hec_multidot")


# ------------------------------------------------------------------ preconditioner
class Precond:
    """RAS blocks with ILU(k) factors (Sections 2.4-2.6)."""

    def __init__(self, handle, A):
        self._h = handle
        self.A = A  # keeps the matrix alive

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = PrecondInfo_t()
        _check(_lib.hec_precond_info(self._h, C.byref(inf)), "hec_precond_info")
        return {f: getattr(inf, f) for f, _ in PrecondInfo_t._fields_}

    def block(self, b):
        """(rows of V_b, own_lo, own_hi)."""
        nv, lo, hi = _i32(), _i32(), _i32()
        _check(_lib.hec_precond_get_block(self._h, b, C.byref(nv), C.byref(lo), C.byref(hi), None),
               "hec_precond_get_block")
        rows = np.zeros(nv.value, np.int32)
        _check(_lib.hec_precond_get_block(self._h, b, None, None, None, _ptr(rows)),
               "hec_precond_get_block")
        return rows, lo.value, hi.value

    def factor(self, b):
        """Combined ILU(k) factor of block b: (row_ptr, col, val, lev), local indices."""
        nnz = _i32()
        _check(_lib.hec_precond_get_factor(self._h, b, C.byref(nnz), None, None, None, None),
               "hec_precond_get_factor")
        nv = self.block(b)[0].shape[0]
        rp = np.zeros(nv + 1, np.int32)
        ci = np.zeros(nnz.value, np.int32)
        va = np.zeros(nnz.value, np.float64)
        lev = np.zeros(nnz.value, np.int32)
        _check(_lib.hec_precond_get_factor(self._h, b, C.byref(nnz), _ptr(rp), _ptr(ci), _ptr(va),
                                           _ptr(lev)), "hec_precond_get_factor")
        return rp, ci, va, lev

    def levels(self, b, which):
        """Level sets of L_b (which=FACTOR_L) or U_b: (level_ptr, level_rows)."""
        nlev = _i32()
        _check(_lib.hec_precond_get_levels(self._h, b, which, C.byref(nlev), None, None),
               "hec_precond_get_levels")
        nv = self.block(b)[0].shape[0]
        ptr = np.zeros(nlev.value + 1, np.int32)
        rows = np.zeros(nv, np.int32)
        _check(_lib.hec_precond_get_levels(self._h, b, which, C.byref(nlev), _ptr(ptr), _ptr(rows)),
               "hec_precond_get_levels")
        return ptr, rows

    def layout(self, fp32=False, stream=None):
        """The triangular solves' level-major chunk layout, host copies:
        dict(pack=uint8 bytes, chunks=(nchunks, 2) uint32 {offset/16, bytes},
        programs=(nblocks * parts, 8) int64, ring_slots, import_slots, parts,
        fixed_width, vbytes)."""
        nb, nc, ring, imp, parts, fw = _i64(), _i32(), _i32(), _i32(), _i32(), _i32()
        st = C.c_void_p(0) if self.A is not None and _is_host_only(self) else _stream(stream)

        def call(*arrays):
            _check(_lib.hec_precond_get_layout(self._h, int(bool(fp32)), C.byref(nb), C.byref(nc),
                                               C.byref(ring), C.byref(imp), C.byref(parts),
                                               C.byref(fw), *arrays, st), "hec_precond_get_layout")
        call(None, None, None)
        pack = np.zeros(nb.value, np.uint8)
        chunks = np.zeros((nc.value, 2), np.uint32)
        programs = np.zeros((self.info()["nblocks"] * parts.value, 8), np.int64)
        call(_ptr(pack), _ptr(chunks), _ptr(programs))
        return {"pack": pack, "chunks": chunks, "programs": programs, "ring_slots": ring.value,
                "import_slots": imp.value, "parts": parts.value, "fixed_width": fw.value,
                "vbytes": 4 if fp32 else 8}

    def destroy(self):
        if self._h and _lib is not None:
            _lib.hec_precond_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hec_refactor(A: Matrix, M, val, stream=None):
    """Same pattern, new values (numpy array or torch tensor in A's CSR
    order): A and, if given, its preconditioner are refactored on the GPU."""
    if not hasattr(val, "data_ptr"):
        val = np.ascontiguousarray(val, np.float64)
    _check(load_library().hec_refactor(A.handle, M.handle if M is not None else None, _ptr(val),
                                       _stream(stream)), "hec_refactor")


def jacobi_setup(A: Matrix, omega: float = 1.0, stream=None) -> Precond:
    """Damped Jacobi z = omega D^{-1} r as a preconditioner handle."""
    h = C.c_void_p()
    _check(load_library().hec_jacobi_setup(A.handle, float(omega), _stream(stream), C.byref(h)),
           "hec_jacobi_setup")
    return Precond(h, A)


def ilu_k_setup(A: Matrix, k: int, nblocks: int, overlap: int, stream=None) -> Precond:
    h = C.c_void_p()
    _check(load_library().ilu_k_setup(A.handle, int(k), int(nblocks), int(overlap), None,
                                      C.byref(h)), "ilu_k_setup")
    return Precond(h, A)


def level_schedule(M: Precond, stream=None, parts: int = 0, kernel: int = 0):
    """Eq. 11 level sets and the triangular-solve layout.  parts: CTAs per
    RAS block of the triangular solve (0: automatic; 1, 2, 4 or 8).  kernel:
    TRSV_AUTO, TRSV_STREAMED or TRSV_RESIDENT."""
    if kernel:
        _check(load_library().hec_precond_set_trsv_kernel(M.handle, int(kernel)),
               "hec_precond_set_trsv_kernel")
    if parts:
        _check(load_library().hec_precond_set_trsv_parts(M.handle, int(parts)),
               "hec_precond_set_trsv_parts")
    st = C.c_void_p(0) if M.A is not None and _is_host_only(M) else _stream(stream)
    _check(load_library().level_schedule(M.handle, st), "level_schedule")


def _is_host_only(M):
    return M.A.info()["device_bytes"] == 0


def hec_precond_apply(M: Precond, r, z, spin_limit: int = 0, stream=None):
    _check(load_library().hec_precond_apply(M.handle, _ptr(r), _ptr(z), int(spin_limit),
                                            _stream(stream)), "hec_precond_apply")


def hec_precond_apply_noalloc(M: Precond, r, z, spin_limit: int = 0, stream=None):
    """z = M^{-1} r without any device allocation (for callers with a fixed
    device-memory budget or that must avoid cudaMalloc's implicit
    synchronisation); scratch is a static 8 MiB array in the library, shared
    by all calls, so overlapping calls race."""
    _check(load_library().hec_precond_apply_noalloc(M.handle, _ptr(r), _ptr(z), int(spin_limit),
                                                    _stream(stream)), "hec_precond_apply_noalloc")


def hec_precond_apply_f32(M: Precond, r, z, spin_limit: int = 0, stream=None):
    """FP32 preconditioner apply of the mixed-precision inner solves (float32 tensors)."""
    _check(load_library().hec_precond_apply_f32(M.handle, _ptr(r), _ptr(z), int(spin_limit),
                                                _stream(stream)), "hec_precond_apply_f32")


def hec_precond_status(M: Precond, stream=None) -> int:
    return load_library().hec_precond_status(M.handle, _stream(stream))


# ------------------------------------------------------------------ Krylov
def krylov_solve(A: Matrix, M, b, x, tol=1e-8, maxit=1000, restart=30, method=GMRES, flags=0,
                 spin_limit=0, stream=None):
    """Section 2.7.  Returns a dict of hec_solve_info_t; raises on errors
    (HEC_MAXIT / HEC_BREAKDOWN are returned in info['status'])."""
    o = SolveOpts_t(int(method), int(flags), int(spin_limit))
    inf = SolveInfo_t()
    rc = load_library().krylov_solve(A.handle, M.handle if M is not None else None, _ptr(b), _ptr(x),
                                     float(tol), int(maxit), int(restart), C.byref(o),
                                     _stream(stream), C.byref(inf))
    _check(rc, "krylov_solve", ok=(OK, MAXIT, BREAKDOWN))
    return {f: getattr(inf, f) for f, _ in SolveInfo_t._fields_ if f != "reserved"}


def hec_workspace_bytes(A: Matrix, M, restart=30, method=GMRES, flags=0) -> int:
    """Device bytes the first krylov_solve with these arguments allocates
    beyond what the handles hold (0 once such a solve has run)."""
    o = SolveOpts_t(int(method), int(flags), 0)
    nb = _i64()
    _check(load_library().hec_workspace_bytes(A.handle, M.handle if M is not None else None,
                                              int(restart), C.byref(o), C.byref(nb)),
           "hec_workspace_bytes")
    return nb.value


# ------------------------------------------------------------------ batches
BATCH_SPMV64 = 0
BATCH_SPMV32 = 1
BATCH_PRECOND32 = 2
BATCH_PRECOND64 = 3


def _cfg_dict(c):
    return {f: getattr(c, f) for f, _ in BatchConfig_t._fields_}


class Batch:
    """A batch of independent systems solved by one persistent launch."""

    def __init__(self, handle, sys_ptr):
        self._h = handle
        self.sys_ptr = sys_ptr
        self.nsys = len(sys_ptr) - 1
        self.rows = int(sys_ptr[-1])

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = BatchInfo_t()
        _check(_lib.hec_batch_info(self._h, C.byref(inf)), "hec_batch_info")
        d = {f: getattr(inf, f) for f, _ in BatchInfo_t._fields_ if f != "config"}
        d["config"] = _cfg_dict(inf.config)
        return d

    def set_config(self, threads=0, ctas_per_sm=0, ell_width=0, nstages=0):
        c = BatchConfig_t(int(threads), int(ctas_per_sm), int(ell_width), int(nstages))
        _check(_lib.hec_batch_set_config(self._h, C.byref(c)), "hec_batch_set_config")

    def destroy(self):
        if self._h and _lib is not None:
            _lib.hec_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hec_build_batched(systems, threads=0, ctas_per_sm=0, ell_width=0, nstages=0, stream=None):
    """systems: a list of CSR matrices (objects with row_ptr, col, val) or a
    tuple (sys_ptr, row_ptr, col, val) of the concatenated form."""
    lib = load_library()
    if isinstance(systems, tuple):
        sp, rp, ci, va = systems
        sp = np.ascontiguousarray(sp, np.int64)
        rp = np.ascontiguousarray(rp, np.int64)
        ci = np.ascontiguousarray(ci, np.int32)
        va = np.ascontiguousarray(va, np.float64)
    else:
        ns = [int(len(A.row_ptr) - 1) for A in systems]
        sp = np.zeros(len(systems) + 1, np.int64)
        sp[1:] = np.cumsum(ns)
        nnz = [int(A.row_ptr[-1]) for A in systems]
        off = np.concatenate([[0], np.cumsum(nnz)]).astype(np.int64)
        rp = np.concatenate([np.asarray(A.row_ptr[:-1], np.int64) + off[i]
                             for i, A in enumerate(systems)] + [[off[-1]]]).astype(np.int64)
        ci = np.ascontiguousarray(np.concatenate([np.asarray(A.col) for A in systems]), np.int32)
        va = np.ascontiguousarray(np.concatenate([np.asarray(A.val) for A in systems]), np.float64)
    csr = BatchCSR_t(len(sp) - 1, 0, sp.ctypes.data, rp.ctypes.data, ci.ctypes.data, va.ctypes.data)
    c = BatchConfig_t(int(threads), int(ctas_per_sm), int(ell_width), int(nstages))
    h = C.c_void_p()
    _check(lib.hec_build_batched(C.byref(csr), C.byref(c), _stream(stream), C.byref(h)),
           "hec_build_batched")
    return Batch(h, sp)


def ilu_k_setup_batched(B: Batch, k: int):
    _check(load_library().ilu_k_setup_batched(B.handle, int(k)), "ilu_k_setup_batched")


def hec_batch_autotune(B: Batch, nrhs=1, restart=30, flags=0, stream=None):
    o = SolveOpts_t(GMRES, int(flags), 0)
    c = BatchConfig_t()
    _check(load_library().hec_batch_autotune(B.handle, int(nrhs), int(restart), C.byref(o),
                                             _stream(stream), C.byref(c)), "hec_batch_autotune")
    return _cfg_dict(c)


def krylov_solve_batched(B: Batch, b, x, nrhs=1, tol=1e-8, maxit=1000, restart=30, flags=0,
                         spin_limit=0, stream=None, per_system=False):
    """Returns the summary dict (and, with per_system, a list of per-system dicts)."""
    o = SolveOpts_t(GMRES, int(flags), int(spin_limit))
    inf = SolveInfo_t()
    si = (BatchSysInfo_t * B.nsys)() if per_system else None
    rc = load_library().krylov_solve_batched(B.handle, _ptr(b), _ptr(x), int(nrhs), float(tol),
                                             int(maxit), int(restart), C.byref(o),
                                             _stream(stream), C.byref(inf),
                                             C.cast(si, C.c_void_p) if si is not None else None)
    _check(rc, "krylov_solve_batched", ok=(OK, MAXIT, BREAKDOWN))
    summary = {f: getattr(inf, f) for f, _ in SolveInfo_t._fields_ if f != "reserved"}
    if not per_system:
        return summary
    return summary, [{f: getattr(v, f) for f, _ in BatchSysInfo_t._fields_ if f != "reserved"}
                     for v in si]


def hec_batch_apply(B: Batch, op, b, x, nrhs=1, stream=None):
    _check(load_library().hec_batch_apply(B.handle, int(op), _ptr(b), _ptr(x), int(nrhs),
                                          _stream(stream)), "hec_batch_apply")


# ------------------------------------------------------------------ serving
class Server:
    """The solve server (continuous batching over lanes of CUDA streams)."""

    def __init__(self, device_budget=0, lanes=0, restart=0, maxit=0, flags=0, tol=0.0,
                 small_rows=0, block_rows=0, keep_solutions=True):
        lib = load_library()
        o = ServerOpts_t(int(device_budget), int(lanes), int(restart), int(maxit), int(flags),
                         float(tol), int(small_rows), int(block_rows), int(bool(keep_solutions)), 0)
        h = C.c_void_p()
        _check(lib.hec_server_create(C.byref(o), C.byref(h)), "hec_server_create")
        self._h = h

    def submit(self, A, b, ilu_k=0, key=0, tag=0):
        """A: a CSR matrix, or None to solve with the system resident under key."""
        bb = np.ascontiguousarray(b, np.float64)
        if A is None:
            csr = CSR_t(len(bb), 0, None, None, None, 0)
        else:
            rp = np.ascontiguousarray(A.row_ptr, np.int32)
            ci = np.ascontiguousarray(A.col, np.int32)
            va = np.ascontiguousarray(A.val, np.float64)
            csr = CSR_t(len(rp) - 1, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0)
        req = Request_t(csr, bb.ctypes.data, int(ilu_k), 0, int(key), int(tag))
        t = C.c_uint64()
        _check(_lib.hec_server_submit(self._h, C.byref(req), C.byref(t)), "hec_server_submit")
        return t.value

    def poll(self, max_results=256, wait_ms=0):
        buf = (Result_t * max_results)()
        cnt = C.c_int32()
        _check(_lib.hec_server_poll(self._h, C.cast(buf, C.c_void_p), int(max_results),
                                    C.byref(cnt), int(wait_ms)), "hec_server_poll")
        return [{f: getattr(buf[i], f) for f, _ in Result_t._fields_} for i in range(cnt.value)]

    def solution(self, ticket, n):
        x = np.empty(n, np.float64)
        _check(_lib.hec_server_solution(self._h, int(ticket), x.ctypes.data, int(n)),
               "hec_server_solution")
        return x

    def clock(self):
        return _lib.hec_server_clock(self._h)

    def stats(self):
        q, r, f = C.c_int32(), C.c_int32(), C.c_int32()
        b = C.c_int64()
        _check(_lib.hec_server_stats(self._h, C.byref(q), C.byref(r), C.byref(f), C.byref(b)),
               "hec_server_stats")
        return {"queued": q.value, "running": r.value, "finished": f.value, "reserved": b.value}

    def close(self):
        if self._h and _lib is not None:
            _lib.hec_server_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
